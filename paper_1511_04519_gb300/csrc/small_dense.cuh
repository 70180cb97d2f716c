// Small dense linear algebra on m x m matrices in shared memory with leading
// dimension LD, executed cooperatively by all threads of one CTA: products, a
// pivoted Gaussian solve, the matrix exponential by scaling and squaring with
// the [13/13] Pade approximant (Higham 2005) and the rational Hessenberg map of
// Eq. 9.  Used for e^{h H_m} (LD = 20) and for Frechet derivatives through the
// 2m x 2m block exponential (LD = 40).
#pragma once
#include "kernels.h"

namespace matex {

constexpr int kSmallThreads = 128;
// theta_13 of Higham (2005), "The scaling and squaring method for the matrix
// exponential revisited", Table 2.3: the largest 1-norm for which the [13/13]
// Pade approximant reaches double-precision backward accuracy.
constexpr double kTheta13 = 5.371920351148152;

template <int LD>
struct Small {
  static constexpr int kLd = LD;
  static constexpr int kMat = LD * LD;

  struct Work {
    double A[kMat], A2[kMat], A4[kMat], A6[kMat], U[kMat], V[kMat], T[kMat];
    double b[14];
    double red[kSmallThreads];
    int piv;
    int s;
  };
  static __device__ void mat_mul(const double* A, const double* B, double* C, int m) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(A[i * kLd + k], B[k * kLd + j], s);
    C[i * kLd + j] = s;
  }
  __syncthreads();
}

// Solve Q X = P in place (X overwrites P), Gaussian elimination with partial
// pivoting; Q is destroyed.
  static __device__ void lu_solve(double* Q, double* P, int m, int* piv_sh) {
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(Q[k * kLd + k]);
      for (int i = k + 1; i < m; ++i) {
        const double a = fabs(Q[i * kLd + k]);
        if (a > best) { best = a; p = i; }
      }
      *piv_sh = p;
    }
    __syncthreads();
    const int p = *piv_sh;
    if (p != k) {
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double t = Q[k * kLd + c]; Q[k * kLd + c] = Q[p * kLd + c]; Q[p * kLd + c] = t;
        t = P[k * kLd + c]; P[k * kLd + c] = P[p * kLd + c]; P[p * kLd + c] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / Q[k * kLd + k];
    const int rows = m - k - 1;
    for (int e = threadIdx.x; e < rows * (2 * m - k); e += blockDim.x) {
      const int i = k + 1 + e / (2 * m - k);
      const int c = e % (2 * m - k);
      const double f = Q[i * kLd + k] * inv;
      if (c < m - k) {
        const int cc = k + c;
        if (cc > k) Q[i * kLd + cc] = fma(-f, Q[k * kLd + cc], Q[i * kLd + cc]);
      } else {
        const int cc = c - (m - k);
        P[i * kLd + cc] = fma(-f, P[k * kLd + cc], P[i * kLd + cc]);
      }
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) Q[i * kLd + k] = Q[i * kLd + k] * inv;
    __syncthreads();
  }
  // back substitution, one thread per right-hand-side column
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int k = m - 1; k >= 0; --k) {
      double s = P[k * kLd + c];
      for (int i = k + 1; i < m; ++i) s = fma(-Q[k * kLd + i], P[i * kLd + c], s);
      P[k * kLd + c] = s / Q[k * kLd + k];
    }
  }
  __syncthreads();
}


// E = expm(h * M) by scaling and squaring with the [13/13] Pade approximant
// (Higham 2005).  M and E may not alias work arrays; E may alias M.
  static __device__ void expm(const double* M, double h, double* E, int m, Work& w) {
  if (threadIdx.x == 0) {
    // Pade coefficients b_k = (26-k)! 13! / (26! k! (13-k)!), scaled to b_0 = 1
    w.b[0] = 1.0;
    for (int k = 0; k < 13; ++k) w.b[k + 1] = w.b[k] * (double)(13 - k) / ((double)(26 - k) * (k + 1));
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    w.A[i * kLd + j] = h * M[i * kLd + j];
  }
  __syncthreads();
  // 1-norm
  double cs = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += fabs(w.A[i * kLd + j]);
    cs = fmax(cs, t);
  }
  w.red[threadIdx.x] = cs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) nrm = fmax(nrm, w.red[i]);
    int s = 0;
    if (nrm > kTheta13) {
      // bounded even for an infinite norm: 2^-1074 scales any finite matrix to zero
      const double l = ceil(log2(nrm / kTheta13));
      s = l < 1074.0 ? (int)l : 1074;
    }
    w.s = s > 0 ? s : 0;
  }
  __syncthreads();
  const double sc = ldexp(1.0, -w.s);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    w.A[i * kLd + j] *= sc;
  }
  __syncthreads();
  mat_mul(w.A, w.A, w.A2, m);
  mat_mul(w.A2, w.A2, w.A4, m);
  mat_mul(w.A4, w.A2, w.A6, m);
  const double* b = w.b;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    w.U[x] = b[13] * w.A6[x] + b[11] * w.A4[x] + b[9] * w.A2[x];
    w.V[x] = b[12] * w.A6[x] + b[10] * w.A4[x] + b[8] * w.A2[x];
  }
  __syncthreads();
  mat_mul(w.A6, w.U, w.T, m);  // T = A6 * (b13 A6 + b11 A4 + b9 A2)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    w.T[x] += b[7] * w.A6[x] + b[5] * w.A4[x] + b[3] * w.A2[x] + (i == j ? b[1] : 0.0);
  }
  __syncthreads();
  mat_mul(w.A, w.T, w.U, m);  // U = A * (...)
  mat_mul(w.A6, w.V, w.T, m);  // T = A6 * (b12 A6 + b10 A4 + b8 A2)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    const double vv = w.T[x] + b[6] * w.A6[x] + b[4] * w.A4[x] + b[2] * w.A2[x] + (i == j ? b[0] : 0.0);
    w.V[x] = vv - w.U[x];  // Q = V - U
    w.T[x] = vv + w.U[x];  // P = V + U
  }
  __syncthreads();
  lu_solve(w.V, w.T, m, &w.piv);  // T = Q^{-1} P
  double* cur = w.T;
  double* nxt = w.A2;
  for (int k = 0; k < w.s; ++k) {
    mat_mul(cur, cur, nxt, m);
    double* t = cur; cur = nxt; nxt = t;
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    E[i * kLd + j] = cur[i * kLd + j];
  }
  __syncthreads();
}

// The exponent matrix of the Krylov space from its Arnoldi Hessenberg Ht (the
// column's kMaxB x kMaxM array): variant 0 rational, H = (I - Ht_m^{-1}) / gamma
// (Eq. 9); 1 inverted, H = -Ht_m^{-1} (the Arnoldi of G^{-1} C = -A^{-1},
// Sec. 3.3.1); 2 standard, H = Ht_m (the Arnoldi of A, Sec. 2.3).
  static __device__ void rational_H(const double* Ht, int m, double gamma, double* H, Work& w,
                                    int variant = 0) {
  if (variant == 2) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = Ht[i * kMaxM + j];
    }
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    w.V[i * kLd + j] = Ht[i * kMaxM + j];
    w.T[i * kLd + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  lu_solve(w.V, w.T, m, &w.piv);  // T = Ht_m^{-1}
  if (variant == 1) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = -w.T[i * kLd + j];
    }
  } else {
    const double ig = 1.0 / gamma;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = ((i == j ? 1.0 : 0.0) - w.T[i * kLd + j]) * ig;
    }
  }
  __syncthreads();
}

};

}  // namespace matex
