// Small dense linear algebra on m x m matrices in shared memory with leading
// dimension LD, executed cooperatively by a thread group (a CTA or one warp:
// the template parameter G): products, a pivoted Gaussian solve, the matrix
// exponential by scaling and squaring with the [13/13] Pade approximant
// (Higham 2005) and the rational Hessenberg map of Eq. 9.  Used for e^{h H_m} (LD = 20) and for Frechet derivatives through the
// 2m x 2m block exponential (LD = 40).
#pragma once
#include "kernels.h"

namespace matex {

constexpr int kSmallThreads = 128;
// theta_13 of Higham (2005), "The scaling and squaring method for the matrix
// exponential revisited", Table 2.3: the largest 1-norm for which the [13/13]
// Pade approximant reaches double-precision backward accuracy.
constexpr double kTheta13 = 5.371920351148152;

// Coefficients of the [13/13] Pade approximant of e^x, b_k = (26-k)! 13! /
// (26! k! (13-k)!), scaled to b_0 = 1: evaluated by the compiler.
struct Pade13 {
  double b[14];
};
__host__ __device__ constexpr Pade13 pade13_coefficients() {
  Pade13 r{};
  r.b[0] = 1.0;
  for (int k = 0; k < 13; ++k) r.b[k + 1] = r.b[k] * (double)(13 - k) / ((double)(26 - k) * (k + 1));
  return r;
}

// Work arrays of one exponential (shared memory)
template <int LD>
struct SmallWork {
  double A[LD * LD], A2[LD * LD], A4[LD * LD], A6[LD * LD], U[LD * LD], V[LD * LD], T[LD * LD];
  double red[kSmallThreads];
  int piv;
  int s;
};

// The threads that run the routines below together: a whole CTA, or one warp
// of it (the other warps do not take part and must not touch the work arrays).
struct CtaGroup {
  static __device__ __forceinline__ int rank() { return threadIdx.x; }
  static __device__ __forceinline__ int size() { return blockDim.x; }
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};
struct WarpGroup {
  static __device__ __forceinline__ int rank() { return threadIdx.x & 31; }
  static __device__ __forceinline__ int size() { return 32; }
  static __device__ __forceinline__ void sync() { __syncwarp(); }
};

template <int LD, class G = CtaGroup>
struct Small {
  static constexpr int kLd = LD;
  static constexpr int kMat = LD * LD;
  using Work = SmallWork<LD>;
  static __device__ void mat_mul(const double* A, const double* B, double* C, int m) {
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(A[i * kLd + k], B[k * kLd + j], s);
    C[i * kLd + j] = s;
  }
  G::sync();
}

// Solve Q X = P in place (X overwrites P), Gaussian elimination with partial
// pivoting; Q is destroyed.
  static __device__ void lu_solve(double* Q, double* P, int m, int* piv_sh) {
  for (int k = 0; k < m; ++k) {
    if (G::rank() == 0) {
      int p = k;
      double best = fabs(Q[k * kLd + k]);
      for (int i = k + 1; i < m; ++i) {
        const double a = fabs(Q[i * kLd + k]);
        if (a > best) { best = a; p = i; }
      }
      *piv_sh = p;
    }
    G::sync();
    const int p = *piv_sh;
    if (p != k) {
      for (int c = G::rank(); c < m; c += G::size()) {
        double t = Q[k * kLd + c]; Q[k * kLd + c] = Q[p * kLd + c]; Q[p * kLd + c] = t;
        t = P[k * kLd + c]; P[k * kLd + c] = P[p * kLd + c]; P[p * kLd + c] = t;
      }
    }
    G::sync();
    const double inv = 1.0 / Q[k * kLd + k];
    const int rows = m - k - 1;
    for (int e = G::rank(); e < rows * (2 * m - k); e += G::size()) {
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
    G::sync();
    for (int i = k + 1 + G::rank(); i < m; i += G::size()) Q[i * kLd + k] = Q[i * kLd + k] * inv;
    G::sync();
  }
  // back substitution, one thread per right-hand-side column
  for (int c = G::rank(); c < m; c += G::size()) {
    for (int k = m - 1; k >= 0; --k) {
      double s = P[k * kLd + c];
      for (int i = k + 1; i < m; ++i) s = fma(-Q[k * kLd + i], P[i * kLd + c], s);
      P[k * kLd + c] = s / Q[k * kLd + k];
    }
  }
  G::sync();
}


// E = expm(h * M) by scaling and squaring with the [13/13] Pade approximant
// (Higham 2005).  M and E may not alias work arrays; E may alias M.
  static __device__ void expm(const double* M, double h, double* E, int m, Work& w) {
  constexpr Pade13 pade = pade13_coefficients();
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m;
    w.A[i * kLd + j] = h * M[i * kLd + j];
  }
  G::sync();
  // 1-norm
  double cs = 0.0;
  for (int j = G::rank(); j < m; j += G::size()) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += fabs(w.A[i * kLd + j]);
    cs = fmax(cs, t);
  }
  // m <= 2 kMaxM < kSmallThreads: threads past the first kSmallThreads hold no column
  if (G::rank() < kSmallThreads) w.red[G::rank()] = cs;
  G::sync();
  if (G::rank() == 0) {
    double nrm = 0.0;
    // only threads below m hold a column
    const int nred = min(min(G::size(), kSmallThreads), m);
    for (int i = 0; i < nred; ++i) nrm = fmax(nrm, w.red[i]);
    int s = 0;
    if (nrm > kTheta13) {
      // bounded even for an infinite norm: 2^-1074 scales any finite matrix to zero
      const double l = ceil(log2(nrm / kTheta13));
      s = l < 1074.0 ? (int)l : 1074;
    }
    w.s = s > 0 ? s : 0;
  }
  G::sync();
  const double sc = ldexp(1.0, -w.s);
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m;
    w.A[i * kLd + j] *= sc;
  }
  G::sync();
  mat_mul(w.A, w.A, w.A2, m);
  mat_mul(w.A2, w.A2, w.A4, m);
  mat_mul(w.A4, w.A2, w.A6, m);
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    w.U[x] = pade.b[13] * w.A6[x] + pade.b[11] * w.A4[x] + pade.b[9] * w.A2[x];
    w.V[x] = pade.b[12] * w.A6[x] + pade.b[10] * w.A4[x] + pade.b[8] * w.A2[x];
  }
  G::sync();
  mat_mul(w.A6, w.U, w.T, m);  // T = A6 * (b13 A6 + b11 A4 + b9 A2)
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    w.T[x] += pade.b[7] * w.A6[x] + pade.b[5] * w.A4[x] + pade.b[3] * w.A2[x] +
              (i == j ? pade.b[1] : 0.0);
  }
  G::sync();
  mat_mul(w.A, w.T, w.U, m);  // U = A * (...)
  mat_mul(w.A6, w.V, w.T, m);  // T = A6 * (b12 A6 + b10 A4 + b8 A2)
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m, x = i * kLd + j;
    const double vv = w.T[x] + pade.b[6] * w.A6[x] + pade.b[4] * w.A4[x] + pade.b[2] * w.A2[x] +
                      (i == j ? pade.b[0] : 0.0);
    w.V[x] = vv - w.U[x];  // Q = V - U
    w.T[x] = vv + w.U[x];  // P = V + U
  }
  G::sync();
  lu_solve(w.V, w.T, m, &w.piv);  // T = Q^{-1} P
  double* cur = w.T;
  double* nxt = w.A2;
  for (int k = 0; k < w.s; ++k) {
    mat_mul(cur, cur, nxt, m);
    double* t = cur; cur = nxt; nxt = t;
  }
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m;
    E[i * kLd + j] = cur[i * kLd + j];
  }
  G::sync();
}

// The exponent matrix of the Krylov space from its Arnoldi Hessenberg Ht (the
// column's kMaxB x kMaxM array): variant 0 rational, H = (I - Ht_m^{-1}) / gamma
// (Eq. 9); 1 inverted, H = -Ht_m^{-1} (the Arnoldi of G^{-1} C = -A^{-1},
// Sec. 3.3.1); 2 standard, H = Ht_m (the Arnoldi of A, Sec. 2.3).
  static __device__ void rational_H(const double* Ht, int m, double gamma, double* H, Work& w,
                                    int variant = 0) {
  if (variant == 2) {
    for (int e = G::rank(); e < m * m; e += G::size()) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = Ht[i * kMaxM + j];
    }
    G::sync();
    return;
  }
  for (int e = G::rank(); e < m * m; e += G::size()) {
    const int i = e / m, j = e - i * m;
    w.V[i * kLd + j] = Ht[i * kMaxM + j];
    w.T[i * kLd + j] = (i == j) ? 1.0 : 0.0;
  }
  G::sync();
  lu_solve(w.V, w.T, m, &w.piv);  // T = Ht_m^{-1}
  if (variant == 1) {
    for (int e = G::rank(); e < m * m; e += G::size()) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = -w.T[i * kLd + j];
    }
  } else {
    const double ig = 1.0 / gamma;
    for (int e = G::rank(); e < m * m; e += G::size()) {
      const int i = e / m, j = e - i * m;
      H[i * kLd + j] = ((i == j ? 1.0 : 0.0) - w.T[i * kLd + j]) * ig;
    }
  }
  G::sync();
}

};

}  // namespace matex
