// Internal declarations shared by the host setup and the CUDA translation
// units of the R-MATEX library.  Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace matex {

// Symmetric sparse matrix in CSR (both triangles), original numbering.
struct CsrSym {
  int64_t n = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
};

// Supernodal structure of L for a fill-reducing, post-ordered permutation.
// Supernode s owns columns [sup_first[s], sup_first[s+1]) (new numbering).
// Its row list R_s = sup_rows[sup_rowptr[s] .. sup_rowptr[s+1]) starts with
// its own w_s columns, followed by the r_s off-diagonal rows (ascending).
struct Symbolic {
  int64_t n = 0;
  std::vector<int32_t> perm;        // new -> old
  std::vector<int32_t> iperm;       // old -> new
  int32_t nsup = 0;
  std::vector<int32_t> sup_first;   // nsup+1
  std::vector<int64_t> sup_rowptr;  // nsup+1
  std::vector<int32_t> sup_rows;
  std::vector<int32_t> sup_parent;  // -1 for roots
  std::vector<int64_t> pan_off;     // nsup+1, offsets of the (w+r) x w solve panels
  std::vector<int32_t> level_ptr;   // levels of the supernodal tree, leaves first
  std::vector<int32_t> level_sups;
  int64_t nnz_L = 0;                // strictly lower entries of the dense panels (after
                                    // relaxed amalgamation, explicit zeros included)
  int64_t nnz_L_exact = 0;          // strictly lower nonzeros of L itself for this ordering
                                    // (column counts before any amalgamation)
  double flops_factor = 0.0;
};

// M = L D L^T on the symbolic structure (L unit lower).  What the solves read
// per supernode s is the panel P_s = [L_ss^{-1}; L_Rs L_ss^{-1}] ((w+r) x w):
//   forward   y_s = L_ss^{-1} b_s and b_R -= L_Rs y_s  are  P_s b_s,
//   backward  x_s = L_ss^{-T} (D_s^{-1} y_s - L_Rs^T x_R)  is  P_s^T [D_s^{-1} y_s; -x_R],
// so neither direction has a sequential step inside a supernode.  P_s is
// stored column-major (forward reads) and row-major (backward reads).
struct Numeric {
  std::vector<double> dinv;         // n, 1/D in new numbering
  std::vector<double> pan_cm, pan_rm;
};

// Host setup (host_symbolic.cpp / host_numeric.cpp).  Both return an empty
// string on success, else a message.
std::string nested_dissection(const CsrSym& A, std::vector<int32_t>& perm);
std::string symbolic_analysis(const CsrSym& A, const std::vector<int32_t>& nd_perm,
                              int32_t max_width, Symbolic& S);
// Factor diag(dshift) + alpha*A; dshift may be null (then just alpha*A).
std::string numeric_ldlt(const CsrSym& A, const double* dshift, double alpha,
                         const Symbolic& S, Numeric& F);

}  // namespace matex
