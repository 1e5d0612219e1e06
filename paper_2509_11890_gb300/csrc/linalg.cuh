// Small dense factorisations used by TT rounding, the AMEn block-index move,
// the local solves and the step-length eigenproblems.
#pragma once

#include "common.cuh"

namespace ttsdp {

// Strided view of an m x n matrix: element (i, j) at p[i * rs + j * cs].
template <typename T>
struct MatView {
  const T* p;
  int m, n;
  long long rs, cs;
};

// Thin Householder QR of A (m x n): Q (m x k) and R (k x n), k = min(m, n),
// both written row-major and dense. Single CTA.
template <typename T>
void qr_thin(MatView<T> A, T* Q, T* R, cudaStream_t st);

// Thin SVD A = U diag(S) Vt by one-sided Jacobi (Hestenes), k = min(m, n),
// singular values descending; U (m x k), S (k), Vt (k x n) row-major.
// Single CTA. Returns nothing; the sweep count is bounded (60).
// Which singular vectors a caller reads: both, only U (left) or only Vt
// (right). With one side the Jacobi sweeps skip the other side's rotations
// when the requested side is the one they orthogonalise; the unrequested
// output is left unspecified.
enum SvdSide { kSvdBoth = 0, kSvdLeft = 1, kSvdRight = 2 };

template <typename T>
void svd_thin(MatView<T> A, T* U, T* S, T* Vt, cudaStream_t st, SvdSide side = kSvdBoth);

// While one is in scope on this thread, svd_thin treats a pair of columns
// whose squared norms are both below rel2 * ||A||_F^2 as converged (the
// default floor is the rounding noise, m eps^2 ||A||_F^2). A caller that
// truncates the spectrum at a relative level far above sqrt(rel2) keeps the
// subspace it keeps exact and gives up only the order of directions it drops
// anyway; the Jacobi sweeps then stop on clusters of such values.
struct SvdNoiseFloor {
  explicit SvdNoiseFloor(double rel2) : prev_(slot()) { slot() = rel2; }
  ~SvdNoiseFloor() { slot() = prev_; }
  SvdNoiseFloor(const SvdNoiseFloor&) = delete;
  SvdNoiseFloor& operator=(const SvdNoiseFloor&) = delete;
  static double current() { return slot(); }

 private:
  static double& slot();
  double prev_;
};

// Solves A x = b in place (A n x n row-major, destroyed; b n-vector becomes x)
// by LU with partial pivoting, right-looking and blocked (panel width 32).
template <typename T>
void lu_solve(int n, T* A, T* b, cudaStream_t st);

// The two halves of lu_solve: lu_factor overwrites the row-major A with the
// factors of its transpose (P A^T = L U with partial pivoting, stored
// column-major: the buffer read row-major holds L^T and U^T; interchanges in
// ipiv, n entries); lu_solve_factored then solves A x = b in place for one
// right-hand side and may be called any number of times on the same factors.
// Systems of 160 unknowns or more are solved by a cluster of eight CTAs in
// 64-row steps; perm (from lu_perm, or any array giving the final order when
// the interchanges are known otherwise) saves composing the interchanges on
// every call.
template <typename T>
void lu_factor(int n, T* A, int* ipiv, cudaStream_t st);
template <typename T>
void lu_solve_factored(int n, const T* LU, const int* ipiv, T* b, cudaStream_t st, const int* perm = nullptr,
                       const T* dinv = nullptr);
// The inverses of the 64 x 64 diagonal blocks of the factors that the
// cluster solves of lu_solve_factored use (dinv: lu_diag_inv_size(n)
// entries); computed once per factorisation they save one launch per solve.
size_t lu_diag_inv_size(int n);
template <typename T>
void lu_diag_inverses(int n, const T* LU, T* dinv, cudaStream_t st);
// perm[i] = the row of the solution of the permuted system that lands at
// position i: the interchanges ipiv of lu_factor composed (n <= 25600).
void lu_perm(int n, const int* ipiv, int* perm, cudaStream_t st);

// Lower Cholesky factor in place (row-major n x n; upper part zeroed) and
// the inverse of a lower triangular matrix in place. Single CTA.
template <typename T>
void cholesky_lower(int n, T* A, cudaStream_t st, int* nonpos = nullptr);  // *nonpos = 1 on a pivot <= 0
template <typename T>
void tri_lower_inverse(int n, T* L, cudaStream_t st);

// y = x transposed copy: out (n x m) = in (m x n)^T, both row-major.
template <typename T>
void transpose(int m, int n, const T* in, T* out, cudaStream_t st);

}  // namespace ttsdp
