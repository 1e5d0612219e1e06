// Block elimination for the reduced projected Newton system (Section 3.3,
// eq. reduced_kkt_system and the block-elimination paragraph after it).
//
// The system K x = b (N x N, row-major FP64) has unknowns [dX; dl] (dX: n
// entries, dl: the nm = N - n multiplier entries) and equations [m; c]:
//   E dX + F dl = b_m      (the multiplier rows: primal, inequality)
//   LZ dX + G dl = b_c     (the last n rows: complementarity)
// with LZ = W^T L_Z W symmetric positive definite while Z is. With the
// Cholesky factor LZ = U^T U, W = U^-T E^T and V = U^-T G, the multipliers
// solve (F - W^T V) dl = b_m - E LZ^-1 b_c, and dX = LZ^-1 (b_c - G dl).
#pragma once

#include "common.cuh"

namespace ttsdp {

// Factors of one reduced system in the element type T (double, or float for
// the reduced-precision solves whose refinement runs in FP64).
template <typename T>
struct KktFactors {
  int N = 0, n = 0, nm = 0;
  DBuf<T> lz;      // LZ = U^T U in the layout lu_solve_factored reads (identity interchanges)
  DBuf<T> s;       // LU factors of the Schur complement F - W^T V
  DBuf<int> ipiv;  // its interchanges
  DBuf<int> perm;  // composed (lu_perm)
  DBuf<int> ident; // 0, 1, ..., n-1
  DBuf<T> lz_dinv, s_dinv;  // diagonal-block inverses of both (lu_diag_inverses)
};

// Factors K (kept). Returns false when the symmetric part of the LZ block is
// not numerically positive definite (a pivot <= 0 or not finite); the caller
// then solves the whole system by LU.
template <typename T>
bool kkt_factor(int N, int n, const double* K, KktFactors<T>& f, cudaStream_t st);

// x = K^-1 b with the factors (b and x FP64 device vectors of N entries, not
// aliased; K the FP64 matrix the factors came from).
template <typename T>
void kkt_apply(const KktFactors<T>& f, const double* K, const double* b, double* x, cudaStream_t st);

// Reduction of the symmetric-definite pencil (D, M) of the step-length
// eigenproblems (Section 3.4) with the same bordered Cholesky, carrying D and
// I as right-hand sides: M_s = L L^T for the symmetric parts M_s, D_s of M,
// D (n x n row-major FP64), S = L^-1 D_s L^-T (n x n) and Linv = L^-1 (lower
// triangular, n x n row-major). Returns false when M_s is not numerically
// positive definite (S and Linv then unspecified).
bool chol_reduce(int n, const double* M, const double* D, double* S, double* Linv, cudaStream_t st);

// Algorithmic flops of one factorisation and of one application.
double kkt_factor_flops(int N, int n);
double kkt_apply_flops(int N, int n);

}  // namespace ttsdp
