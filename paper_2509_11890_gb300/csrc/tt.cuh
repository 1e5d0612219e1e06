// Device tensor trains and the TT arithmetic of Sections 2.3 and 3.3.
#pragma once

#include <memory>
#include <utility>
#include <vector>

#include "common.cuh"

namespace ttsdp {

// A tensor train with uniform modes (m x n per core; n = 1 for TT vectors),
// FP64 cores on the device, row-major [r_k][m][n][r_{k+1}]. Cores are shared
// pointers so reshaped views (vec_TT, unvec) cost nothing.
struct DTT {
  int d = 0, m = 1, n = 1;
  std::vector<int> r;
  std::vector<std::shared_ptr<DBuf<double>>> c;

  size_t csize(int k) const { return (size_t)r[k] * m * n * r[k + 1]; }
  size_t count() const {
    size_t s = 0;
    for (int k = 0; k < d; ++k) s += csize(k);
    return s;
  }
  double* core(int k) const { return c[k]->get(); }
  int maxrank() const {
    int x = 1;
    for (int v : r) x = v > x ? v : x;
    return x;
  }
  // same storage with another split of the per-core mode (m * n == m2 * n2)
  DTT view(int m2, int n2) const {
    DTT o = *this;
    o.m = m2;
    o.n = n2;
    return o;
  }
};

DTT tt_alloc(int d, const std::vector<int>& r, int m, int n);
DTT tt_from_host(int d, const int* ranks, int m, int n, const double* cores);
DTT tt_from_device(int d, const int* ranks, int m, int n, const double* cores);
void tt_to_host(const DTT& a, double* out);
void tt_to_device(const DTT& a, double* out);
DTT tt_copy(const DTT& a);
DTT tt_add(const DTT& a, const DTT& b, double alpha, double beta);
DTT tt_scale(const DTT& a, double s);
DTT tt_transpose(const DTT& a);                 // TT matrix: swap row / column modes
DTT tt_sym(const DTT& a);                       // (A + A^T) / 2
DTT tt_kron(const DTT& a, const DTT& b);        // Definition "Kronecker product of TT matrices"
DTT tt_hadamard(const DTT& a, const DTT& b);    // element-wise, ranks multiply
DTT tt_matvec(const DTT& op, const DTT& v);     // op (m x n) applied to v (mode n)
DTT tt_diag(const DTT& v);                      // Definition "TT Diagonalisation"
DTT tt_op_diag(const DTT& op);                  // the diagonal of a square TT matrix, as a TT vector
bool tt_is_diag_op(const DTT& op);              // all off-diagonal mode entries are zero
// Operator cores k, k+1 as one core [r_k][(i1 i2)][(j1 j2)][r_{k+2}] (modes m^2 x n^2)
std::shared_ptr<DBuf<double>> tt_merge_cores(const DTT& op, int k);
DTT tt_identity(int d, int m);                  // I_m kron ... kron I_m, rank 1
DTT tt_ones_mat(int d, int m);                  // J_m kron ... kron J_m, rank 1
DTT tt_zeros_like_modes(int d, int m, int n);   // rank-1 zero TT
double tt_inner(const DTT& a, const DTT& b);    // <a, b> over all entries
double tt_norm(const DTT& a);

// round_TT: right-to-left QR then left-to-right truncated SVD. Bond k keeps
// the smallest rank whose discarded energy is <= (delta / sqrt(d-1))^2, then
// at most cap (cap <= 0: none). Works on the vector view (m * n per core).
// Returns the rounded TT (same m, n) and zeta = sqrt(sum discarded sigma^2).
class RankPredictor;
struct Counter;

// Optional context of one rounding: features of the learned rank predictor,
// the predictor itself, trace collection and counters.
struct RoundHook {
  int var_id = 0;                      // 0 X, 1 Y, 2 T, 3 Z
  double mu = 1.0, iter_frac = 0.0;
  std::vector<int>* prev = nullptr;    // previous rounded ranks of this variable (d + 1), updated
  std::vector<float>* decay = nullptr; // singular-value decay per bond at the previous rounding (d + 1), updated
  const RankPredictor* pred = nullptr; // when set: fixed-rank randomised range finder per bond
  std::vector<float>* trace_x = nullptr;
  std::vector<float>* trace_y = nullptr;
  Counter* rnd = nullptr;              // sketch matrices
  long long used = 0, fallbacks = 0;
};

std::pair<DTT, double> tt_round(const DTT& a, double delta, int cap, RoundHook* hook = nullptr);

// TT-SVD (Oseledets 2011) of a dense n^d x n^d matrix given row-major on the
// device: the matrix is permuted to its vec_TT order (Section 3.1) and split
// by sequential truncated SVDs with per-bond threshold eps_rel ||M||_F / sqrt(d-1)
// and at most `cap` (<= 0: none). Returns a TT matrix with n x n modes.
DTT tt_from_dense(const double* dense, int d, int n, double eps_rel, int cap);

// right-to-left orthogonalisation (cores 1..d-1 right-orthonormal)
DTT tt_orth_right(const DTT& a);

// Host-side rank rule shared by rounding and AMEn truncation.
int truncation_rank(const std::vector<double>& s, double thr, int cap);

// SplitMix64 counter stream (Steele, Lea & Flood 2014): value j of a draw is
// splitmix64(seed ^ ((counter + j) * golden)) mapped to [-1, 1) by its top 53 bits.
struct Counter {
  uint64_t seed = 0, n = 0;
  std::vector<double> draw(size_t count);
  // a counter seeded by the raw 64-bit value of this stream's next draw (one
  // draw consumed): a sub-stream whose length does not move this one
  Counter fork();
};

// misc device helpers
void dev_fill(double* p, size_t n, double v, cudaStream_t st);
void dev_scale(double* p, size_t n, double s, cudaStream_t st);
void dev_axpy(double* y, const double* x, size_t n, double a, cudaStream_t st);  // y += a x
void dev_copy(double* dst, const double* src, size_t n, cudaStream_t st);
// dst (rows x dcols, ld dld) <- alpha * src (rows x cols, ld sld) at column offset
void dev_copy2d(double* dst, long long dld, const double* src, long long sld, int rows, int cols,
                double alpha, cudaStream_t st);
void dev_scale_rows(double* a, int rows, int cols, const double* s, cudaStream_t st);
void dev_scale_cols(double* a, int rows, int cols, const double* s, cudaStream_t st);
double dev_dot(const double* a, const double* b, size_t n, cudaStream_t st);
// *out (device) = a . b, left on the device (no host synchronisation)
void dev_dot_async(const double* a, const double* b, size_t n, double* out, cudaStream_t st);
// out[i] = <V_i, w> for the rows of a row-major nvec x N matrix (device output)
void dev_multi_dot(const double* V, int nvec, size_t N, const double* w, double* out, cudaStream_t st);

}  // namespace ttsdp
