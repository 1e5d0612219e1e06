// Strided tensor-contraction GEMM: C[b][m][n] = alpha * sum_k A[b][m][k] B[b][k][n] + beta * C,
// where each of the combined indices b, m, n, k is a row-major product of up
// to four sub-indices, every sub-index with its own stride in each operand.
// This expresses every environment update, local product and projected-matrix
// assembly of the TT solver directly on the cores' natural layouts.
#pragma once

#include <initializer_list>
#include <utility>

#include "common.cuh"

namespace ttsdp {

constexpr int kMaxSub = 4;

struct IdxN {
  int nsub = 0;
  int ext[kMaxSub] = {1, 1, 1, 1};
  long long total() const {
    long long t = 1;
    for (int i = 0; i < nsub; ++i) t *= ext[i];
    return t;
  }
};

struct StrN {
  long long s[kMaxSub] = {0, 0, 0, 0};
};

struct GemmND {
  IdxN M, N, K, B;
  StrN aM, aK, aB;  // A strides along M, K, batch
  StrN bK, bN, bB;  // B strides along K, N, batch
  StrN cM, cN, cB;  // C strides along M, N, batch
};

// A combined index with its sub-extents and the strides of the (up to three)
// operands that carry it. Build with dim({ {ext, sA, sB, sC}, ... }).
struct SubDim {
  int ext;
  long long s0, s1;
};

inline void set_dim(IdxN& idx, StrN& first, StrN& second, std::initializer_list<SubDim> subs) {
  idx.nsub = 0;
  for (const SubDim& s : subs) {
    if (s.ext == 1) continue;  // unit extents carry no offset
    TT_CHECK(idx.nsub < kMaxSub, TT_E_INTERNAL, "gemm_nd: too many sub-indices");
    idx.ext[idx.nsub] = s.ext;
    first.s[idx.nsub] = s.s0;
    second.s[idx.nsub] = s.s1;
    ++idx.nsub;
  }
  if (idx.nsub == 0) {
    idx.nsub = 1;
    idx.ext[0] = 1;
    first.s[0] = 0;
    second.s[0] = 0;
  }
}

// Batch indices are carried by all three operands.
struct SubDim3 {
  int ext;
  long long sa, sb, sc;
};
inline void set_batch(GemmND& g, std::initializer_list<SubDim3> subs) {
  g.B.nsub = 0;
  for (const SubDim3& s : subs) {
    if (s.ext == 1) continue;
    TT_CHECK(g.B.nsub < kMaxSub, TT_E_INTERNAL, "gemm_nd: too many batch sub-indices");
    int i = g.B.nsub++;
    g.B.ext[i] = s.ext;
    g.aB.s[i] = s.sa;
    g.bB.s[i] = s.sb;
    g.cB.s[i] = s.sc;
  }
  if (g.B.nsub == 0) {
    g.B.nsub = 1;
    g.B.ext[0] = 1;
    g.aB.s[0] = g.bB.s[0] = g.cB.s[0] = 0;
  }
}

// nA, nB, nC are the element counts of the three buffers: the largest offset
// the spec can reach is checked against them before any launch.
template <typename T>
void gemm_nd(const GemmND& g, const T* A, size_t nA, const T* B, size_t nB, T* C, size_t nC, T alpha, T beta,
             cudaStream_t st);

// Plain row-major batched GEMM helper: C[b] (MxN) = alpha op(A[b]) op(B[b]) + beta C[b].
template <typename T>
void gemm_rm(bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda, long long sA,
             const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch,
             cudaStream_t st, size_t nA = 0, size_t nB = 0, size_t nC = 0);

// Largest offset reachable along a combined index with the given strides.
inline long long max_offset(const IdxN& idx, const StrN& s) {
  long long o = 0;
  for (int i = 0; i < idx.nsub; ++i) {
    TT_CHECK(s.s[i] >= 0, TT_E_INTERNAL, "gemm_nd: negative stride");
    o += (long long)(idx.ext[i] - 1) * s.s[i];
  }
  return o;
}

}  // namespace ttsdp
