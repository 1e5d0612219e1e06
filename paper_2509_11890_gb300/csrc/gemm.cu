// SIMT strided tensor-contraction GEMM (FP64 / FP32).
//
// One CTA computes a 64 x 64 tile of C for one batch entry, 256 threads with
// a 4 x 4 register tile each. The offsets of the tile's rows, columns and
// of each 16-wide K slice are decomposed once into shared memory, so loading
// an element is one add; out-of-range rows / columns / k read zero.
#include "gemm.cuh"

namespace ttsdp {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ long long offset_of(long long l, const IdxN& idx, const StrN& st) {
  long long off = 0;
#pragma unroll
  for (int i = kMaxSub - 1; i >= 0; --i) {
    if (i < idx.nsub) {
      long long e = idx.ext[i];
      long long dgt = l % e;
      l /= e;
      off += dgt * st.s[i];
    }
  }
  return off;
}

template <typename T>
__global__ void __launch_bounds__(NT) gemm_nd_kernel(GemmND g, const T* __restrict__ A,
                                                     const T* __restrict__ B, T* __restrict__ C,
                                                     T alpha, T beta, long long Mt, long long Nt,
                                                     long long Kt) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ long long offAM[BM], offCM[BM], offBN[BN], offCN[BN];
  __shared__ long long offAK[BK], offBK[BK];

  const long long m0 = (long long)blockIdx.y * BM;
  const long long n0 = (long long)blockIdx.x * BN;
  const long long b = blockIdx.z;
  const int tid = threadIdx.x;

  const long long baseA = offset_of(b, g.B, g.aB);
  const long long baseB = offset_of(b, g.B, g.bB);
  const long long baseC = offset_of(b, g.B, g.cB);

  if (tid < BM) {
    long long m = m0 + tid;
    offAM[tid] = m < Mt ? offset_of(m, g.M, g.aM) : -1;
    offCM[tid] = m < Mt ? offset_of(m, g.M, g.cM) : -1;
  } else if (tid < BM + BN) {
    int t = tid - BM;
    long long n = n0 + t;
    offBN[t] = n < Nt ? offset_of(n, g.N, g.bN) : -1;
    offCN[t] = n < Nt ? offset_of(n, g.N, g.cN) : -1;
  }

  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (long long k0 = 0; k0 < Kt; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      long long k = k0 + tid;
      offAK[tid] = k < Kt ? offset_of(k, g.K, g.aK) : -1;
    } else if (tid < 2 * BK) {
      int t = tid - BK;
      long long k = k0 + t;
      offBK[t] = k < Kt ? offset_of(k, g.K, g.bK) : -1;
    }
    __syncthreads();
    // A tile: BM x BK elements, k fastest across threads
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int e = tid + r * NT;
      int kk = e % BK, mm = e / BK;
      long long om = offAM[mm], ok = offAK[kk];
      As[kk][mm] = (om >= 0 && ok >= 0) ? A[baseA + om + ok] : T(0);
    }
    // B tile: BK x BN elements, n fastest across threads
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int e = tid + r * NT;
      int nn = e % BN, kk = e / BN;
      long long on = offBN[nn], ok = offBK[kk];
      Bs[kk][nn] = (on >= 0 && ok >= 0) ? B[baseB + ok + on] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long om = offCM[ty + 16 * i];
    if (om < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long on = offCN[tx + 16 * j];
      if (on < 0) continue;
      T* c = C + baseC + om + on;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * (*c);
      *c = v;
    }
  }
}

}  // namespace

template <typename T>
void gemm_nd(const GemmND& g, const T* A, size_t nA, const T* B, size_t nB, T* C, size_t nC, T alpha, T beta,
             cudaStream_t st) {
  long long Mt = g.M.total(), Nt = g.N.total(), Kt = g.K.total(), Bt = g.B.total();
  if (Mt == 0 || Nt == 0 || Bt == 0) return;
  // every reachable offset must lie inside the caller's buffers
  long long ra = max_offset(g.M, g.aM) + max_offset(g.B, g.aB) + (Kt > 0 ? max_offset(g.K, g.aK) : 0);
  long long rb = max_offset(g.N, g.bN) + max_offset(g.B, g.bB) + (Kt > 0 ? max_offset(g.K, g.bK) : 0);
  long long rc = max_offset(g.M, g.cM) + max_offset(g.N, g.cN) + max_offset(g.B, g.cB);
  TT_CHECK((Kt == 0 || ((size_t)ra < nA && (size_t)rb < nB)) && (size_t)rc < nC, TT_E_INTERNAL,
           "gemm_nd: operand extent exceeds its buffer");
  TT_CHECK(Bt <= 65535, TT_E_SHAPE, "gemm_nd: batch too large");
  TT_CHECK((Mt + BM - 1) / BM < 65536, TT_E_SHAPE, "gemm_nd: M too large");
  dim3 grid((unsigned)((Nt + BN - 1) / BN), (unsigned)((Mt + BM - 1) / BM), (unsigned)Bt);
  gemm_nd_kernel<T><<<grid, NT, 0, st>>>(g, A, B, C, alpha, beta, Mt, Nt, Kt);
  count_launch();
  check_launch("gemm_nd_kernel");
}

template <typename T>
void gemm_rm(bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda, long long sA,
             const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch,
             cudaStream_t st, size_t nA, size_t nB, size_t nC) {
  GemmND g;
  // A: row-major M x K (lda) or its transpose stored K x M
  set_dim(g.M, g.aM, g.cM, {{M, ta ? 1LL : (long long)lda, (long long)ldc}});
  set_dim(g.N, g.bN, g.cN, {{N, tb ? (long long)ldb : 1LL, 1LL}});
  set_dim(g.K, g.aK, g.bK, {{K, ta ? (long long)lda : 1LL, tb ? 1LL : (long long)ldb}});
  set_batch(g, {{batch, sA, sB, sC}});
  // callers that pass no sizes get the extents implied by the leading dimensions
  if (!nA) nA = (size_t)(max_offset(g.M, g.aM) + max_offset(g.K, g.aK) + max_offset(g.B, g.aB)) + 1;
  if (!nB) nB = (size_t)(max_offset(g.N, g.bN) + max_offset(g.K, g.bK) + max_offset(g.B, g.bB)) + 1;
  if (!nC) nC = (size_t)(max_offset(g.M, g.cM) + max_offset(g.N, g.cN) + max_offset(g.B, g.cB)) + 1;
  TT_CHECK(lda >= (ta ? M : K) && ldb >= (tb ? K : N) && ldc >= N, TT_E_INTERNAL, "gemm_rm: leading dimension");
  gemm_nd<T>(g, A, nA, B, nB, C, nC, alpha, beta, st);
}

template void gemm_nd<double>(const GemmND&, const double*, size_t, const double*, size_t, double*, size_t,
                              double, double, cudaStream_t);
template void gemm_nd<float>(const GemmND&, const float*, size_t, const float*, size_t, float*, size_t, float,
                             float, cudaStream_t);
template void gemm_rm<double>(bool, bool, int, int, int, double, const double*, int, long long,
                              const double*, int, long long, double, double*, int, long long, int,
                              cudaStream_t, size_t, size_t, size_t);
template void gemm_rm<float>(bool, bool, int, int, int, float, const float*, int, long long,
                             const float*, int, long long, float, float*, int, long long, int,
                             cudaStream_t, size_t, size_t, size_t);

}  // namespace ttsdp
