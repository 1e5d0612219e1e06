// SIMT strided tensor-contraction GEMM (FP64 / FP32).
//
// One CTA computes a 64 x 64 tile of C for one batch entry, 256 threads with
// a 4 x 4 register tile each. The offsets of the tile's rows, columns and
// of each 16-wide K slice are decomposed once into shared memory, so loading
// an element is one add; out-of-range rows / columns / k read zero.
#include <algorithm>

#include "contract.cuh"
#include "gemm.cuh"

namespace ttsdp {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int KTAB = 2048;  // K offsets precomputed once per CTA up to this length

// device copy of a combined index with 32-bit extents / strides
struct Idx32 {
  int nsub;
  int ext[kMaxSub];
  int s0[kMaxSub], s1[kMaxSub];
};
struct Gemm32 {
  Idx32 M, N, K, B;   // M: (aM, cM), N: (bN, cN), K: (aK, bK)
  int bA[kMaxSub], bB[kMaxSub], bC[kMaxSub];
};

__device__ __forceinline__ void offsets_of(int l, const Idx32& idx, int& o0, int& o1) {
  o0 = 0;
  o1 = 0;
#pragma unroll
  for (int i = kMaxSub - 1; i >= 0; --i) {
    if (i < idx.nsub) {
      const int e = idx.ext[i];
      const int dgt = l % e;
      l /= e;
      o0 += dgt * idx.s0[i];
      o1 += dgt * idx.s1[i];
    }
  }
}

// With ksplit > 1, blockIdx.z = batch * ksplit + split: the CTA sums the K range
// [split * kchunk, min(Kt, (split + 1) * kchunk)) and writes its partial tile,
// unscaled, to the dense workspace W[batch][split][m][n] (C is not touched);
// `split_reduce_kernel` then adds the partials in split order into C.
template <typename T>
__global__ void __launch_bounds__(NT) gemm_nd_kernel(Gemm32 g, const T* __restrict__ A,
                                                     const T* __restrict__ B, T* __restrict__ C,
                                                     T alpha, T beta, int Mt, int Nt, int Kfull, int ksplit,
                                                     int kchunk, T* __restrict__ W) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ int offAM[BM], offCM[BM], offBN[BN], offCN[BN];
  __shared__ int offAK[KTAB], offBK[KTAB];

  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;

  const int split = ksplit > 1 ? (int)(blockIdx.z % ksplit) : 0;
  const int bz = ksplit > 1 ? (int)(blockIdx.z / ksplit) : (int)blockIdx.z;
  const int kbeg = split * kchunk;
  const int Kt = ksplit > 1 ? min(Kfull - kbeg, kchunk) : Kfull;  // this CTA's K length
  int baseA = 0, baseB = 0, baseC = 0;
  {
    int l = bz;
#pragma unroll
    for (int i = kMaxSub - 1; i >= 0; --i) {
      if (i < g.B.nsub) {
        const int e = g.B.ext[i];
        const int dgt = l % e;
        l /= e;
        baseA += dgt * g.bA[i];
        baseB += dgt * g.bB[i];
        baseC += dgt * g.bC[i];
      }
    }
  }
  if (tid < BM) {
    const int m = m0 + tid;
    int oa = -1, oc = -1;
    if (m < Mt) offsets_of(m, g.M, oa, oc);
    offAM[tid] = oa;
    offCM[tid] = oc;
  } else if (tid < BM + BN) {
    const int t = tid - BM;
    const int n = n0 + t;
    int ob = -1, oc = -1;
    if (n < Nt) offsets_of(n, g.N, ob, oc);
    offBN[t] = ob;
    offCN[t] = oc;
  }
  const bool ktab = Kt <= KTAB;
  if (ktab) {
    for (int k = tid; k < Kt; k += NT) {
      int oa, ob;
      offsets_of(kbeg + k, g.K, oa, ob);
      offAK[k] = oa;
      offBK[k] = ob;
    }
  }

  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < Kt; k0 += BK) {
    __syncthreads();
    if (!ktab && tid < BK) {
      const int k = k0 + tid;
      int oa = -1, ob = -1;
      if (k < Kt) offsets_of(kbeg + k, g.K, oa, ob);
      offAK[tid] = oa;
      offBK[tid] = ob;
    }
    __syncthreads();
    const int kb = ktab ? k0 : 0;
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      const int e = tid + r * NT;
      const int kk = e % BK, mm = e / BK;
      const int om = offAM[mm];
      const bool kin = k0 + kk < Kt;
      As[kk][mm] = (om >= 0 && kin) ? A[baseA + om + offAK[kb + kk]] : T(0);
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      const int e = tid + r * NT;
      const int nn = e % BN, kk = e / BN;
      const int on = offBN[nn];
      const bool kin = k0 + kk < Kt;
      Bs[kk][nn] = (on >= 0 && kin) ? B[baseB + offBK[kb + kk] + on] : T(0);
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
  if (ksplit > 1) {
    T* w = W + ((long long)bz * ksplit + split) * (long long)Mt * Nt;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty + 16 * i;
      if (m >= Mt) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n < Nt) w[(long long)m * Nt + n] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int om = offCM[ty + 16 * i];
    if (om < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int on = offCN[tx + 16 * j];
      if (on < 0) continue;
      T* c = C + baseC + om + on;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * (*c);
      *c = v;
    }
  }
}

// C[batch][m][n] = alpha * sum over the splits of W[batch][split][m][n] + beta * C,
// the splits added in index order (deterministic)
template <typename T>
__global__ void split_reduce_kernel(Gemm32 g, T* __restrict__ C, const T* __restrict__ W, T alpha, T beta,
                                    int Mt, int Nt, int Bt, int ksplit) {
  const long long tot = (long long)Bt * Mt * Nt;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e % Nt), m = (int)((e / Nt) % Mt), bz = (int)(e / ((long long)Nt * Mt));
    T acc = T(0);
    for (int s = 0; s < ksplit; ++s) acc += W[(((long long)bz * ksplit + s) * Mt + m) * Nt + n];
    int baseC = 0, l = bz;
    for (int i = kMaxSub - 1; i >= 0; --i) {
      if (i < g.B.nsub) {
        const int ex = g.B.ext[i];
        baseC += (l % ex) * g.bC[i];
        l /= ex;
      }
    }
    int oa, om, ob, on;
    offsets_of(m, g.M, oa, om);
    offsets_of(n, g.N, ob, on);
    T* c = C + baseC + om + on;
    T v = alpha * acc;
    if (beta != T(0)) v += beta * (*c);
    *c = v;
  }
}

Idx32 to32(const IdxN& idx, const StrN& a, const StrN& b) {
  Idx32 o;
  o.nsub = idx.nsub;
  for (int i = 0; i < kMaxSub; ++i) {
    o.ext[i] = idx.ext[i];
    o.s0[i] = (int)a.s[i];
    o.s1[i] = (int)b.s[i];
  }
  return o;
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
  // offsets are 32-bit on the device
  const long long lim = 2147483647LL;
  TT_CHECK(ra < lim && rb < lim && rc < lim && Mt < lim && Nt < lim && Kt < lim, TT_E_SHAPE,
           "gemm_nd: operand too large for 32-bit offsets");
  Gemm32 d;
  d.M = to32(g.M, g.aM, g.cM);
  d.N = to32(g.N, g.bN, g.cN);
  d.K = to32(g.K, g.aK, g.bK);
  d.B.nsub = g.B.nsub;
  for (int i = 0; i < kMaxSub; ++i) {
    d.B.ext[i] = g.B.ext[i];
    d.bA[i] = (int)g.aB.s[i];
    d.bB[i] = (int)g.bB.s[i];
    d.bC[i] = (int)g.cB.s[i];
  }
  // few output tiles and a long K: split K over CTAs so that the launch fills
  // the SMs (at least 256 k per split, at most 64 splits)
  const long long tiles = ((Nt + BN - 1) / BN) * ((Mt + BM - 1) / BM) * Bt;
  int ksplit = 1;
  if (tiles < 152 && Kt >= 512) {
    ksplit = (int)std::min<long long>(std::min<long long>((2 * 152 + tiles - 1) / tiles, Kt / 256), 64);
    while (ksplit > 1 && Bt * ksplit > 65535) --ksplit;
  }
  const int kchunk = ksplit > 1 ? (int)((Kt + ksplit - 1) / ksplit) : (int)Kt;
  if (ksplit > 1) ksplit = (int)((Kt + kchunk - 1) / kchunk);
  DBuf<T> work;
  if (ksplit > 1) work.alloc((size_t)Bt * ksplit * Mt * Nt);
  dim3 grid((unsigned)((Nt + BN - 1) / BN), (unsigned)((Mt + BM - 1) / BM), (unsigned)(Bt * ksplit));
  // every eighth FP64 launch of this thread is timed (CUDA events) and
  // counted with its 2 M N K flops: the rate, at an eighth of the events
  static thread_local unsigned sample = 0;
  const bool kTimed = std::is_same<T, double>::value && (sample++ % 8) == 0;
  if (kTimed) stats_begin(st, 3);
  gemm_nd_kernel<T><<<grid, NT, 0, st>>>(d, A, B, C, alpha, beta, (int)Mt, (int)Nt, (int)Kt, ksplit, kchunk,
                                         work.get());
  count_launch();
  check_launch("gemm_nd_kernel");
  if (ksplit > 1) {
    const long long tot = Bt * Mt * Nt;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 16);
    split_reduce_kernel<T><<<blocks, 256, 0, st>>>(d, C, work.get(), alpha, beta, (int)Mt, (int)Nt, (int)Bt, ksplit);
    count_launch();
    check_launch("split_reduce_kernel");
  }
  if (kTimed) stats_end(st, 2.0 * (double)Mt * (double)Nt * (double)Kt * (double)Bt, 3);
}

namespace {
// y = alpha A x + beta y for row-major A (M x K, row stride lda): one warp
// per row, coalesced along the row, four independent partial sums per lane.
template <typename T>
__global__ void gemv_rows_kernel(int M, int K, T alpha, const T* __restrict__ A, long long lda,
                                 const T* __restrict__ x, long long incx, T beta, T* __restrict__ y,
                                 long long incy) {
  const int lane = threadIdx.x & 31;
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= M) return;
  const T* a = A + row * lda;
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int k = lane;
  for (; k + 96 < K; k += 128) {
    s0 += a[k] * x[k * incx];
    s1 += a[k + 32] * x[(k + 32) * incx];
    s2 += a[k + 64] * x[(k + 64) * incx];
    s3 += a[k + 96] * x[(k + 96) * incx];
  }
  for (; k < K; k += 32) s0 += a[k] * x[k * incx];
  T s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row * incy] = alpha * s + (beta != T(0) ? beta * y[row * incy] : T(0));
}

// y = alpha A^T x + beta y for row-major A (K x M, row stride lda): one
// thread per output, reading row k of A coalesced across the threads.
template <typename T>
__global__ void gemv_cols_kernel(int M, int K, T alpha, const T* __restrict__ A, long long lda,
                                 const T* __restrict__ x, long long incx, T beta, T* __restrict__ y,
                                 long long incy) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  T s = T(0);
  for (int k = 0; k < K; ++k) s += A[(long long)k * lda + m] * x[k * incx];
  y[m * incy] = alpha * s + (beta != T(0) ? beta * y[m * incy] : T(0));
}
}  // namespace

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
  if (N == 1 && batch == 1 && M > 0 && K > 0) {
    // matrix-vector product: x is column 0 of B (stride ldb, or 1 when B is
    // given transposed), y column 0 of C (stride ldc)
    const long long incx = tb ? 1 : ldb;
    TT_CHECK(max_offset(g.M, g.aM) + max_offset(g.K, g.aK) < (long long)nA &&
                 (long long)(K - 1) * incx < (long long)nB && (long long)(M - 1) * ldc < (long long)nC,
             TT_E_INTERNAL, "gemm_rm: operand extent");
    if (!ta) {
      gemv_rows_kernel<T><<<ceil_div((long)M * 32, 256), 256, 0, st>>>(M, K, alpha, A, lda, B, incx, beta, C, ldc);
    } else {
      gemv_cols_kernel<T><<<ceil_div(M, 256), 256, 0, st>>>(M, K, alpha, A, lda, B, incx, beta, C, ldc);
    }
    count_launch();
    check_launch("gemv");
    return;
  }
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
