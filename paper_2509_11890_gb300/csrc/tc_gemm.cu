// Tensor-core (tcgen05 / TMEM) GEMM fed by TMA, for the heavy middle stage of
// the environment update and the local product:
//   T2[(i,q)][(a',b)] = sum_{(p,j)} Op[p][i][j][q] T1[a'][p][j][b]
// computed as one TN GEMM C (M x N, fp32) = A (M x K) B (N x K)^T with both
// operands K-major: A = the operator core reordered to [(i,q)][(p,j)], B = the
// stage-1 result reordered to [(a',b)][(p,j)].
//
// Kernel structure (one 128 x 128 output tile per CTA, 128 threads):
//  - thread 0 of warp 0 streams 128-byte-wide K slices of A and B into a
//    4-stage shared-memory ring with cp.async.bulk.tensor (128B swizzle);
//  - thread 0 of warp 1 issues tcgen05.mma (kind::tf32 or kind::f16 with BF16
//    operands) into a 128 x 128 FP32 accumulator in tensor memory and releases
//    each stage with tcgen05.commit;
//  - all four warps read the accumulator back with tcgen05.ld and store the
//    in-range part of the tile.
// Every mbarrier wait is bounded; a wait that gives up records an error code
// that the host reads with tc_check_error().
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "contract.cuh"
#include "tc_gemm.cuh"

namespace ttsdp {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_STAGES = 4, TC_THREADS = 128;
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr int kFmtBF16 = 1, kFmtTF32 = 2;

__device__ int g_tc_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok = 0;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, atoms of
// 8 rows x 128 bytes stacked every 1024 bytes along M (or N).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused by 128B-swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, both K-major, N>>3, M>>4.
__host__ __device__ constexpr uint32_t make_idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float* C,
                   int M, int N, int K, long long ldc) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int ESZ = FMT == kFmtTF32 ? 4 : 2;
  constexpr int BK = 128 / ESZ;  // elements per 128-byte row of a K slice
  constexpr int UK = 32 / ESZ;   // K of one MMA instruction (32 bytes)
  constexpr uint32_t A_BYTES = TC_BM * 128, B_BYTES = TC_BN * 128;
  uint8_t* sA = smem;
  uint8_t* sB = smem + TC_STAGES * A_BYTES;
  uint64_t* full = (uint64_t*)(smem + TC_STAGES * (A_BYTES + B_BYTES));
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t round = kb / TC_STAGES;
      if (kb >= TC_STAGES && !mbar_wait(&empty[s], (round - 1) & 1)) {
        s_fail = 1;
        break;
      }
      mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, &ta, &full[s], kb * BK, m0);
      tma_load_2d(sB + s * B_BYTES, &tb, &full[s], kb * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = make_idesc(FMT, TC_BM, TC_BN);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t round = kb / TC_STAGES;
      if (!mbar_wait(&full[s], round & 1)) {
        s_fail = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_base = smem_u32(sA + s * A_BYTES), b_base = smem_u32(sB + s * B_BYTES);
#pragma unroll
      for (int k = 0; k < BK / UK; ++k) {
        const uint64_t da = smem_desc_sw128(a_base + k * 32), db = smem_desc_sw128(b_base + k * 32);
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        if constexpr (FMT == kFmtTF32) {
          asm volatile(
              "{\n"
              " .reg .pred p;\n"
              " setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
              "}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        } else {
          asm volatile(
              "{\n"
              " .reg .pred p;\n"
              " setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
              "}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    if (ok)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(done))
                   : "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (ok) {
    // the accumulator goes out through shared memory (the operand ring is idle
    // once `done` has fired): each lane holds 32 columns of its own row after
    // tcgen05.ld, the warp transposes them through a padded 32 x 33 buffer and
    // then stores one row per instruction, 128 contiguous bytes
    float* stage = reinterpret_cast<float*>(sA) + warp * 32 * 33;
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int lim = N - (n0 + c0);
      for (int r = 0; r < 32; ++r) {
        const int row = m0 + warp * 32 + r;
        if (row < M && lane < lim) C[(long long)row * ldc + n0 + c0 + lane] = stage[r * 33 + lane];
      }
      __syncwarp();
    }
  }
  if (!ok || s_fail) {
    if (threadIdx.x == 0) atomicExch(&g_tc_error, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
  }
}

// [(i,q)][(p,j)] <- Op[p][i][j][q], leading dimension ld (K padded with zeros)
template <typename TO>
__global__ void pack_op_kernel(const float* __restrict__ op, int R, int m, int n, int R2, long long ld, TO* out) {
  const long long M = (long long)m * R2, tot = M * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld, k = e % ld;
    float v = 0.f;
    if (k < (long long)R * n) {
      const int i = (int)(row / R2), q = (int)(row % R2), p = (int)(k / n), j = (int)(k % n);
      v = op[(((long long)p * m + i) * n + j) * R2 + q];
    }
    out[e] = (TO)v;
  }
}

// [(a',b)][(p,j)] <- T1[a'][p][j][b], leading dimension ld (K padded with zeros)
template <typename TO>
__global__ void pack_t1_kernel(const float* __restrict__ t1, int rw, int R, int n, int rv2, long long ld, TO* out) {
  const long long Nr = (long long)rw * rv2, tot = Nr * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld, k = e % ld;
    float v = 0.f;
    if (k < (long long)R * n) {
      const int a = (int)(row / rv2), b = (int)(row % rv2), p = (int)(k / n), j = (int)(k % n);
      v = t1[(((long long)a * R + p) * n + j) * rv2 + b];
    }
    out[e] = (TO)v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  TT_CHECK(fn != nullptr, TT_E_CUDA, "cuTensorMapEncodeTiled unavailable");
  return fn;
}

CUtensorMap make_map(const void* base, bool bf16, long long inner, long long outer, long long ld) {
  const int esz = bf16 ? 2 : 4;
  TT_CHECK(((uintptr_t)base % 16) == 0, TT_E_INTERNAL, "TMA base must be 16-byte aligned");
  TT_CHECK((ld * esz) % 16 == 0, TT_E_INTERNAL, "TMA row stride must be a multiple of 16 bytes");
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encoder()(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TT_CHECK(r == CUDA_SUCCESS, TT_E_CUDA, "cuTensorMapEncodeTiled failed");
  return map;
}

constexpr size_t kSmemBytes = TC_STAGES * (TC_BM + TC_BN) * 128 + 1024 + 256;

int grid1(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  return (int)(g > 152 * 16 ? 152 * 16 : g);
}

}  // namespace

void tc_gemm_tn(int prec, int M, int N, int K, int batch, const void* A, long long sA, const void* B, long long sB,
                float* C, long long sC, cudaStream_t st, double stat_flops) {
  TT_CHECK(prec == TT_MIXED_TF32 || prec == TT_MIXED_BF16, TT_E_INVALID_ARG, "tensor-core precision expected");
  TT_CHECK(M > 0 && N > 0 && K > 0 && batch > 0, TT_E_SHAPE, "tc_gemm_tn: empty shape");
  const bool bf16 = prec == TT_MIXED_BF16;
  const int esz = bf16 ? 2 : 4;
  const long long ld = K;  // operands are packed with a padded K (multiple of 8)
  TT_CHECK((ld * esz) % 16 == 0, TT_E_INTERNAL, "tc_gemm_tn: K must be padded to 16 bytes");
  static std::once_flag attr_once[2];
  cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once[bf16], [&]() {
    attr_err = bf16 ? cudaFuncSetAttribute(tc_gemm_kernel<kFmtBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kSmemBytes)
                    : cudaFuncSetAttribute(tc_gemm_kernel<kFmtTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kSmemBytes);
  });
  TT_CUDA(attr_err);
  dim3 grid((unsigned)((N + TC_BN - 1) / TC_BN), (unsigned)((M + TC_BM - 1) / TC_BM));
  // tensor maps are encoded on the host before the timed region opens, so the
  // recorded time is the kernels' device time only
  std::vector<std::pair<CUtensorMap, CUtensorMap>> maps((size_t)batch);
  for (int b = 0; b < batch; ++b) {
    const char* pa = (const char*)A + (size_t)b * sA * esz;
    const char* pb = (const char*)B + (size_t)b * sB * esz;
    maps[(size_t)b] = {make_map(pa, bf16, K, M, ld), make_map(pb, bf16, K, N, ld)};
  }
  if (stat_flops > 0) stats_begin(st, 1);
  for (int b = 0; b < batch; ++b) {
    const CUtensorMap& ma = maps[(size_t)b].first;
    const CUtensorMap& mb = maps[(size_t)b].second;
    if (bf16)
      tc_gemm_kernel<kFmtBF16><<<grid, TC_THREADS, kSmemBytes, st>>>(ma, mb, C + (size_t)b * sC, M, N, K, N);
    else
      tc_gemm_kernel<kFmtTF32><<<grid, TC_THREADS, kSmemBytes, st>>>(ma, mb, C + (size_t)b * sC, M, N, K, N);
    count_launch();
    check_launch("tc_gemm_kernel");
  }
  if (stat_flops > 0) stats_end(st, stat_flops, 1);
}

namespace {
// dst (rows x ld, fp32, zero-padded columns) <- src (rows x cols, fp64, row stride sld)
__global__ void pack_f64_kernel(const double* __restrict__ src, int rows, int cols, long long sld, long long ld,
                                float* dst) {
  const long long tot = (long long)rows * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ld, j = e % ld;
    dst[e] = j < cols ? (float)src[i * sld + j] : 0.f;
  }
}
__global__ void widen_kernel(const float* __restrict__ src, long long n, double* dst) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}
}  // namespace

void tc_gemm_f64_tn(int M, int N, int K, const double* A, long long lda, const double* B, long long ldb, double* C,
                    cudaStream_t st) {
  const long long Kp = (K + 7) / 8 * 8;
  DBuf<float> a((size_t)M * Kp), b((size_t)N * Kp), c((size_t)M * N);
  pack_f64_kernel<<<grid1((long long)M * Kp), 256, 0, st>>>(A, M, K, lda, Kp, a.get());
  pack_f64_kernel<<<grid1((long long)N * Kp), 256, 0, st>>>(B, N, K, ldb, Kp, b.get());
  count_launch();
  count_launch();
  tc_gemm_tn(TT_MIXED_TF32, M, N, (int)Kp, 1, a.get(), 0, b.get(), 0, c.get(), 0, st);
  widen_kernel<<<grid1((long long)M * N), 256, 0, st>>>(c.get(), (long long)M * N, C);
  count_launch();
  check_launch("tc_gemm_f64_tn");
}

int tc_check_error(bool reset) {
  // read on the caller's stream, after the work it has queued (contexts solved
  // concurrently run on non-blocking streams the legacy stream does not order)
  cudaStream_t st = cur_stream();
  int h = 0;
  TT_CUDA(cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  if (reset && h) {
    int z = 0;
    TT_CUDA(cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    TT_CUDA(sync_stream(st));
  }
  return h;
}

template <typename T>
bool tc_stage2(int prec, long long rw, long long R, long long R2, long long m, long long n, long long rv2, const T* op,
               const T* t1, T* t2, cudaStream_t st) {
  if (prec == TT_FP64 || prec == TT_FP32) return false;
  if constexpr (!std::is_same<T, float>::value) {
    throw TTError(TT_E_INTERNAL, "tensor-core stage needs float operands");
  } else {
    const bool bf16 = prec == TT_MIXED_BF16;
    const long long M = m * R2, N = rw * rv2, Kr = R * n;
    const long long Kp = (Kr + 7) / 8 * 8;
    const int esz = bf16 ? 2 : 4;
    DBuf<uint8_t> a((size_t)(M * Kp * esz)), b((size_t)(N * Kp * esz));
    if (bf16) {
      pack_op_kernel<__nv_bfloat16><<<grid1(M * Kp), 256, 0, st>>>(op, (int)R, (int)m, (int)n, (int)R2, Kp,
                                                                    (__nv_bfloat16*)a.get());
      pack_t1_kernel<__nv_bfloat16><<<grid1(N * Kp), 256, 0, st>>>(t1, (int)rw, (int)R, (int)n, (int)rv2, Kp,
                                                                    (__nv_bfloat16*)b.get());
    } else {
      pack_op_kernel<float><<<grid1(M * Kp), 256, 0, st>>>(op, (int)R, (int)m, (int)n, (int)R2, Kp, (float*)a.get());
      pack_t1_kernel<float><<<grid1(N * Kp), 256, 0, st>>>(t1, (int)rw, (int)R, (int)n, (int)rv2, Kp,
                                                            (float*)b.get());
    }
    count_launch();
    count_launch();
    check_launch("tc pack");
    // C layout [(i,q)][(a',b)], fp32; timed as one kernel with its algorithmic K
    tc_gemm_tn(prec, (int)M, (int)N, (int)Kp, 1, a.get(), 0, b.get(), 0, t2, 0, st,
               2.0 * (double)M * (double)N * (double)Kr);
    return true;
  }
}

namespace {
// [(p,i)][(j,q)] <- Op[p][i][j][q]: the natural layout with K padded to ld
template <typename TO>
__global__ void pack_op_right_kernel(const float* __restrict__ op, long long rows, long long K, long long ld,
                                     TO* out) {
  const long long tot = rows * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld, k = e % ld;
    out[e] = (TO)(k < K ? op[row * K + k] : 0.f);
  }
}

// [(a,b')][(j,q)] <- T1[a][j][b'][q], K padded to ld
template <typename TO>
__global__ void pack_t1_right_kernel(const float* __restrict__ t1, int rv, int n, int rw2, int R2, long long ld,
                                     TO* out) {
  const long long Nr = (long long)rv * rw2, tot = Nr * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld, k = e % ld;
    float v = 0.f;
    if (k < (long long)n * R2) {
      const int a = (int)(row / rw2), b = (int)(row % rw2), j = (int)(k / R2), q = (int)(k % R2);
      v = t1[(((long long)a * n + j) * rw2 + b) * R2 + q];
    }
    out[e] = (TO)v;
  }
}
}  // namespace

template <typename T>
bool tc_stage2_right(int prec, long long rv, long long R, long long R2, long long m, long long n, long long rw2,
                     const T* op, const T* t1, T* t2, cudaStream_t st) {
  if (prec == TT_FP64 || prec == TT_FP32) return false;
  if constexpr (!std::is_same<T, float>::value) {
    throw TTError(TT_E_INTERNAL, "tensor-core stage needs float operands");
  } else {
    const bool bf16 = prec == TT_MIXED_BF16;
    const long long M = R * m, N = rv * rw2, Kr = n * R2;
    const long long Kp = (Kr + 7) / 8 * 8;
    const int esz = bf16 ? 2 : 4;
    DBuf<uint8_t> a((size_t)(M * Kp * esz)), b((size_t)(N * Kp * esz));
    if (bf16) {
      pack_op_right_kernel<__nv_bfloat16><<<grid1(M * Kp), 256, 0, st>>>(op, M, Kr, Kp, (__nv_bfloat16*)a.get());
      pack_t1_right_kernel<__nv_bfloat16><<<grid1(N * Kp), 256, 0, st>>>(t1, (int)rv, (int)n, (int)rw2, (int)R2, Kp,
                                                                          (__nv_bfloat16*)b.get());
    } else {
      pack_op_right_kernel<float><<<grid1(M * Kp), 256, 0, st>>>(op, M, Kr, Kp, (float*)a.get());
      pack_t1_right_kernel<float><<<grid1(N * Kp), 256, 0, st>>>(t1, (int)rv, (int)n, (int)rw2, (int)R2, Kp,
                                                                  (float*)b.get());
    }
    count_launch();
    count_launch();
    check_launch("tc pack (right)");
    tc_gemm_tn(prec, (int)M, (int)N, (int)Kp, 1, a.get(), 0, b.get(), 0, t2, 0, st,
               2.0 * (double)M * (double)N * (double)Kr);
    return true;
  }
}

template bool tc_stage2_right<double>(int, long long, long long, long long, long long, long long, long long,
                                      const double*, const double*, double*, cudaStream_t);
template bool tc_stage2_right<float>(int, long long, long long, long long, long long, long long, long long,
                                     const float*, const float*, float*, cudaStream_t);

template bool tc_stage2<double>(int, long long, long long, long long, long long, long long, long long,
                                const double*, const double*, double*, cudaStream_t);
template bool tc_stage2<float>(int, long long, long long, long long, long long, long long, long long, const float*,
                               const float*, float*, cudaStream_t);

}  // namespace ttsdp
