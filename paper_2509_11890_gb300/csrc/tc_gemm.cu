// Tensor-core path for the middle contraction stage (TF32 / BF16 inputs,
// FP32 accumulation). Placeholder dispatch: the SIMT path handles FP64/FP32.
#include "tc_gemm.cuh"

namespace ttsdp {

template <typename T>
bool tc_stage2(int prec, long long, long long, long long, long long, long long, long long, const T*, const T*, T*,
               cudaStream_t) {
  if (prec == TT_FP64 || prec == TT_FP32) return false;
  throw TTError(TT_E_INVALID_ARG, "tensor-core precisions are not available in this build");
}

template bool tc_stage2<double>(int, long long, long long, long long, long long, long long, long long,
                                const double*, const double*, double*, cudaStream_t);
template bool tc_stage2<float>(int, long long, long long, long long, long long, long long, long long, const float*,
                               const float*, float*, cudaStream_t);

void tc_gemm_tn(int, int, int, int, int, const void*, long long, const void*, long long, float*, long long,
                cudaStream_t) {
  throw TTError(TT_E_INVALID_ARG, "tensor-core GEMM not available in this build");
}

}  // namespace ttsdp
