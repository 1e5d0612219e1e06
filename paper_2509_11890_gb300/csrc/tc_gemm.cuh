// Tensor-core (tcgen05 / TMEM, TMA-fed) path for the heavy middle stage of
// the environment update and the local product:
//   T2[a'][i][q][b] = sum_{p,j} Op[p][i][j][q] T1[a'][p][j][b]
// for TF32 or BF16 inputs with FP32 accumulation.
#pragma once

#include "common.cuh"

namespace ttsdp {

// Returns true when the stage was executed on the tensor cores (TF32 / BF16
// precisions with float operands); false lets the caller run the SIMT path.
template <typename T>
bool tc_stage2(int prec, long long rw, long long R, long long R2, long long m, long long n,
               long long rv2, const T* op, const T* t1, T* t2, cudaStream_t st);

// The middle stage of the right environment update on the tensor cores:
//   T2[(p,i)][(a,b')] = sum_{j,q} Op[p][i][j][q] T1[a][j][b'][q]
// (C row-major, (R m) x (rv rw2)); same contract as tc_stage2.
template <typename T>
bool tc_stage2_right(int prec, long long rv, long long R, long long R2, long long m, long long n, long long rw2,
                     const T* op, const T* t1, T* t2, cudaStream_t st);

// Plain tensor-core GEMM C[b] (M x N, fp32 row-major) = A[b] (M x K) * B[b] (N x K)^T,
// both operands K-major in the given element type (TT_MIXED_TF32: fp32 storage
// read as TF32; TT_MIXED_BF16: bf16 storage). Used by stage 2 and by the
// benchmark's kernel timing.
// stat_flops > 0: the launches are timed with CUDA events and counted with
// that many algorithmic flops in the tensor-core statistics
void tc_gemm_tn(int prec, int M, int N, int K, int batch, const void* A, long long sA,
                const void* B, long long sB, float* C, long long sC, cudaStream_t st, double stat_flops = 0.0);

// C (M x N, fp64) = A (M x K, fp64, row stride lda) B (N x K, fp64, row stride
// ldb)^T with the product on the TF32 tensor cores (operands rounded to TF32,
// FP32 accumulation). Used by the randomised range finder of TT rounding.
void tc_gemm_f64_tn(int M, int N, int K, const double* A, long long lda, const double* B, long long ldb, double* C,
                    cudaStream_t st);

// Reads (and with reset clears) the error word a tensor-core kernel sets when
// one of its bounded waits gives up; 0 means no failure.
int tc_check_error(bool reset);

}  // namespace ttsdp
