// Three-operand TT contractions of the block-AMEn solver (Section 3.3, the
// matrix-free local products with cached environments): left / right
// environment updates, the local product and the dense projected operator.
#pragma once

#include "common.cuh"

namespace ttsdp {

struct CDims {
  int rw, rw2, R, R2, rv, rv2, m, n;
};

// Algorithmic flops of one environment update or local product
// (three GEMM stages; 2 flops per multiply-add).
double contract_flops(const CDims& d);

// All pointers device, FP64 storage; `prec` is a tt_precision.
void env_left_step(const CDims& d, const double* phi, const double* u, const double* op,
                   const double* v, double* out, int prec, cudaStream_t st);
void env_right_step(const CDims& d, const double* psi, const double* u, const double* op,
                    const double* v, double* out, int prec, cudaStream_t st);
void local_apply(const CDims& d, const double* phi, const double* op, const double* psi,
                 const double* x, double* y, int prec, cudaStream_t st);
void local_matrix(const CDims& d, const double* phi, const double* op, const double* psi,
                  double* out, int prec, cudaStream_t st);

// FP64 <-> FP32 conversion of n contiguous elements.
void to_f32(const double* a, float* b, size_t n, cudaStream_t st);
void to_f64(const float* a, double* b, size_t n, cudaStream_t st);

// Statistics of timed work (device time via CUDA events and algorithmic
// flops). key 0: whole contraction calls; key 1: tensor-core GEMM launches;
// key 2: LU factorisations and solves of the dense local systems.
constexpr int kStatKeys = 4;  // contractions, tensor-core GEMMs, dense local solves, FP64 strided GEMMs
void stats_begin(cudaStream_t st, int key = 0);
void stats_end(cudaStream_t st, double flops, int key = 0);
void stats_read(double* flops, double* seconds, int key = 0, unsigned long long* calls = nullptr);
void stats_reset();

}  // namespace ttsdp
