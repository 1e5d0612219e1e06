// Environment updates, local products and projected matrices as three
// strided GEMM stages on the cores' natural row-major layouts:
//   stage 1  contract the environment with the vector core over its rank,
//   stage 2  contract with the operator core over (operator rank, mode),
//   stage 3  contract with the frame core (or the other environment).
// FP64 runs the stages in FP64; FP32 converts the operands once and runs
// the same stages in FP32 with FP32 accumulation.
#include <memory>
#include <mutex>

#include "contract.cuh"
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace ttsdp {

namespace {

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long s = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += s) b[i] = (float)a[i];
}
__global__ void to_double_kernel(const float* __restrict__ a, double* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long s = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += s) b[i] = (double)a[i];
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

// Per-core norm scaling of the reduced-precision contractions: every FP64
// operand is scaled to unit Frobenius norm before it is rounded to FP32 (and
// from there to TF32 or BF16 on the tensor cores), and the FP64 result is
// multiplied back by the product of the norms, kept in FP64. The contraction
// is linear in each operand, so the scaling changes only the rounding: every
// operand's entries are O(1) whatever the magnitude of the iterate.
constexpr int kMaxOps = 4;
struct OpSet {
  const double* src[kMaxOps];
  float* dst[kMaxOps];
  long long n[kMaxOps];
  int count;
};

// nrm2[k] += sum of squares of operand blockIdx.y (nrm2 zeroed beforehand)
__global__ void sumsq_kernel(OpSet ops, double* nrm2) {
  const int k = blockIdx.y;
  const double* a = ops.src[k];
  const long long n = ops.n[k];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i] * a[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(&nrm2[k], s);
  }
}

// dst = (float)(src / ||src||) for operand blockIdx.y (unscaled when the norm is 0)
__global__ void to_float_scaled_kernel(OpSet ops, const double* __restrict__ nrm2) {
  const int k = blockIdx.y;
  const double v = nrm2[k];
  const double inv = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  const double* a = ops.src[k];
  float* b = ops.dst[k];
  const long long n = ops.n[k];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)(a[i] * inv);
}

// out = (double)e * prod_k ||operand k|| (the norms of the operands that were scaled)
__global__ void to_double_scaled_kernel(const float* __restrict__ e, double* __restrict__ out, long long n,
                                        const double* __restrict__ nrm2, int count) {
  double s = 1.0;
  for (int k = 0; k < count; ++k) s *= nrm2[k] > 0.0 ? sqrt(nrm2[k]) : 1.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)e[i] * s;
}

// Scaled conversion of up to four operands; returns the device array of
// their squared norms (owned by the caller's scratch `nrm2`).
void to_float_scaled(const OpSet& ops, double* nrm2, cudaStream_t st) {
  long long mx = 1;
  for (int k = 0; k < ops.count; ++k) mx = ops.n[k] > mx ? ops.n[k] : mx;
  TT_CUDA(cudaMemsetAsync(nrm2, 0, sizeof(double) * kMaxOps, st));
  const int gx = grid_for(mx) < 64 ? grid_for(mx) : 64;
  sumsq_kernel<<<dim3(gx, ops.count), 256, 0, st>>>(ops, nrm2);
  count_launch();
  check_launch("sumsq_kernel");
  to_float_scaled_kernel<<<dim3(grid_for(mx), ops.count), 256, 0, st>>>(ops, nrm2);
  count_launch();
  check_launch("to_float_scaled_kernel");
}

void to_double_scaled(const float* e, double* out, long long n, const double* nrm2, int count, cudaStream_t st) {
  if (n <= 0) return;
  to_double_scaled_kernel<<<grid_for(n), 256, 0, st>>>(e, out, n, nrm2, count);
  count_launch();
  check_launch("to_double_scaled_kernel");
}

}  // namespace

void to_float(const double* a, float* b, long long n, cudaStream_t st) {
  if (n <= 0) return;
  to_float_kernel<<<grid_for(n), 256, 0, st>>>(a, b, n);
  count_launch();
  check_launch("to_float");
}
void to_double(const float* a, double* b, long long n, cudaStream_t st) {
  if (n <= 0) return;
  to_double_kernel<<<grid_for(n), 256, 0, st>>>(a, b, n);
  count_launch();
  check_launch("to_double");
}

void to_f32(const double* a, float* b, size_t n, cudaStream_t st) { to_float(a, b, (long long)n, st); }
void to_f64(const float* a, double* b, size_t n, cudaStream_t st) { to_double(a, b, (long long)n, st); }

double contract_flops(const CDims& d) {
  double s1 = 2.0 * d.rw * d.R * d.rv * d.n * d.rv2;
  double s2 = 2.0 * d.rw * d.rv2 * (double)(d.R * d.n) * (double)(d.m * d.R2);
  double s3 = 2.0 * d.rw2 * d.R2 * d.rv2 * (double)(d.rw * d.m);
  return s1 + s2 + s3;
}

// ---------------------------------------------------------------------------
// typed implementations
// ---------------------------------------------------------------------------

template <typename T>
static void env_left_t(const CDims& d, const T* phi, const T* u, const T* op, const T* v, T* out,
                       T* t1, T* t2, cudaStream_t st, int prec) {
  const long long rw = d.rw, rw2 = d.rw2, R = d.R, R2 = d.R2, rv = d.rv, rv2 = d.rv2, m = d.m,
                  n = d.n;
  const size_t nphi = rw * R * rv, nu = rw * m * rw2, nop = R * m * n * R2, nv = rv * n * rv2;
  const size_t nt1 = rw * R * n * rv2, nt2 = rw * m * R2 * rv2, nout = rw2 * R2 * rv2;
  // stage 1: T1[a'][p][j][b] = sum_a Phi[a'][p][a] V[a][j][b]
  {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)(rw * R), rv, n * rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)(n * rv2), 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)rv, 1, n * rv2}});
    set_batch(g, {});
    gemm_nd<T>(g, phi, nphi, v, nv, t1, nt1, T(1), T(0), st);
  }
  // stage 2: T2[a'][i][q][b] = sum_{p,j} Op[p][i][j][q] T1[a'][p][j][b]; on the
  // tensor cores T2 comes back as [(i,q)][(a',b)] and stage 3 reads it so
  const bool tc = tc_stage2<T>(prec, rw, R, R2, m, n, rv2, op, t1, t2, st);
  if (!tc) {
    GemmND g;
    set_batch(g, {{(int)rw, 0, R * n * rv2, m * R2 * rv2}});
    set_dim(g.M, g.aM, g.cM, {{(int)m, n * R2, R2 * rv2}, {(int)R2, 1, rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)rv2, 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)R, m * n * R2, n * rv2}, {(int)n, R2, rv2}});
    gemm_nd<T>(g, op, nop, t1, nt1, t2, nt2, T(1), T(0), st);
  }
  // stage 3: out[b'][q][b] = sum_{a',i} U[a'][i][b'] T2[a'][i][q][b]
  if (tc) {
    const long long nc = rw * rv2;  // row stride of the [(i,q)][(a',b)] layout
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw2, 1, R2 * rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)R2, nc, rv2}, {(int)rv2, 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)rw, m * rw2, rv2}, {(int)m, rw2, R2 * nc}});
    set_batch(g, {});
    gemm_nd<T>(g, u, nu, t2, nt2, out, nout, T(1), T(0), st);
  } else {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw2, 1, R2 * rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)(R2 * rv2), 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)(rw * m), rw2, R2 * rv2}});
    set_batch(g, {});
    gemm_nd<T>(g, u, nu, t2, nt2, out, nout, T(1), T(0), st);
  }
}

template <typename T>
static void env_right_t(const CDims& d, const T* psi, const T* u, const T* op, const T* v, T* out,
                        T* t1, T* t2, cudaStream_t st, int prec) {
  const long long rw = d.rw, rw2 = d.rw2, R = d.R, R2 = d.R2, rv = d.rv, rv2 = d.rv2, m = d.m,
                  n = d.n;
  const size_t npsi = rw2 * R2 * rv2, nu = rw * m * rw2, nop = R * m * n * R2, nv = rv * n * rv2;
  const size_t nt1 = rv * n * rw2 * R2, nt2 = rv * R * m * rw2, nout = rw * R * rv;
  // stage 1: T1[a][j][b'][q] = sum_b V[a][j][b] Psi[b'][q][b]
  {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)(rv * n), rv2, rw2 * R2}});
    set_dim(g.N, g.bN, g.cN, {{(int)(rw2 * R2), rv2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)rv2, 1, 1}});
    set_batch(g, {});
    gemm_nd<T>(g, v, nv, psi, npsi, t1, nt1, T(1), T(0), st);
  }
  // stage 2: T2[a][p][i][b'] = sum_{j,q} Op[p][i][j][q] T1[a][j][b'][q]; on the
  // tensor cores T2 comes back as [(p,i)][(a,b')] and stage 3 reads it so
  const bool tc = tc_stage2_right<T>(prec, rv, R, R2, m, n, rw2, op, t1, t2, st);
  if (!tc) {
    GemmND g;
    set_batch(g, {{(int)rv, 0, n * rw2 * R2, R * m * rw2}});
    set_dim(g.M, g.aM, g.cM, {{(int)(R * m), n * R2, rw2}});
    set_dim(g.N, g.bN, g.cN, {{(int)rw2, R2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)n, R2, rw2 * R2}, {(int)R2, 1, 1}});
    gemm_nd<T>(g, op, nop, t1, nt1, t2, nt2, T(1), T(0), st);
  }
  // stage 3: out[a'][p][a] = sum_{i,b'} U[a'][i][b'] T2[a][p][i][b']
  if (tc) {
    const long long nc = rv * rw2;  // row stride of the [(p,i)][(a,b')] layout
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw, m * rw2, R * rv}});
    set_dim(g.N, g.bN, g.cN, {{(int)R, m * nc, rv}, {(int)rv, rw2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)m, rw2, nc}, {(int)rw2, 1, 1}});
    set_batch(g, {});
    gemm_nd<T>(g, u, nu, t2, nt2, out, nout, T(1), T(0), st);
  } else {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw, m * rw2, R * rv}});
    set_dim(g.N, g.bN, g.cN, {{(int)R, m * rw2, rv}, {(int)rv, R * m * rw2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)(m * rw2), 1, 1}});
    set_batch(g, {});
    gemm_nd<T>(g, u, nu, t2, nt2, out, nout, T(1), T(0), st);
  }
}

template <typename T>
static void apply_t(const CDims& d, const T* phi, const T* op, const T* psi, const T* x, T* y,
                    T* t1, T* t2, cudaStream_t st, int prec) {
  const long long rw = d.rw, rw2 = d.rw2, R = d.R, R2 = d.R2, rv = d.rv, rv2 = d.rv2, m = d.m,
                  n = d.n;
  const size_t nphi = rw * R * rv, npsi = rw2 * R2 * rv2, nop = R * m * n * R2, nx = rv * n * rv2;
  const size_t nt1 = rw * R * n * rv2, nt2 = rw * m * R2 * rv2, ny = rw * m * rw2;
  {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)(rw * R), rv, n * rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)(n * rv2), 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)rv, 1, n * rv2}});
    set_batch(g, {});
    gemm_nd<T>(g, phi, nphi, x, nx, t1, nt1, T(1), T(0), st);
  }
  const bool tc = tc_stage2<T>(prec, rw, R, R2, m, n, rv2, op, t1, t2, st);
  if (!tc) {
    GemmND g;
    set_batch(g, {{(int)rw, 0, R * n * rv2, m * R2 * rv2}});
    set_dim(g.M, g.aM, g.cM, {{(int)m, n * R2, R2 * rv2}, {(int)R2, 1, rv2}});
    set_dim(g.N, g.bN, g.cN, {{(int)rv2, 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)R, m * n * R2, n * rv2}, {(int)n, R2, rv2}});
    gemm_nd<T>(g, op, nop, t1, nt1, t2, nt2, T(1), T(0), st);
  }
  // stage 3: y[a'][i][b'] = sum_{q,b} T2[a'][i][q][b] Psi[b'][q][b]
  if (tc) {
    const long long nc = rw * rv2;
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw, rv2, m * rw2}, {(int)m, R2 * nc, rw2}});
    set_dim(g.N, g.bN, g.cN, {{(int)rw2, R2 * rv2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)R2, nc, rv2}, {(int)rv2, 1, 1}});
    set_batch(g, {});
    gemm_nd<T>(g, t2, nt2, psi, npsi, y, ny, T(1), T(0), st);
  } else {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)(rw * m), R2 * rv2, rw2}});
    set_dim(g.N, g.bN, g.cN, {{(int)rw2, R2 * rv2, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)(R2 * rv2), 1, 1}});
    set_batch(g, {});
    gemm_nd<T>(g, t2, nt2, psi, npsi, y, ny, T(1), T(0), st);
  }
}

template <typename T>
static void local_matrix_t(const CDims& d, const T* phi, const T* op, const T* psi, T* out, T* t1,
                           cudaStream_t st) {
  const long long rw = d.rw, rw2 = d.rw2, R = d.R, R2 = d.R2, rv = d.rv, rv2 = d.rv2, m = d.m,
                  n = d.n;
  const long long nloc = rv * n * rv2;
  const size_t nphi = rw * R * rv, npsi = rw2 * R2 * rv2, nop = R * m * n * R2;
  const size_t nt1 = rw * rv * m * n * R2, nout = (size_t)(rw * m * rw2) * nloc;
  // stage 1: T1[a'][a][i][j][q] = sum_p Phi[a'][p][a] Op[p][i][j][q]
  {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw, R * rv, rv * m * n * R2}, {(int)rv, 1, m * n * R2}});
    set_dim(g.N, g.bN, g.cN, {{(int)(m * n * R2), 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)R, rv, m * n * R2}});
    set_batch(g, {});
    gemm_nd<T>(g, phi, nphi, op, nop, t1, nt1, T(1), T(0), st);
  }
  // stage 2: out[(a',i,b')][(a,j,b)] = sum_q Psi[b'][q][b] T1[a'][a][i][j][q]
  {
    GemmND g;
    set_dim(g.M, g.aM, g.cM, {{(int)rw2, R2 * rv2, nloc}, {(int)rv2, 1, 1}});
    set_dim(g.K, g.aK, g.bK, {{(int)R2, rv2, 1}});
    set_dim(g.N, g.bN, g.cN,
            {{(int)rw, rv * m * n * R2, m * rw2 * nloc},
             {(int)m, n * R2, rw2 * nloc},
             {(int)rv, m * n * R2, n * rv2},
             {(int)n, R2, rv2}});
    set_batch(g, {});
    gemm_nd<T>(g, psi, npsi, t1, nt1, out, nout, T(1), T(0), st);
  }
}

// ---------------------------------------------------------------------------
// precision dispatch
// ---------------------------------------------------------------------------

namespace {

struct F32Scratch {
  DBuf<float> a, b, c, d, e, t1, t2;
  DBuf<double> nrm;  // squared Frobenius norms of the scaled operands
};

size_t sz_phi(const CDims& d) { return (size_t)d.rw * d.R * d.rv; }
size_t sz_psi(const CDims& d) { return (size_t)d.rw2 * d.R2 * d.rv2; }
size_t sz_u(const CDims& d) { return (size_t)d.rw * d.m * d.rw2; }
size_t sz_op(const CDims& d) { return (size_t)d.R * d.m * d.n * d.R2; }
size_t sz_v(const CDims& d) { return (size_t)d.rv * d.n * d.rv2; }

void check_prec(int prec) {
  TT_CHECK(prec == TT_FP64 || prec == TT_FP32 || prec == TT_MIXED_TF32 || prec == TT_MIXED_BF16,
           TT_E_INVALID_ARG, "unknown precision");
}

}  // namespace

void env_left_step(const CDims& d, const double* phi, const double* u, const double* op,
                   const double* v, double* out, int prec, cudaStream_t st) {
  check_prec(prec);
  size_t t1n = (size_t)d.rw * d.R * d.n * d.rv2, t2n = (size_t)d.rw * d.m * d.R2 * d.rv2;
  stats_begin(st);
  if (prec == TT_FP64) {
    DBuf<double> t1(t1n), t2(t2n);
    env_left_t<double>(d, phi, u, op, v, out, t1.get(), t2.get(), st, prec);
  } else {
    F32Scratch s;
    s.a.alloc(sz_phi(d)); s.b.alloc(sz_u(d)); s.c.alloc(sz_op(d)); s.d.alloc(sz_v(d));
    s.e.alloc(sz_psi(d)); s.t1.alloc(t1n); s.t2.alloc(t2n); s.nrm.alloc(kMaxOps);
    to_float_scaled(OpSet{{phi, u, op, v}, {s.a.get(), s.b.get(), s.c.get(), s.d.get()},
                          {(long long)sz_phi(d), (long long)sz_u(d), (long long)sz_op(d), (long long)sz_v(d)}, 4},
                    s.nrm.get(), st);
    env_left_t<float>(d, s.a.get(), s.b.get(), s.c.get(), s.d.get(), s.e.get(), s.t1.get(),
                      s.t2.get(), st, prec);
    to_double_scaled(s.e.get(), out, (long long)sz_psi(d), s.nrm.get(), 4, st);
  }
  stats_end(st, contract_flops(d));
}

void env_right_step(const CDims& d, const double* psi, const double* u, const double* op,
                    const double* v, double* out, int prec, cudaStream_t st) {
  check_prec(prec);
  size_t t1n = (size_t)d.rv * d.n * d.rw2 * d.R2, t2n = (size_t)d.rv * d.R * d.m * d.rw2;
  stats_begin(st);
  if (prec == TT_FP64) {
    DBuf<double> t1(t1n), t2(t2n);
    env_right_t<double>(d, psi, u, op, v, out, t1.get(), t2.get(), st, prec);
  } else {
    F32Scratch s;
    s.a.alloc(sz_psi(d)); s.b.alloc(sz_u(d)); s.c.alloc(sz_op(d)); s.d.alloc(sz_v(d));
    s.e.alloc(sz_phi(d)); s.t1.alloc(t1n); s.t2.alloc(t2n); s.nrm.alloc(kMaxOps);
    to_float_scaled(OpSet{{psi, u, op, v}, {s.a.get(), s.b.get(), s.c.get(), s.d.get()},
                          {(long long)sz_psi(d), (long long)sz_u(d), (long long)sz_op(d), (long long)sz_v(d)}, 4},
                    s.nrm.get(), st);
    env_right_t<float>(d, s.a.get(), s.b.get(), s.c.get(), s.d.get(), s.e.get(), s.t1.get(),
                       s.t2.get(), st, prec);
    to_double_scaled(s.e.get(), out, (long long)sz_phi(d), s.nrm.get(), 4, st);
  }
  stats_end(st, contract_flops(d));
}

void local_apply(const CDims& d, const double* phi, const double* op, const double* psi,
                 const double* x, double* y, int prec, cudaStream_t st) {
  check_prec(prec);
  size_t t1n = (size_t)d.rw * d.R * d.n * d.rv2, t2n = (size_t)d.rw * d.m * d.R2 * d.rv2;
  size_t yn = (size_t)d.rw * d.m * d.rw2;
  stats_begin(st);
  if (prec == TT_FP64) {
    DBuf<double> t1(t1n), t2(t2n);
    apply_t<double>(d, phi, op, psi, x, y, t1.get(), t2.get(), st, prec);
  } else {
    F32Scratch s;
    s.a.alloc(sz_phi(d)); s.b.alloc(sz_psi(d)); s.c.alloc(sz_op(d)); s.d.alloc(sz_v(d));
    s.e.alloc(yn); s.t1.alloc(t1n); s.t2.alloc(t2n); s.nrm.alloc(kMaxOps);
    to_float_scaled(OpSet{{phi, psi, op, x}, {s.a.get(), s.b.get(), s.c.get(), s.d.get()},
                          {(long long)sz_phi(d), (long long)sz_psi(d), (long long)sz_op(d), (long long)sz_v(d)}, 4},
                    s.nrm.get(), st);
    apply_t<float>(d, s.a.get(), s.c.get(), s.b.get(), s.d.get(), s.e.get(), s.t1.get(),
                   s.t2.get(), st, prec);
    to_double_scaled(s.e.get(), y, (long long)yn, s.nrm.get(), 4, st);
  }
  stats_end(st, contract_flops(d));
}

void local_matrix(const CDims& d, const double* phi, const double* op, const double* psi,
                  double* out, int prec, cudaStream_t st) {
  check_prec(prec);
  size_t t1n = (size_t)d.rw * d.rv * d.m * d.n * d.R2;
  size_t on = (size_t)d.rw * d.m * d.rw2 * (size_t)d.rv * d.n * d.rv2;
  if (prec == TT_FP64) {
    DBuf<double> t1(t1n);
    local_matrix_t<double>(d, phi, op, psi, out, t1.get(), st);
  } else {
    F32Scratch s;
    s.a.alloc(sz_phi(d)); s.b.alloc(sz_psi(d)); s.c.alloc(sz_op(d));
    s.e.alloc(on); s.t1.alloc(t1n); s.nrm.alloc(kMaxOps);
    to_float_scaled(OpSet{{phi, psi, op, nullptr}, {s.a.get(), s.b.get(), s.c.get(), nullptr},
                          {(long long)sz_phi(d), (long long)sz_psi(d), (long long)sz_op(d), 0}, 3},
                    s.nrm.get(), st);
    local_matrix_t<float>(d, s.a.get(), s.c.get(), s.b.get(), s.e.get(), s.t1.get(), st);
    to_double_scaled(s.e.get(), out, (long long)on, s.nrm.get(), 3, st);
  }
}

// ---------------------------------------------------------------------------
// statistics: one event pair per contraction, resolved lazily
// ---------------------------------------------------------------------------

namespace {
// Each host thread keeps its own records (threads that solve contexts
// concurrently never wait on one another here); readers visit every thread's
// records through a registry.
struct Stats {
  std::mutex mu;  // taken by the owning thread and by readers
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  std::pair<cudaEvent_t, cudaEvent_t> open_ev{nullptr, nullptr};
  bool open = false;
  double flops = 0.0, seconds = 0.0;
  unsigned long long calls = 0;
};
struct Registry {
  std::mutex mu;
  std::vector<std::shared_ptr<Stats>> all[kStatKeys];
};
Registry& registry() {
  static Registry r;
  return r;
}
Stats& stats(int key) {
  static thread_local std::shared_ptr<Stats> mine[kStatKeys];
  std::shared_ptr<Stats>& m = mine[key % kStatKeys];
  if (!m) {
    m = std::make_shared<Stats>();
    Registry& r = registry();
    std::lock_guard<std::mutex> lk(r.mu);
    r.all[key % kStatKeys].push_back(m);
  }
  return *m;
}
void resolve(Stats& s) {
  for (auto& ev : s.pending) {
    TT_CUDA(cudaEventSynchronize(ev.second));
    float ms = 0.f;
    TT_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
    s.seconds += ms * 1e-3;
    s.pool.push_back(ev);
  }
  s.pending.clear();
}
}  // namespace

void stats_begin(cudaStream_t st, int key) {
  Stats& s = stats(key);
  std::lock_guard<std::mutex> lk(s.mu);
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!s.pool.empty()) {
    ev = s.pool.back();
    s.pool.pop_back();
  } else {
    TT_CUDA(cudaEventCreate(&ev.first));
    TT_CUDA(cudaEventCreate(&ev.second));
  }
  if (s.open) s.pool.push_back(s.open_ev);  // a begin without an end (an exception in between)
  TT_CUDA(cudaEventRecord(ev.first, st));
  s.open_ev = ev;
  s.open = true;
}

void stats_end(cudaStream_t st, double flops, int key) {
  Stats& s = stats(key);
  std::lock_guard<std::mutex> lk(s.mu);
  if (!s.open) return;
  TT_CUDA(cudaEventRecord(s.open_ev.second, st));
  s.open = false;
  s.pending.push_back(s.open_ev);
  s.flops += flops;
  ++s.calls;
  if (s.pending.size() > 4096) resolve(s);
}

void stats_read(double* flops, double* seconds, int key, unsigned long long* calls) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  double f = 0.0, sec = 0.0;
  unsigned long long c = 0;
  for (auto& sp : r.all[key % kStatKeys]) {
    std::lock_guard<std::mutex> lk2(sp->mu);
    resolve(*sp);
    f += sp->flops;
    sec += sp->seconds;
    c += sp->calls;
  }
  if (flops) *flops = f;
  if (seconds) *seconds = sec;
  if (calls) *calls = c;
}

void stats_reset() {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  for (int key = 0; key < kStatKeys; ++key)
    for (auto& sp : r.all[key]) {
      std::lock_guard<std::mutex> lk2(sp->mu);
      resolve(*sp);
      sp->flops = 0.0;
      sp->seconds = 0.0;
      sp->calls = 0;
    }
}

}  // namespace ttsdp

// ---------------------------------------------------------------------------
// Allocation-free left environment update.
//
// Some callers cannot allocate device memory while they run: a host
// framework that owns the whole device heap through its own allocator (a
// raw cudaMalloc would bypass its accounting and could fail once the heap is
// handed out), or a latency-critical loop that must not pay for an
// allocation or the device-wide synchronisation cudaFree can imply. For them
// this entry point runs the FP64 left environment update with its two
// intermediate tensors in a fixed file-scope device array instead of
// stream-ordered scratch. The array is created when the library is loaded
// and every device that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace ttsdp {
namespace {

constexpr size_t kNoAllocScratch = size_t(1) << 22;  // doubles (32 MiB)
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

// Host code cannot use g_noalloc_scratch's name as a device address: the
// address is looked up with the calling thread's current device, on every
// call (cheap once the module is loaded), so a context that was reset and
// recreated never sees a stale address.
double* noalloc_scratch_ptr() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) throw TTError(TT_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  return static_cast<double*>(p);
}

}  // namespace

}  // namespace ttsdp

extern "C" tt_status tt_env_left_step_noalloc(const tt_contract_dims* dims, const double* phi, const double* u,
                                              const double* op, const double* v, double* out, void* stream) {
  using namespace ttsdp;
  try {
    TT_CHECK(dims && phi && u && op && v && out, TT_E_INVALID_ARG, "null argument");
    TT_CHECK(dims->rw > 0 && dims->rw2 > 0 && dims->R > 0 && dims->R2 > 0 && dims->rv > 0 && dims->rv2 > 0 &&
                 dims->m > 0 && dims->n > 0,
             TT_E_SHAPE, "dimensions must be positive");
    const CDims d{dims->rw, dims->rw2, dims->R, dims->R2, dims->rv, dims->rv2, dims->m, dims->n};
    const size_t t1n = (size_t)d.rw * d.R * d.n * d.rv2, t2n = (size_t)d.rw * d.m * d.R2 * d.rv2;
    if (t1n + t2n > kNoAllocScratch)
      return TT_E_NOMEM;  // intermediates exceed the fixed scratch (see tt_sdp.h)
    double* s = noalloc_scratch_ptr();
    // both intermediates are written in full before they are read, so the
    // previous call's contents need no clearing
    env_left_t<double>(d, phi, u, op, v, out, s, s + t1n, (cudaStream_t)stream, TT_FP64);
    return TT_OK;
  } catch (const TTError& e) {
    return e.status;
  } catch (...) {
    return TT_E_INTERNAL;
  }
}

