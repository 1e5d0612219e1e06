// TT arithmetic on the device (Sections 2.3 and 3.3): core-wise kernels for
// sums, Kronecker and Hadamard products, operator application and
// diagonalisation; inner products by environment sweeps; TT rounding by
// Householder QR and one-sided Jacobi SVD.
#include <cmath>

#include "gemm.cuh"
#include "linalg.cuh"
#include "rankpred.cuh"
#include "tc_gemm.cuh"
#include "tt.cuh"

namespace ttsdp {

namespace {

int grid1(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  return (int)(g > 152 * 32 ? 152 * 32 : g);
}

#define GRID_LOOP(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void fill_kernel(double* p, long long n, double v) { GRID_LOOP(i, n) p[i] = v; }
__global__ void scale_kernel(double* p, long long n, double s) { GRID_LOOP(i, n) p[i] *= s; }
__global__ void axpy_kernel(double* y, const double* x, long long n, double a) { GRID_LOOP(i, n) y[i] += a * x[i]; }

__global__ void copy2d_kernel(double* dst, long long dld, const double* src, long long sld, int rows,
                              int cols, double alpha) {
  long long n = (long long)rows * cols;
  GRID_LOOP(e, n) {
    long long i = e / cols, j = e % cols;
    dst[i * dld + j] = alpha * src[i * sld + j];
  }
}

__global__ void scale_rows_kernel(double* a, int rows, int cols, const double* s) {
  long long n = (long long)rows * cols;
  GRID_LOOP(e, n) a[e] *= s[e / cols];
}

__global__ void scale_cols_kernel(double* a, int rows, int cols, const double* s) {
  long long n = (long long)rows * cols;
  GRID_LOOP(e, n) a[e] *= s[e % cols];
}

// dst core [R][M][R2], place alpha * src [r][M][r2] at rank offsets (o1, o2)
__global__ void place_kernel(double* dst, int R, int M, int R2, const double* src, int r, int r2,
                             int o1, int o2, double alpha) {
  long long n = (long long)r * M * r2;
  GRID_LOOP(e, n) {
    long long a = e / ((long long)M * r2), rem = e % ((long long)M * r2);
    long long s = rem / r2, b = rem % r2;
    dst[((a + o1) * M + s) * R2 + (b + o2)] = alpha * src[e];
  }
}

// out[(a,x)][s][(b,y)] = A[a][s][b] * B[x][s][y]
__global__ void hadamard_kernel(const double* A, int ra, int ra2, const double* B, int rb, int rb2,
                                int M, double* out) {
  long long n = (long long)ra * rb * M * ra2 * rb2;
  GRID_LOOP(e, n) {
    long long t = e;
    int y = (int)(t % rb2); t /= rb2;
    int b = (int)(t % ra2); t /= ra2;
    int s = (int)(t % M); t /= M;
    int x = (int)(t % rb); t /= rb;
    int a = (int)t;
    out[e] = A[((long long)a * M + s) * ra2 + b] * B[((long long)x * M + s) * rb2 + y];
  }
}

// out[(p,a)][i][(q,b)] = sum_j Op[p][i][j][q] V[a][j][b]
__global__ void matvec_kernel(const double* op, int R, int R2, int m, int n, const double* V, int rv,
                              int rv2, double* out) {
  long long tot = (long long)R * rv * m * R2 * rv2;
  GRID_LOOP(e, tot) {
    long long t = e;
    int b = (int)(t % rv2); t /= rv2;
    int q = (int)(t % R2); t /= R2;
    int i = (int)(t % m); t /= m;
    int a = (int)(t % rv); t /= rv;
    int p = (int)t;
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      s += op[(((long long)p * m + i) * n + j) * R2 + q] * V[((long long)a * n + j) * rv2 + b];
    out[e] = s;
  }
}

// C[(a,x)][(i1,i2)][(j1,j2)][(b,y)] = A[a][i1][j1][b] B[x][i2][j2][y]
__global__ void kron_kernel(const double* A, int ra, int ma, int na, int ra2, const double* B, int rb,
                            int mb, int nb, int rb2, double* out) {
  long long tot = (long long)ra * rb * ma * mb * na * nb * ra2 * rb2;
  GRID_LOOP(e, tot) {
    long long t = e;
    int y = (int)(t % rb2); t /= rb2;
    int b = (int)(t % ra2); t /= ra2;
    int j2 = (int)(t % nb); t /= nb;
    int j1 = (int)(t % na); t /= na;
    int i2 = (int)(t % mb); t /= mb;
    int i1 = (int)(t % ma); t /= ma;
    int x = (int)(t % rb); t /= rb;
    int a = (int)t;
    out[e] = A[(((long long)a * ma + i1) * na + j1) * ra2 + b] * B[(((long long)x * mb + i2) * nb + j2) * rb2 + y];
  }
}

__global__ void transpose_core_kernel(const double* A, int r, int m, int n, int r2, double* out) {
  long long tot = (long long)r * m * n * r2;
  GRID_LOOP(e, tot) {
    long long t = e;
    int b = (int)(t % r2); t /= r2;
    int i = (int)(t % m); t /= m;   // out index order [a][j][i][b]: here i is the new column mode
    int j = (int)(t % n); t /= n;
    int a = (int)t;
    out[e] = A[(((long long)a * m + i) * n + j) * r2 + b];
  }
}

// out[p][(i1 i2)][(j1 j2)][q] = sum_s A[p][i1][j1][s] B[s][i2][j2][q]
__global__ void merge_cores_kernel(const double* A, int R, int m1, int n1, int S, const double* B, int m2,
                                   int n2, int R2, double* out) {
  long long tot = (long long)R * m1 * m2 * n1 * n2 * R2;
  GRID_LOOP(e, tot) {
    long long t = e;
    int q = (int)(t % R2); t /= R2;
    int j2 = (int)(t % n2); t /= n2;
    int j1 = (int)(t % n1); t /= n1;
    int i2 = (int)(t % m2); t /= m2;
    int i1 = (int)(t % m1); t /= m1;
    int p = (int)t;
    const double* a = A + (((long long)p * m1 + i1) * n1 + j1) * S;
    const double* b = B + ((long long)i2 * n2 + j2) * R2 + q;
    const long long bs = (long long)m2 * n2 * R2;
    double acc = 0.0;
    for (int x = 0; x < S; ++x) acc += a[x] * b[x * bs];
    out[e] = acc;
  }
}

__global__ void diag_core_kernel(const double* v, int r, int m, int r2, double* out) {
  long long tot = (long long)r * m * m * r2;
  GRID_LOOP(e, tot) {
    long long t = e;
    int b = (int)(t % r2); t /= r2;
    int j = (int)(t % m); t /= m;
    int i = (int)(t % m); t /= m;
    int a = (int)t;
    out[e] = i == j ? v[((long long)a * m + i) * r2 + b] : 0.0;
  }
}

// out[vec_TT position] = M[row][col] for an n^d x n^d row-major matrix
__global__ void vec_tt_perm_kernel(const double* M, int d, int n, long long N, double* out) {
  long long tot = N * N;
  GRID_LOOP(pos, tot) {
    long long rem = pos, row = 0, col = 0, w = 1;
    for (int k = d - 1; k >= 0; --k) {  // digits from least significant: (a_k, b_k) pairs
      long long b = rem % n;
      rem /= n;
      long long a = rem % n;
      rem /= n;
      row += a * w;
      col += b * w;
      w *= n;
    }
    out[pos] = M[row * N + col];
  }
}

// out[i] = <V_i, w> for the nvec rows V_i of a row-major nvec x N matrix; one CTA per row
__global__ void multi_dot_kernel(const double* __restrict__ V, long long N, const double* __restrict__ w,
                                 double* out) {
  __shared__ double red[32];
  const double* v = V + (long long)blockIdx.x * N;
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) s += v[i] * w[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    out[blockIdx.x] = t;
  }
}

// part[row][blockIdx.x] = partial <V_row, w> over a fixed strided slice
__global__ void multi_dot_split_kernel(const double* __restrict__ V, long long N, const double* __restrict__ w,
                                       double* __restrict__ part) {
  __shared__ double red[32];
  const double* v = V + (long long)blockIdx.y * N;
  double s = 0.0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    if (i < N) s += v[i] * w[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// out[row] = sum of part[row][0..G) in index order (one warp per row)
__global__ void sum_rows_kernel(const double* __restrict__ part, int G, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int g = 0; g < G; ++g) t += part[(long long)blockIdx.x * G + g];
    out[blockIdx.x] = t;
  }
}

// <a, b> by one block; with b == nullptr and n = -count: the plain sum of a[0..count)
__global__ void dot_kernel(const double* a, const double* b, long long n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  if (b) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  } else {
    for (long long i = threadIdx.x; i < -n; i += blockDim.x) s += a[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// Partial sums of a long dot product: block b sums the strided slice
// b, b + G, b + 2G, ... of 1024-element chunks into part[b]; a fixed
// partition, so the result does not depend on scheduling.
__global__ void dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                   double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    if (i < n) s += a[i] * b[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
void dev_fill(double* p, size_t n, double v, cudaStream_t st) {
  if (!n) return;
  fill_kernel<<<grid1(n), 256, 0, st>>>(p, n, v);
  count_launch();
  check_launch("fill");
}
void dev_scale(double* p, size_t n, double s, cudaStream_t st) {
  if (!n) return;
  scale_kernel<<<grid1(n), 256, 0, st>>>(p, n, s);
  count_launch();
  check_launch("scale");
}
void dev_axpy(double* y, const double* x, size_t n, double a, cudaStream_t st) {
  if (!n) return;
  axpy_kernel<<<grid1(n), 256, 0, st>>>(y, x, n, a);
  count_launch();
  check_launch("axpy");
}
void dev_copy(double* dst, const double* src, size_t n, cudaStream_t st) {
  if (!n) return;
  TT_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
}
void dev_copy2d(double* dst, long long dld, const double* src, long long sld, int rows, int cols,
                double alpha, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  copy2d_kernel<<<grid1((long long)rows * cols), 256, 0, st>>>(dst, dld, src, sld, rows, cols, alpha);
  count_launch();
  check_launch("copy2d");
}
void dev_scale_rows(double* a, int rows, int cols, const double* s, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  scale_rows_kernel<<<grid1((long long)rows * cols), 256, 0, st>>>(a, rows, cols, s);
  count_launch();
  check_launch("scale_rows");
}
void dev_scale_cols(double* a, int rows, int cols, const double* s, cudaStream_t st) {
  if ((long long)rows * cols == 0) return;
  scale_cols_kernel<<<grid1((long long)rows * cols), 256, 0, st>>>(a, rows, cols, s);
  count_launch();
  check_launch("scale_cols");
}
void dev_multi_dot(const double* V, int nvec, size_t N, const double* w, double* out, cudaStream_t st) {
  if (nvec <= 0) return;
  if (N < (size_t(1) << 16) || nvec >= 152) {
    multi_dot_kernel<<<nvec, 512, 0, st>>>(V, (long long)N, w, out);
    count_launch();
  } else {
    // few long vectors: split every row over G blocks, then add the partials
    // of each row in a fixed order
    const long long chunks = ((long long)N + 511) / 512;
    const int G = (int)std::min<long long>(chunks, std::max(1, 304 / nvec));
    DBuf<double> part((size_t)nvec * G);
    multi_dot_split_kernel<<<dim3(G, nvec), 512, 0, st>>>(V, (long long)N, w, part.get());
    sum_rows_kernel<<<nvec, 32, 0, st>>>(part.get(), G, out);
    count_launch();
    count_launch();
  }
  check_launch("multi_dot");
}

void dev_dot_async(const double* a, const double* b, size_t n, double* out, cudaStream_t st) {
  if (n < (size_t(1) << 16)) {
    dot_kernel<<<1, 1024, 0, st>>>(a, b, (long long)n, out);
    count_launch();
  } else {
    // long vectors (GMRES bases of large local systems): partial sums on many
    // SMs, then one block adds them in a fixed order
    const long long chunks = ((long long)n + 1023) / 1024;
    const int G = (int)(chunks < 304 ? chunks : 304);
    DBuf<double> part((size_t)G);
    dot_partial_kernel<<<G, 1024, 0, st>>>(a, b, (long long)n, part.get());
    dot_kernel<<<1, 1024, 0, st>>>(part.get(), nullptr, -(long long)G, out);
    count_launch();
    count_launch();
  }
  check_launch("dot");
}

double dev_dot(const double* a, const double* b, size_t n, cudaStream_t st) {
  DBuf<double> out(1);
  dev_dot_async(a, b, n, out.get(), st);
  double h = 0.0;
  TT_CUDA(cudaMemcpyAsync(&h, out.get(), sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  return h;
}

// ---------------------------------------------------------------------------
// containers
// ---------------------------------------------------------------------------
DTT tt_alloc(int d, const std::vector<int>& r, int m, int n) {
  DTT t;
  t.d = d;
  t.m = m;
  t.n = n;
  t.r = r;
  t.c.resize(d);
  for (int k = 0; k < d; ++k) t.c[k] = std::make_shared<DBuf<double>>(t.csize(k));
  return t;
}

static DTT tt_from_ptr(int d, const int* ranks, int m, int n, const double* cores, cudaMemcpyKind kind) {
  TT_CHECK(d > 0 && ranks && cores, TT_E_INVALID_ARG, "bad TT descriptor");
  TT_CHECK(ranks[0] == 1 && ranks[d] == 1, TT_E_SHAPE, "boundary ranks must be 1");
  std::vector<int> r(ranks, ranks + d + 1);
  for (int v : r) TT_CHECK(v > 0, TT_E_SHAPE, "ranks must be positive");
  DTT t = tt_alloc(d, r, m, n);
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    TT_CUDA(cudaMemcpyAsync(t.core(k), cores + off, t.csize(k) * sizeof(double), kind, cur_stream()));
    off += t.csize(k);
  }
  return t;
}

DTT tt_from_host(int d, const int* ranks, int m, int n, const double* cores) {
  return tt_from_ptr(d, ranks, m, n, cores, cudaMemcpyHostToDevice);
}
DTT tt_from_device(int d, const int* ranks, int m, int n, const double* cores) {
  return tt_from_ptr(d, ranks, m, n, cores, cudaMemcpyDeviceToDevice);
}

void tt_to_host(const DTT& a, double* out) {
  size_t off = 0;
  for (int k = 0; k < a.d; ++k) {
    TT_CUDA(cudaMemcpyAsync(out + off, a.core(k), a.csize(k) * sizeof(double), cudaMemcpyDeviceToHost,
                            cur_stream()));
    off += a.csize(k);
  }
  TT_CUDA(sync_stream(cur_stream()));
}

void tt_to_device(const DTT& a, double* out) {
  size_t off = 0;
  for (int k = 0; k < a.d; ++k) {
    dev_copy(out + off, a.core(k), a.csize(k), cur_stream());
    off += a.csize(k);
  }
}

DTT tt_copy(const DTT& a) {
  DTT t = tt_alloc(a.d, a.r, a.m, a.n);
  for (int k = 0; k < a.d; ++k) dev_copy(t.core(k), a.core(k), a.csize(k), cur_stream());
  return t;
}

DTT tt_add(const DTT& a, const DTT& b, double alpha, double beta) {
  TT_CHECK(a.d == b.d && a.m * a.n == b.m * b.n, TT_E_SHAPE, "tt_add: mismatched shapes");
  const int d = a.d, M = a.m * a.n;
  std::vector<int> r(d + 1);
  r[0] = r[d] = 1;
  for (int k = 1; k < d; ++k) r[k] = a.r[k] + b.r[k];
  DTT t = tt_alloc(d, r, a.m, a.n);
  cudaStream_t st = cur_stream();
  for (int k = 0; k < d; ++k) {
    double* dst = t.core(k);
    size_t n = t.csize(k);
    if (d == 1) {
      dev_fill(dst, n, 0.0, st);
      dev_axpy(dst, a.core(k), n, alpha, st);
      dev_axpy(dst, b.core(k), n, beta, st);
      continue;
    }
    dev_fill(dst, n, 0.0, st);
    int R = r[k], R2 = r[k + 1];
    int oa1 = 0, oa2 = 0, ob1 = (k == 0) ? 0 : a.r[k], ob2 = (k == d - 1) ? 0 : a.r[k + 1];
    double sa = k == 0 ? alpha : 1.0, sb = k == 0 ? beta : 1.0;
    long long na = a.csize(k), nb = b.csize(k);
    place_kernel<<<grid1(na), 256, 0, st>>>(dst, R, M, R2, a.core(k), a.r[k], a.r[k + 1], oa1, oa2, sa);
    count_launch();
    place_kernel<<<grid1(nb), 256, 0, st>>>(dst, R, M, R2, b.core(k), b.r[k], b.r[k + 1], ob1, ob2, sb);
    count_launch();
  }
  check_launch("tt_add");
  return t;
}

DTT tt_scale(const DTT& a, double s) {
  DTT t = a;
  t.c[0] = std::make_shared<DBuf<double>>(a.csize(0));
  dev_copy(t.core(0), a.core(0), a.csize(0), cur_stream());
  dev_scale(t.core(0), a.csize(0), s, cur_stream());
  return t;
}

DTT tt_transpose(const DTT& a) {
  DTT t = tt_alloc(a.d, a.r, a.n, a.m);
  for (int k = 0; k < a.d; ++k) {
    long long n = a.csize(k);
    transpose_core_kernel<<<grid1(n), 256, 0, cur_stream()>>>(a.core(k), a.r[k], a.m, a.n, a.r[k + 1],
                                                              t.core(k));
    count_launch();
  }
  check_launch("tt_transpose");
  return t;
}

DTT tt_sym(const DTT& a) { return tt_add(a, tt_transpose(a), 0.5, 0.5); }

DTT tt_kron(const DTT& a, const DTT& b) {
  TT_CHECK(a.d == b.d, TT_E_SHAPE, "tt_kron: order mismatch");
  std::vector<int> r(a.d + 1);
  for (int k = 0; k <= a.d; ++k) r[k] = a.r[k] * b.r[k];
  DTT t = tt_alloc(a.d, r, a.m * b.m, a.n * b.n);
  for (int k = 0; k < a.d; ++k) {
    long long n = t.csize(k);
    kron_kernel<<<grid1(n), 256, 0, cur_stream()>>>(a.core(k), a.r[k], a.m, a.n, a.r[k + 1], b.core(k),
                                                    b.r[k], b.m, b.n, b.r[k + 1], t.core(k));
    count_launch();
  }
  check_launch("tt_kron");
  return t;
}

DTT tt_hadamard(const DTT& a, const DTT& b) {
  TT_CHECK(a.d == b.d && a.m * a.n == b.m * b.n, TT_E_SHAPE, "tt_hadamard: mismatched shapes");
  std::vector<int> r(a.d + 1);
  for (int k = 0; k <= a.d; ++k) r[k] = a.r[k] * b.r[k];
  DTT t = tt_alloc(a.d, r, a.m, a.n);
  for (int k = 0; k < a.d; ++k) {
    long long n = t.csize(k);
    hadamard_kernel<<<grid1(n), 256, 0, cur_stream()>>>(a.core(k), a.r[k], a.r[k + 1], b.core(k), b.r[k],
                                                        b.r[k + 1], a.m * a.n, t.core(k));
    count_launch();
  }
  check_launch("tt_hadamard");
  return t;
}

DTT tt_matvec(const DTT& op, const DTT& v) {
  TT_CHECK(op.d == v.d && op.n == v.m * v.n, TT_E_SHAPE, "tt_matvec: mismatched shapes");
  std::vector<int> r(op.d + 1);
  for (int k = 0; k <= op.d; ++k) r[k] = op.r[k] * v.r[k];
  DTT t = tt_alloc(op.d, r, op.m, 1);
  for (int k = 0; k < op.d; ++k) {
    long long n = t.csize(k);
    matvec_kernel<<<grid1(n), 256, 0, cur_stream()>>>(op.core(k), op.r[k], op.r[k + 1], op.m, op.n,
                                                      v.core(k), v.r[k], v.r[k + 1], t.core(k));
    count_launch();
  }
  check_launch("tt_matvec");
  return t;
}

std::shared_ptr<DBuf<double>> tt_merge_cores(const DTT& op, int k) {
  TT_CHECK(k >= 0 && k + 1 < op.d, TT_E_INVALID_ARG, "tt_merge_cores: bond out of range");
  const int R = op.r[k], S = op.r[k + 1], R2 = op.r[k + 2];
  const long long tot = (long long)R * op.m * op.m * op.n * op.n * R2;
  auto out = std::make_shared<DBuf<double>>((size_t)tot);
  cudaStream_t st = cur_stream();
  merge_cores_kernel<<<grid1(tot), 256, 0, st>>>(op.core(k), R, op.m, op.n, S, op.core(k + 1), op.m, op.n, R2,
                                                 out->get());
  count_launch();
  check_launch("merge_cores_kernel");
  return out;
}

namespace {
// out[p][i][q] = op[p][i][i][q]
__global__ void op_diag_kernel(const double* __restrict__ op, int R, int m, int R2, double* __restrict__ out) {
  const long long tot = (long long)R * m * R2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long q = e % R2, i = (e / R2) % m, p = e / ((long long)R2 * m);
    out[e] = op[((p * m + i) * m + i) * R2 + q];
  }
}
}  // namespace

DTT tt_op_diag(const DTT& op) {
  TT_CHECK(op.m == op.n, TT_E_SHAPE, "tt_op_diag: square modes expected");
  DTT t = tt_alloc(op.d, op.r, op.m, 1);
  for (int k = 0; k < op.d; ++k) {
    const long long n = t.csize(k);
    op_diag_kernel<<<grid1(n), 256, 0, cur_stream()>>>(op.core(k), op.r[k], op.m, op.r[k + 1], t.core(k));
    count_launch();
  }
  check_launch("tt_op_diag");
  return t;
}

bool tt_is_diag_op(const DTT& op) {
  if (op.m != op.n) return false;
  const double all = tt_inner(op, op), dg = tt_norm(tt_op_diag(op));
  return std::fabs(all - dg * dg) <= 1e-12 * std::max(all, 1e-300);
}

DTT tt_diag(const DTT& v) {
  int M = v.m * v.n;
  DTT t = tt_alloc(v.d, v.r, M, M);
  for (int k = 0; k < v.d; ++k) {
    long long n = t.csize(k);
    diag_core_kernel<<<grid1(n), 256, 0, cur_stream()>>>(v.core(k), v.r[k], M, v.r[k + 1], t.core(k));
    count_launch();
  }
  check_launch("tt_diag");
  return t;
}

DTT tt_identity(int d, int m) {
  DTT t = tt_alloc(d, std::vector<int>(d + 1, 1), m, m);
  std::vector<double> h((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) h[(size_t)i * m + i] = 1.0;
  for (int k = 0; k < d; ++k)
    TT_CUDA(cudaMemcpyAsync(t.core(k), h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
  return t;
}

DTT tt_ones_mat(int d, int m) {
  DTT t = tt_alloc(d, std::vector<int>(d + 1, 1), m, m);
  for (int k = 0; k < d; ++k) dev_fill(t.core(k), t.csize(k), 1.0, cur_stream());
  return t;
}

DTT tt_zeros_like_modes(int d, int m, int n) {
  DTT t = tt_alloc(d, std::vector<int>(d + 1, 1), m, n);
  for (int k = 0; k < d; ++k) dev_fill(t.core(k), t.csize(k), 0.0, cur_stream());
  return t;
}

double tt_inner(const DTT& a, const DTT& b) {
  TT_CHECK(a.d == b.d && a.m * a.n == b.m * b.n, TT_E_SHAPE, "tt_inner: mismatched shapes");
  const int M = a.m * a.n;
  cudaStream_t st = cur_stream();
  DBuf<double> phi(1);
  dev_fill(phi.get(), 1, 1.0, st);
  for (int k = 0; k < a.d; ++k) {
    long long ra = a.r[k], ra2 = a.r[k + 1], rb = b.r[k], rb2 = b.r[k + 1];
    DBuf<double> t1((size_t)ra * M * rb2);
    {  // T1[a][s][y] = sum_x Phi[a][x] B[x][s][y]
      GemmND g;
      set_dim(g.M, g.aM, g.cM, {{(int)ra, rb, M * rb2}});
      set_dim(g.N, g.bN, g.cN, {{(int)(M * rb2), 1, 1}});
      set_dim(g.K, g.aK, g.bK, {{(int)rb, 1, M * rb2}});
      set_batch(g, {});
      gemm_nd<double>(g, phi.get(), phi.size(), b.core(k), b.csize(k), t1.get(), t1.size(), 1.0, 0.0, st);
    }
    DBuf<double> nphi((size_t)ra2 * rb2);
    {  // Phi'[b][y] = sum_{a,s} A[a][s][b] T1[a][s][y]
      GemmND g;
      set_dim(g.M, g.aM, g.cM, {{(int)ra2, 1, rb2}});
      set_dim(g.N, g.bN, g.cN, {{(int)rb2, 1, 1}});
      set_dim(g.K, g.aK, g.bK, {{(int)(ra * M), ra2, rb2}});
      set_batch(g, {});
      gemm_nd<double>(g, a.core(k), a.csize(k), t1.get(), t1.size(), nphi.get(), nphi.size(), 1.0, 0.0, st);
    }
    phi = std::move(nphi);
  }
  double h = 0.0;
  TT_CUDA(cudaMemcpyAsync(&h, phi.get(), sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  return h;
}

double tt_norm(const DTT& a) {
  double v = tt_inner(a, a);
  return v > 0 ? std::sqrt(v) : 0.0;
}

// ---------------------------------------------------------------------------
// orthogonalisation and rounding
// ---------------------------------------------------------------------------
DTT tt_orth_right(const DTT& a) {
  const int d = a.d, M = a.m * a.n;
  cudaStream_t st = cur_stream();
  DTT t = tt_copy(a);
  for (int k = d - 1; k >= 1; --k) {
    int r = t.r[k], r2 = t.r[k + 1];
    int rows = M * r2;  // the transposed unfolding is (M r2) x r
    int kk = rows < r ? rows : r;
    DBuf<double> Q((size_t)rows * kk), R((size_t)kk * r);
    MatView<double> v{t.core(k), rows, r, 1, (long long)M * r2};
    qr_thin<double>(v, Q.get(), R.get(), st);
    auto nc = std::make_shared<DBuf<double>>((size_t)kk * rows);
    transpose<double>(rows, kk, Q.get(), nc->get(), st);  // core_k = Q^T
    // core_{k-1} (r_{k-1} M x r) <- core_{k-1} R^T
    int rp = t.r[k - 1];
    auto pc = std::make_shared<DBuf<double>>((size_t)rp * M * kk);
    gemm_rm<double>(false, true, rp * M, kk, r, 1.0, t.core(k - 1), r, 0, R.get(), r, 0, 0.0, pc->get(),
                    kk, 0, 1, st);
    t.c[k] = nc;
    t.c[k - 1] = pc;
    t.r[k] = kk;
  }
  return t;
}

DTT tt_from_dense(const double* dense, int d, int n, double eps_rel, int cap) {
  TT_CHECK(d >= 1 && n >= 1 && dense, TT_E_INVALID_ARG, "tt_from_dense: bad arguments");
  cudaStream_t st = cur_stream();
  long long N = 1;
  for (int k = 0; k < d; ++k) N *= n;
  const long long tot = N * N;
  const int M = n * n;
  auto cur = std::make_shared<DBuf<double>>((size_t)tot);
  vec_tt_perm_kernel<<<grid1(tot), 256, 0, st>>>(dense, d, n, N, cur->get());
  count_launch();
  check_launch("vec_tt_perm");
  const double nrm = std::sqrt(std::max(0.0, dev_dot(cur->get(), cur->get(), (size_t)tot, st)));
  const double thr = eps_rel * nrm / std::sqrt((double)(d > 1 ? d - 1 : 1));
  std::vector<int> r(d + 1, 1);
  std::vector<std::shared_ptr<DBuf<double>>> cores(d);
  long long rest = tot;
  for (int k = 0; k + 1 < d; ++k) {
    const int rows = r[k] * M;
    rest /= M;
    const long long cols = rest;
    const int kk = (int)std::min<long long>(rows, cols);
    DBuf<double> U((size_t)rows * kk), S((size_t)kk), Vt((size_t)kk * cols);
    svd_thin<double>(MatView<double>{cur->get(), rows, (int)cols, cols, 1}, U.get(), S.get(), Vt.get(), st);
    std::vector<double> hs(kk);
    TT_CUDA(cudaMemcpyAsync(hs.data(), S.get(), kk * sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    const int keep = truncation_rank(hs, thr, cap);
    cores[k] = std::make_shared<DBuf<double>>((size_t)rows * keep);
    dev_copy2d(cores[k]->get(), keep, U.get(), kk, rows, keep, 1.0, st);
    dev_scale_rows(Vt.get(), keep, (int)cols, S.get(), st);
    auto nxt = std::make_shared<DBuf<double>>((size_t)keep * cols);
    dev_copy(nxt->get(), Vt.get(), (size_t)keep * cols, st);
    cur = nxt;
    r[k + 1] = keep;
  }
  cores[d - 1] = cur;
  DTT t;
  t.d = d;
  t.m = n;
  t.n = n;
  t.r = r;
  t.c = cores;
  return t;
}

int truncation_rank(const std::vector<double>& s, double thr, int cap) {
  const double thr2 = thr * thr;
  double tail = 0.0;
  int keep = (int)s.size();
  for (int j = (int)s.size() - 1; j >= 1; --j) {
    if (tail + s[j] * s[j] <= thr2) {
      tail += s[j] * s[j];
      keep = j;
    } else {
      break;
    }
  }
  if (keep < 1) keep = 1;
  if (cap > 0 && keep > cap) keep = cap;
  return keep;
}

// Features of the learned rank predictor for bond k (10 values): one-hot variable,
// bond position, log10(mu) / 10, input rank / cap, previous rank / cap, iteration
// fraction, and the singular-value decay of this bond at the previous rounding.
static void bond_features(const RoundHook& h, int k, int d, int in_rank, int cap, float* f) {
  for (int i = 0; i < 4; ++i) f[i] = (h.var_id == i) ? 1.f : 0.f;
  f[4] = d > 2 ? (float)k / (float)(d - 2) : 0.f;
  f[5] = (float)(std::log10(std::max(h.mu, 1e-300)) / 10.0);
  f[6] = (float)in_rank / (float)std::max(cap, 1);
  const int prev = h.prev && (int)h.prev->size() > k + 1 ? (*h.prev)[k + 1] : 0;
  f[7] = (float)prev / (float)std::max(cap, 1);
  f[8] = (float)h.iter_frac;
  f[9] = h.decay && (int)h.decay->size() > k + 1 ? (*h.decay)[k + 1] : 0.f;
}

// log10(sigma_keep / sigma_1) / 16 of a bond's spectrum at its kept rank
static float spectrum_decay(const std::vector<double>& s, int keep) {
  if (s.empty() || s[0] <= 0.0 || keep < 1) return 0.f;
  const double last = s[(size_t)std::min<int>(keep, (int)s.size()) - 1];
  return (float)(std::log10(std::max(last, 1e-300) / s[0]) / 16.0);
}

// One bond by the fixed-rank randomised range finder (Halko, Martinsson & Tropp
// 2011): Y = A Omega on the TF32 tensor cores, Q = qr(Y), B = Q^T A and the SVD
// of the small B in FP64. The exact FP64 truncation error ||A||^2 - sum of the
// kept sigma^2 must stay within the bond threshold, otherwise the caller falls
// back to the adaptive SVD. Returns the kept rank (0: rejected).
static int round_bond_sketch(DTT& t, int k, int l, double thr, int cap, Counter& rnd, double* err2,
                             float* decay) {
  cudaStream_t st = cur_stream();
  const int M = t.m * t.n, r = t.r[k], r2 = t.r[k + 1], rows = r * M;
  const double* A = t.core(k);
  DBuf<double> Om((size_t)l * r2), Y((size_t)rows * l), Q((size_t)rows * l), Rq((size_t)l * l), Bm((size_t)l * r2);
  {
    std::vector<double> h = rnd.draw((size_t)l * r2);
    TT_CUDA(cudaMemcpyAsync(Om.get(), h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    TT_CUDA(sync_stream(st));
  }
  tc_gemm_f64_tn(rows, l, r2, A, r2, Om.get(), r2, Y.get(), st);  // Y = A Omega, Omega^T stored l x r2
  qr_thin<double>(MatView<double>{Y.get(), rows, l, l, 1}, Q.get(), Rq.get(), st);
  gemm_rm<double>(true, false, l, r2, rows, 1.0, Q.get(), l, 0, A, r2, 0, 0.0, Bm.get(), r2, 0, 1, st);
  const int kk = std::min(l, r2);
  DBuf<double> UB((size_t)l * kk), S(kk), Vt((size_t)kk * r2);
  svd_thin<double>(MatView<double>{Bm.get(), l, r2, r2, 1}, UB.get(), S.get(), Vt.get(), st);
  std::vector<double> hs(kk);
  TT_CUDA(cudaMemcpyAsync(hs.data(), S.get(), kk * sizeof(double), cudaMemcpyDeviceToHost, st));
  const double a2 = dev_dot(A, A, (size_t)rows * r2, st);
  double s2 = 0.0;
  for (double v : hs) s2 += v * v;
  const double missing = std::max(a2 - s2, 0.0);
  // smallest rank whose error (missing energy + discarded sigma^2) is within thr^2
  double tail = missing;
  int keep = kk;
  if (tail > thr * thr) return 0;
  for (int j = kk - 1; j >= 1; --j) {
    if (tail + hs[j] * hs[j] <= thr * thr) {
      tail += hs[j] * hs[j];
      keep = j;
    } else {
      break;
    }
  }
  if (cap > 0 && keep > cap) return 0;  // the cap would bind: let the adaptive SVD decide
  // new core = Q UB[:, :keep]; next core = diag(S) Vt[:keep] core_{k+1}
  auto nc = std::make_shared<DBuf<double>>((size_t)rows * keep);
  gemm_rm<double>(false, false, rows, keep, l, 1.0, Q.get(), l, 0, UB.get(), kk, 0, 0.0, nc->get(), keep, 0, 1, st);
  dev_scale_rows(Vt.get(), keep, r2, S.get(), st);
  const int r3 = t.r[k + 2];
  auto xc = std::make_shared<DBuf<double>>((size_t)keep * M * r3);
  gemm_rm<double>(false, false, keep, M * r3, r2, 1.0, Vt.get(), r2, 0, t.core(k + 1), M * r3, 0, 0.0, xc->get(),
                  M * r3, 0, 1, st);
  t.c[k] = nc;
  t.c[k + 1] = xc;
  t.r[k + 1] = keep;
  *err2 = tail;
  *decay = spectrum_decay(hs, keep);
  return keep;
}

std::pair<DTT, double> tt_round(const DTT& a, double delta, int cap, RoundHook* hook) {
  const int d = a.d, M = a.m * a.n;
  cudaStream_t st = cur_stream();
  DTT t;
  {
    ProfScope ps("round.orth");
    t = tt_orth_right(a);
  }
  ProfScope ps_trunc("round.trunc");
  const double thr = delta / std::sqrt((double)(d > 1 ? d - 1 : 1));
  double zeta2 = 0.0;
  // features and predicted ranks of all bonds (one MLP evaluation)
  std::vector<float> feats;
  std::vector<float> pred;
  if (hook && d > 1 && (hook->pred || hook->trace_x)) {
    feats.resize((size_t)(d - 1) * kPredIn);
    for (int k = 0; k + 1 < d; ++k) bond_features(*hook, k, d, t.r[k + 1], cap, &feats[(size_t)k * kPredIn]);
    if (hook->pred) pred = hook->pred->predict(feats, d - 1);
  }
  for (int k = 0; k + 1 < d; ++k) {
    int r = t.r[k], r2 = t.r[k + 1];
    int rows = r * M;
    int kk = rows < r2 ? rows : r2;
    if (!pred.empty() && hook->rnd) {
      const int rh = std::max(1, (int)std::ceil(pred[k] * std::max(cap, 1)));
      const int l = std::min(rh + 4, kk);
      if (l < kk) {
        double e2 = 0.0;
        float dec = 0.f;
        const int kept = round_bond_sketch(t, k, l, thr, cap, *hook->rnd, &e2, &dec);
        if (kept > 0) {
          zeta2 += e2;
          ++hook->used;
          if (hook->prev && (int)hook->prev->size() > k + 1) (*hook->prev)[k + 1] = kept;
          if (hook->decay && (int)hook->decay->size() > k + 1) (*hook->decay)[k + 1] = dec;
          continue;
        }
        ++hook->fallbacks;
      }
    }
    DBuf<double> U((size_t)rows * kk), S((size_t)kk), Vt((size_t)kk * r2);
    MatView<double> v{t.core(k), rows, r2, r2, 1};
    {
      ProfScope ps("round.svd");
      svd_thin<double>(v, U.get(), S.get(), Vt.get(), st, kSvdLeft);
    }
    std::vector<double> hs(kk);
    TT_CUDA(cudaMemcpyAsync(hs.data(), S.get(), kk * sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    int keep = truncation_rank(hs, thr, cap);
    for (int j = keep; j < kk; ++j) zeta2 += hs[j] * hs[j];
    if (hook && hook->trace_x && !feats.empty()) {  // the adaptive SVD's choice is the label
      hook->trace_x->insert(hook->trace_x->end(), feats.begin() + (size_t)k * kPredIn,
                            feats.begin() + (size_t)(k + 1) * kPredIn);
      hook->trace_y->push_back((float)keep / (float)std::max(cap, 1));
    }
    if (hook && hook->prev && (int)hook->prev->size() > k + 1) (*hook->prev)[k + 1] = keep;
    if (hook && hook->decay && (int)hook->decay->size() > k + 1) (*hook->decay)[k + 1] = spectrum_decay(hs, keep);
    auto nc = std::make_shared<DBuf<double>>((size_t)rows * keep);
    dev_copy2d(nc->get(), keep, U.get(), kk, rows, keep, 1.0, st);
    // next core <- diag(S[:keep]) Vt[:keep] core_{k+1}, with diag(S) Vt = U^T A
    gemm_rm<double>(true, false, keep, r2, rows, 1.0, U.get(), kk, 0, t.core(k), r2, 0, 0.0, Vt.get(), r2, 0, 1,
                    st);
    int r3 = t.r[k + 2];
    auto xc = std::make_shared<DBuf<double>>((size_t)keep * M * r3);
    gemm_rm<double>(false, false, keep, M * r3, r2, 1.0, Vt.get(), r2, 0, t.core(k + 1), M * r3, 0, 0.0,
                    xc->get(), M * r3, 0, 1, st);
    t.c[k] = nc;
    t.c[k + 1] = xc;
    t.r[k + 1] = keep;
  }
  return {t, std::sqrt(zeta2)};
}

// ---------------------------------------------------------------------------
// SplitMix64 counter stream
// ---------------------------------------------------------------------------
static inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

Counter Counter::fork() {
  Counter c;
  c.seed = splitmix64(seed ^ (n * 0x9E3779B97F4A7C15ULL));
  c.n = 0;
  ++n;
  return c;
}

std::vector<double> Counter::draw(size_t count) {
  std::vector<double> out(count);
  for (size_t j = 0; j < count; ++j) {
    uint64_t x = splitmix64(seed ^ ((n + j) * 0x9E3779B97F4A7C15ULL));
    out[j] = (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  n += count;
  return out;
}

}  // namespace ttsdp
