// Block elimination for the reduced projected Newton system (Section 3.3).
//
// The LZ block is factored by a bordered, right-looking Cholesky that carries
// the right-hand sides E^T and G along: the working matrix is
//   Aug = [ sym(LZ) | E^T | G ]   (n rows, n + 2 nm columns, row-major)
// and each 32-row block step (1) factors the 32 x 32 diagonal block in shared
// memory and overwrites the block row to its right with U11^-T times it
// (which is U12 in the LZ part, and the forward-substituted rows of E^T and G
// in the rest), then (2) updates every row below with one GEMM,
//   Aug[r1:, r1:] -= U12^T Aug[j0:r1, r1:].
// Only the upper triangle of LZ is read, so the factor is that of the
// symmetric part. After the last step the right-hand side columns hold
// W = U^-T E^T and V = U^-T G, and the Schur complement F - W^T V is one GEMM.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "contract.cuh"
#include "gemm.cuh"
#include "kkt.cuh"
#include "linalg.cuh"
#include "tt.cuh"

namespace ttsdp {

namespace {

constexpr int kNb = 32;         // block width of the Cholesky steps
constexpr int kRowThreads = 32;  // one warp per CTA of the block-row kernel

// Aug = [ (LZ + LZ^T) / 2 | E^T | G ], converted to T.
template <typename T>
__global__ void build_aug_kernel(int N, int n, int nm, const double* __restrict__ K, T* __restrict__ aug,
                                 int ld) {
  const long long tot = (long long)n * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), c = (int)(e % ld);
    double v;
    if (c < n) {
      v = 0.5 * (K[(long long)(nm + i) * N + c] + K[(long long)(nm + c) * N + i]);
    } else if (c < n + nm) {
      v = K[(long long)(c - n) * N + i];
    } else {
      v = K[(long long)(nm + i) * N + n + (c - n - nm)];
    }
    aug[e] = (T)v;
  }
}

// One block step of the bordered Cholesky (see the file comment), one warp
// per CTA: every CTA factors the diagonal block [j0, j0 + jb)^2 from its upper
// triangle in shared memory (lane c owns column c), then each lane
// forward-substitutes one column of the block row to the right (columns
// j0 + jb .. ld - 1, the CTAs taking 32 columns each: GB300 issues about two
// FP64 FMAs per clock per SM, so the substitutions must spread over many SMs).
// CTA 0 stores the diagonal of U in dvec and the strictly upper part of U11
// transposed into the block's lower triangle (no CTA reads that half), and
// raises *nonpos on a pivot that is not positive and finite; the step then
// goes on with a unit pivot, so the results stay finite and the caller
// discards them.
template <typename T>
__global__ void __launch_bounds__(kRowThreads, 1) chol_row_kernel(int ld, T* __restrict__ aug,
                                                                  T* __restrict__ dvec, int j0, int jb,
                                                                  int* __restrict__ nonpos) {
  __shared__ T a[kNb][kNb + 1];
  __shared__ T dsh[kNb];
  const int lane = threadIdx.x;
  for (int r = 0; r < kNb; ++r)
    a[r][lane] = (r < jb && lane < jb && r <= lane) ? aug[(long long)(j0 + r) * ld + j0 + lane] : T(0);
  dsh[lane] = T(1);  // rows past jb solve to zero below
  __syncwarp();
  bool bad = false;
  for (int k = 0; k < jb; ++k) {
    T piv = a[k][k];  // final: column k's updates ended at step k - 1
    if (!(piv > T(0)) || !isfinite(piv)) {
      bad = true;
      piv = T(1);
    }
    const T d = sqrt(piv);
    if (lane == 0) dsh[k] = d;
    if (lane > k && lane < jb) a[k][lane] /= d;  // row k of U
    __syncwarp();
    // column c = lane of the trailing upper triangle: a[i][c] -= U[k][i] U[k][c], k < i <= c
    if (lane > k && lane < jb) {
      const T ukc = a[k][lane];
      for (int i = k + 1; i <= lane; ++i) a[i][lane] -= a[k][i] * ukc;
    }
    __syncwarp();
  }
  // U11^T x = y for each column of the block row (column-oriented
  // substitution over all 32 rows with constant indices: x stays in
  // registers; rows past jb read 0 and have a[l][r] = 0, dsh[r] = 1)
  for (long long col = (long long)j0 + jb + blockIdx.x * (long long)kRowThreads + lane; col < ld;
       col += (long long)gridDim.x * kRowThreads) {
    T x[kNb];
#pragma unroll
    for (int r = 0; r < kNb; ++r) x[r] = r < jb ? aug[(long long)(j0 + r) * ld + col] : T(0);
#pragma unroll
    for (int l = 0; l < kNb; ++l) {
      x[l] /= dsh[l];
#pragma unroll
      for (int r = l + 1; r < kNb; ++r) x[r] -= a[l][r] * x[l];
    }
#pragma unroll
    for (int r = 0; r < kNb; ++r)
      if (r < jb) aug[(long long)(j0 + r) * ld + col] = x[r];
  }
  if (blockIdx.x == 0) {
    for (int r = 0; r < lane; ++r)
      if (lane < jb) aug[(long long)(j0 + lane) * ld + j0 + r] = a[r][lane];
    if (lane < jb) dvec[j0 + lane] = dsh[lane];
    if (lane == 0 && bad) *nonpos = 1;
  }
}

// The factor LZ = U^T U written as the factors lu_solve_factored reads for a
// symmetric matrix M = M^T = L' U' with L' = U^T D^-1 (unit lower) and
// U' = D U, D = diag(U), identity interchanges: entry (i, t) of the buffer is
// U[t][i] D[t] for t <= i and U[i][t] / D[i] for t > i.
template <typename T>
__global__ void chol_to_lu_kernel(int n, int ld, const T* __restrict__ aug, const T* __restrict__ dvec,
                                  T* __restrict__ lz) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), t = (int)(e % n);
    const int a = t <= i ? t : i, b = t <= i ? i : t;  // U[a][b], a <= b
    T u;
    if (a == b) u = dvec[a];
    else if ((a / kNb) == (b / kNb)) u = aug[(long long)b * ld + a];
    else u = aug[(long long)a * ld + b];
    lz[e] = t <= i ? u * dvec[t] : u / dvec[i];
  }
}

// S = F = K[0:nm, n:N] converted to T.
template <typename T>
__global__ void copy_f_kernel(int N, int n, int nm, const double* __restrict__ K, T* __restrict__ s) {
  const long long tot = (long long)nm * nm;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nm), j = (int)(e % nm);
    s[e] = (T)K[(long long)i * N + n + j];
  }
}

__global__ void iota_kernel(int n, int* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

inline int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

// out = M^-1 in for factors of type T (interchanges piv, composed in perm,
// diagonal-block inverses dinv); FP64 vectors
template <typename T>
void solve_with(int m, const T* F, const int* piv, const int* perm, const T* dinv, const double* in, double* out,
                cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value) {
    if (out != in) dev_copy(out, in, (size_t)m, st);
    lu_solve_factored<double>(m, F, piv, out, st, perm, dinv);
  } else {
    DBuf<float> v((size_t)m);
    to_f32(in, v.get(), (size_t)m, st);
    lu_solve_factored<float>(m, F, piv, v.get(), st, perm, dinv);
    to_f64(v.get(), out, (size_t)m, st);
  }
}

// aug = [ (M + M^T) / 2 | (D + D^T) / 2 | I ] (n x 3n)
__global__ void build_pencil_aug_kernel(int n, const double* __restrict__ M, const double* __restrict__ D,
                                        double* __restrict__ aug) {
  const long long ld = 3LL * n, tot = (long long)n * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), c = (int)(e % ld);
    double v;
    if (c < n) v = 0.5 * (M[(long long)i * n + c] + M[(long long)c * n + i]);
    else if (c < 2 * n) v = 0.5 * (D[(long long)i * n + c - n] + D[(long long)(c - n) * n + i]);
    else v = (c - 2 * n == i) ? 1.0 : 0.0;
    aug[e] = v;
  }
}

// The bordered Cholesky of the file comment on aug (n rows, ld columns, the
// first n of them the symmetric matrix): returns false when a pivot was not
// positive. dvec receives the diagonal of U.
template <typename T>
bool bordered_cholesky(int n, int ld, T* aug, T* dvec, cudaStream_t st) {
  DBuf<int> bad(1);
  TT_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), st));
  for (int j0 = 0; j0 < n; j0 += kNb) {
    const int jb = std::min(kNb, n - j0), r1 = j0 + jb;
    const int blocks = std::max(1, std::min(ceil_div(ld - r1, kRowThreads), 152 * 8));
    chol_row_kernel<T><<<blocks, kRowThreads, 0, st>>>(ld, aug, dvec, j0, jb, bad.get());
    count_launch();
    if (r1 < n) {
      T* row = aug + (size_t)j0 * ld + r1;
      gemm_rm<T>(true, false, n - r1, ld - r1, jb, T(-1), row, ld, 0, row, ld, 0, T(1), aug + (size_t)r1 * ld + r1,
                 ld, 0, 1, st);
    }
  }
  check_launch("bordered cholesky");
  int hbad = 0;
  TT_CUDA(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  return hbad == 0;
}

}  // namespace

bool chol_reduce(int n, const double* M, const double* D, double* S, double* Linv, cudaStream_t st) {
  TT_CHECK(n > 0, TT_E_INVALID_ARG, "chol_reduce: empty pencil");
  const int ld = 3 * n;
  DBuf<double> aug((size_t)n * ld), dvec((size_t)n);
  build_pencil_aug_kernel<<<grid_of((long long)n * ld), 256, 0, st>>>(n, M, D, aug.get());
  count_launch();
  if (!bordered_cholesky<double>(n, ld, aug.get(), dvec.get(), st)) return false;
  // W = U^-T D_s = L^-1 D_s in columns n..2n-1, L^-1 in columns 2n..3n-1
  dev_copy2d(Linv, n, aug.get() + 2 * n, ld, n, n, 1.0, st);
  gemm_rm<double>(false, true, n, n, n, 1.0, aug.get() + n, ld, 0, Linv, n, 0, 0.0, S, n, 0, 1, st);
  return true;
}

template <typename T>
bool kkt_factor(int N, int n, const double* K, KktFactors<T>& f, cudaStream_t st) {
  const int nm = N - n;
  TT_CHECK(n > 0 && nm > 0, TT_E_INVALID_ARG, "kkt_factor: the LZ block and the multiplier block must be non-empty");
  const int ld = n + 2 * nm;
  f.N = N;
  f.n = n;
  f.nm = nm;
  DBuf<T> aug((size_t)n * ld), dvec((size_t)n);
  build_aug_kernel<T><<<grid_of((long long)n * ld), 256, 0, st>>>(N, n, nm, K, aug.get(), ld);
  count_launch();
  if (!bordered_cholesky<T>(n, ld, aug.get(), dvec.get(), st)) return false;
  f.lz.alloc((size_t)n * n);
  chol_to_lu_kernel<T><<<grid_of((long long)n * n), 256, 0, st>>>(n, ld, aug.get(), dvec.get(), f.lz.get());
  count_launch();
  f.lz_dinv.alloc(lu_diag_inv_size(n));
  lu_diag_inverses<T>(n, f.lz.get(), f.lz_dinv.get(), st);
  f.ident.alloc((size_t)n);
  iota_kernel<<<grid_of(n), 256, 0, st>>>(n, f.ident.get());
  count_launch();
  // Schur complement of the multipliers: F - W^T V
  f.s.alloc((size_t)nm * nm);
  copy_f_kernel<T><<<grid_of((long long)nm * nm), 256, 0, st>>>(N, n, nm, K, f.s.get());
  count_launch();
  check_launch("kkt schur complement");
  gemm_rm<T>(true, false, nm, nm, n, T(-1), aug.get() + n, ld, 0, aug.get() + n + nm, ld, 0, T(1), f.s.get(), nm,
             0, 1, st);
  f.ipiv.alloc((size_t)nm);
  lu_factor<T>(nm, f.s.get(), f.ipiv.get(), st);
  f.perm.alloc((size_t)nm);
  lu_perm(nm, f.ipiv.get(), f.perm.get(), st);
  f.s_dinv.alloc(lu_diag_inv_size(nm));
  lu_diag_inverses<T>(nm, f.s.get(), f.s_dinv.get(), st);
  return true;
}

template <typename T>
void kkt_apply(const KktFactors<T>& f, const double* K, const double* b, double* x, cudaStream_t st) {
  const int N = f.N, n = f.n, nm = f.nm;
  DBuf<double> u((size_t)n), r((size_t)nm);
  // u = LZ^-1 b_c
  solve_with<T>(n, f.lz.get(), f.ident.get(), f.ident.get(), f.lz_dinv.get(), b + nm, u.get(), st);
  // dl = S^-1 (b_m - E u)
  dev_copy(r.get(), b, (size_t)nm, st);
  gemm_rm<double>(false, false, nm, 1, n, -1.0, K, N, 0, u.get(), 1, 0, 1.0, r.get(), 1, 0, 1, st);
  solve_with<T>(nm, f.s.get(), f.ipiv.get(), f.perm.get(), f.s_dinv.get(), r.get(), x + n, st);
  // dX = LZ^-1 (b_c - G dl)
  dev_copy(x, b + nm, (size_t)n, st);
  gemm_rm<double>(false, false, n, 1, nm, -1.0, K + (size_t)nm * N + n, N, 0, x + n, 1, 0, 1.0, x, 1, 0, 1, st);
  solve_with<T>(n, f.lz.get(), f.ident.get(), f.ident.get(), f.lz_dinv.get(), x, x, st);
}

double kkt_factor_flops(int N, int n) {
  const double dn = n, dm = N - n;
  return dn * dn * dn / 3.0 + 2.0 * dn * dn * dm + 2.0 * dn * dm * dm + 2.0 * dm * dm * dm / 3.0;
}

double kkt_apply_flops(int N, int n) {
  const double dn = n, dm = N - n;
  return 4.0 * dn * dn + 2.0 * dm * dm + 4.0 * dn * dm;
}

template bool kkt_factor<double>(int, int, const double*, KktFactors<double>&, cudaStream_t);
template bool kkt_factor<float>(int, int, const double*, KktFactors<float>&, cudaStream_t);
template void kkt_apply<double>(const KktFactors<double>&, const double*, const double*, double*, cudaStream_t);
template void kkt_apply<float>(const KktFactors<float>&, const double*, const double*, double*, cudaStream_t);

}  // namespace ttsdp
