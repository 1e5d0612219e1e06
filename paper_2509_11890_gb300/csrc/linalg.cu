// Dense factorisations for the small matrices of the TT solver.
//
// The matrices are small (unfoldings of TT cores, projected local systems),
// so QR, SVD, Cholesky and the triangular kernels run in one CTA each with
// warp-shuffle reductions and the matrix resident in L2; the LU of the larger
// local systems is blocked so that its trailing updates use the multi-CTA
// strided GEMM.
#include <cfloat>
#include <climits>
#include <cooperative_groups.h>
#include <cmath>
#include <vector>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gemm.cuh"
#include "linalg.cuh"

namespace ttsdp {

double& SvdNoiseFloor::slot() {
  static thread_local double v = 0.0;
  return v;
}

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// dynamic shared memory the Jacobi SVD may use for its working columns
constexpr size_t kJacobiSmem = 200 * 1024;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread receives the result.
template <typename T>
__device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }
template <>
__device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }

// ---------------------------------------------------------------------------
// Householder QR (LAPACK-style reflectors, beta = -sign(alpha) ||x||)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) qr_kernel(MatView<T> A, T* W, T* tau, T* Q, T* R) {
  // W holds A column-major (W[c*m + i]) so that every column operation below
  // reads consecutive addresses across a warp; Q is formed column-major in
  // the first m*k entries of W's companion buffer Q and transposed at the end
  __shared__ T red[kWarps];
  __shared__ T s_beta, s_tau, s_scale;
  const int m = A.m, n = A.n, k = m < n ? m : n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (long long idx = tid; idx < (long long)m * n; idx += kThreads) {
    int c = (int)(idx / m), i = (int)(idx % m);
    W[idx] = A.p[i * A.rs + c * A.cs];
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    T* wj = W + (long long)j * m;
    T loc = T(0);
    for (int i = j + 1 + tid; i < m; i += kThreads) loc += wj[i] * wj[i];
    T sigma = block_sum(loc, red);
    if (tid == 0) {
      T alpha = wj[j];
      if (sigma == T(0)) {
        s_tau = T(0);
        s_beta = alpha;
        s_scale = T(0);
      } else {
        T nrm = sqrt(alpha * alpha + sigma);
        T beta = alpha <= T(0) ? nrm : -nrm;
        s_tau = (beta - alpha) / beta;
        s_scale = T(1) / (alpha - beta);
        s_beta = beta;
      }
      tau[j] = s_tau;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < m; i += kThreads) wj[i] *= s_scale;
    __syncthreads();
    if (tid == 0) wj[j] = s_beta;
    const T tj = s_tau;
    if (tj != T(0)) {
      for (int c = j + 1 + warp; c < n; c += kWarps) {
        T* wc = W + (long long)c * m;
        T dot = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) dot += wj[i] * wc[i];
        dot = warp_sum(dot);
        dot += wc[j];
        T f = tj * dot;
        if (lane == 0) wc[j] -= f;
        for (int i = j + 1 + lane; i < m; i += 32) wc[i] -= f * wj[i];
      }
    }
    __syncthreads();
  }
  for (long long idx = tid; idx < (long long)k * n; idx += kThreads) {
    int i = (int)(idx / n), c = (int)(idx % n);
    R[idx] = c >= i ? W[(long long)c * m + i] : T(0);
  }
  // Q column-major in Qc = Q (m*k entries), then transposed in place through W
  T* Qc = Q;
  for (long long idx = tid; idx < (long long)m * k; idx += kThreads) {
    int c = (int)(idx / m), i = (int)(idx % m);
    Qc[idx] = i == c ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    const T* wj = W + (long long)j * m;
    if (tj != T(0)) {
      for (int c = j + warp; c < k; c += kWarps) {
        T* qc = Qc + (long long)c * m;
        T dot = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) dot += wj[i] * qc[i];
        dot = warp_sum(dot);
        dot += qc[j];
        T f = tj * dot;
        if (lane == 0) qc[j] -= f;
        for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= f * wj[i];
      }
    }
    __syncthreads();
  }
  // the reflectors are no longer needed: stage Q^T-layout through W
  for (long long idx = tid; idx < (long long)m * k; idx += kThreads) W[idx] = Qc[idx];
  __syncthreads();
  for (long long idx = tid; idx < (long long)m * k; idx += kThreads) {
    int i = (int)(idx / k), c = (int)(idx % k);
    Q[idx] = W[(long long)c * m + i];
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD on the columns of an m x n matrix (m >= n), columns
// stored contiguously; round-robin ordering so each round's pairs are disjoint.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) svd_kernel(MatView<T> A, bool transposed, T* Wg, T* Vg, bool w_smem,
                                                       bool v_smem, T* U, T* S, T* Vt, int* perm, const T* V0,
                                                       bool need_v, double rel_floor2) {
  __shared__ int s_rot;
  // the working columns live in shared memory when they fit (every rotation
  // then costs shared-memory latency instead of an L2 round trip)
  extern __shared__ __align__(16) unsigned char jac_smem[];
  // work on B = A (m x n, m >= n) or B = A^T when A is wide
  const int m = transposed ? A.n : A.m;
  const int n = transposed ? A.m : A.n;
  T* Wc = w_smem ? reinterpret_cast<T*>(jac_smem) : Wg;
  T* Vc = v_smem ? reinterpret_cast<T*>(jac_smem) + (w_smem ? (size_t)m * n : 0) : Vg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (long long idx = tid; idx < (long long)m * n; idx += kThreads) {
    int j = (int)(idx / m), i = (int)(idx % m);  // column j, row i of B
    Wc[idx] = transposed ? A.p[j * A.rs + i * A.cs] : A.p[i * A.rs + j * A.cs];
  }
  // accumulated right rotations start from V0 (row-major n x n) when given:
  // B = W V0^T with W = A on entry, so the sweeps only have to finish the job
  if (need_v)
    for (long long idx = tid; idx < (long long)n * n; idx += kThreads) {
      int j = (int)(idx / n), i = (int)(idx % n);
      Vc[idx] = V0 ? V0[(long long)i * n + j] : (i == j ? T(1) : T(0));
    }
  __syncthreads();
  // rotation threshold: a length-m dot product carries about sqrt(m) eps of
  // rounding noise, so a smaller threshold never lets the sweeps terminate
  const T tol = T(4) * sqrt(T(m)) * eps_of<T>();
  // columns whose squared norm is below (eps ||A||_F)^2 are numerical noise:
  // rotating against them cannot change any singular value above that level
  // and would keep the sweep from terminating on rank-deficient inputs
  __shared__ T s_floor, s_floor_hi;
  {
    __shared__ T red[kWarps];
    T loc = T(0);
    for (long long idx = tid; idx < (long long)m * n; idx += kThreads) loc += Wc[idx] * Wc[idx];
    T fro2 = block_sum(loc, red);
    // rotating a large column against a tiny one leaves rounding noise of
    // size ~eps |large| in the tiny one, so the floor sits at the noise level
    // of the whole matrix, (sqrt(m) eps ||A||_F)^2; pairs whose columns are
    // both below rel_floor2 ||A||_F^2 (a caller that truncates far above it)
    // are left as they are
    if (tid == 0) {
      s_floor = T(m) * eps_of<T>() * eps_of<T>() * fro2;
      s_floor_hi = (T)rel_floor2 * fro2;
    }
    __syncthreads();
  }
  const T floor2 = s_floor, floor_hi = s_floor_hi;
  const int nn = n + (n & 1);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < nn - 1; ++r) {
      for (int pi = warp; pi < nn / 2; pi += kWarps) {
        int x = pi, y = nn - 1 - pi;
        int p = x == 0 ? 0 : ((x - 1 + r) % (nn - 1)) + 1;
        int q = ((y - 1 + r) % (nn - 1)) + 1;
        if (p >= n || q >= n) continue;
        T* wp = Wc + (long long)p * m;
        T* wq = Wc + (long long)q * m;
        T a = T(0), b = T(0), g = T(0);
        for (int i = lane; i < m; i += 32) {
          T u = wp[i], v = wq[i];
          a += u * u;
          b += v * v;
          g += u * v;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (g != T(0) && a > floor2 && b > floor2 && (a > floor_hi || b > floor_hi) && fabs(g) > tol * sqrt(a * b)) {
          T zeta = (b - a) / (T(2) * g);
          T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          T c = T(1) / sqrt(T(1) + t * t);
          T s = c * t;
          for (int i = lane; i < m; i += 32) {
            T u = wp[i], v = wq[i];
            wp[i] = c * u - s * v;
            wq[i] = s * u + c * v;
          }
          if (need_v) {
            T* vp = Vc + (long long)p * n;
            T* vq = Vc + (long long)q * n;
            for (int i = lane; i < n; i += 32) {
              T u = vp[i], v = vq[i];
              vp[i] = c * u - s * v;
              vq[i] = s * u + c * v;
            }
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // singular values (column norms) and a descending order
  for (int j = warp; j < n; j += kWarps) {
    T a = T(0);
    for (int i = lane; i < m; i += 32) a += Wc[(long long)j * m + i] * Wc[(long long)j * m + i];
    a = warp_sum(a);
    if (lane == 0) S[j] = sqrt(a);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < n; ++j) perm[j] = j;
    for (int j = 1; j < n; ++j) {  // insertion sort, stable
      int pj = perm[j];
      T v = S[pj];
      int t = j - 1;
      while (t >= 0 && S[perm[t]] < v) {
        perm[t + 1] = perm[t];
        --t;
      }
      perm[t + 1] = pj;
    }
  }
  __syncthreads();
  // B = Ub diag(S) Vb^T with Ub columns Wc/S, Vb = Vc (columns)
  // A = B (not transposed): U = Ub (m x n), Vt = Vb^T (n x n)
  // A = B^T (transposed):  A = Vb S Ub^T: U = Vb (A.m = n rows), Vt = Ub^T (n x m)
  const int k = n;
  for (long long idx = tid; idx < (long long)m * k; idx += kThreads) {
    int i = (int)(idx / k), r = (int)(idx % k);
    int c = perm[r];
    T s = S[c];
    T val = s > T(0) ? Wc[(long long)c * m + i] / s : T(0);
    if (!transposed) U[(long long)i * k + r] = val;       // U (m x k)
    else Vt[(long long)r * m + i] = val;                   // Vt (k x m)
  }
  for (long long idx = tid; need_v && idx < (long long)n * k; idx += kThreads) {
    int j = (int)(idx / k), r = (int)(idx % k);
    T val = Vc[(long long)perm[r] * n + j];
    if (!transposed) Vt[(long long)r * n + j] = val;       // Vt (k x n)
    else U[(long long)j * k + r] = val;                    // U (n x k) = A.m x k
  }
  __syncthreads();
  // S in descending order (reuse Wc's first column as scratch is unsafe; do it serially)
  if (tid == 0) {
    for (int r = 0; r < k; ++r) Wc[r] = S[perm[r]];
    for (int r = 0; r < k; ++r) S[r] = Wc[r];
  }
}

// ---------------------------------------------------------------------------
// Blocked LU with partial pivoting of M = A^T. The row-major buffer of A is
// the column-major buffer of M (M[i][j] at p[j*n + i]), so every column of M
// the panel touches is a contiguous row of A: the pivot search, the scaling
// and the rank-1 updates read consecutive addresses. P M = L U; then
// A = M^T = U^T L^T P and A x = b is solved by U^T y = b, L^T z = y, x = P^T z.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) lu_panel_kernel(int n, T* B, int j0, int jb, int* ipiv) {
  __shared__ T rv[kWarps];
  __shared__ int ri[kWarps];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int jj = j0; jj < j0 + jb; ++jj) {
    T* col = B + (long long)jj * n;  // column jj of M
    T best = T(-1);
    int bi = jj;
    for (int i = jj + tid; i < n; i += kThreads) {
      T v = fabs(col[i]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      T bv = rv[0];
      int bidx = ri[0];
      for (int w = 1; w < kWarps; ++w)
        if (rv[w] > bv || (rv[w] == bv && ri[w] < bidx)) { bv = rv[w]; bidx = ri[w]; }
      s_piv = bidx;
      ipiv[jj] = bidx;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != jj) {
      // interchange rows jj and piv of M inside the panel
      for (int c = j0 + tid; c < j0 + jb; c += kThreads) {
        T* cc = B + (long long)c * n;
        T t = cc[jj];
        cc[jj] = cc[piv];
        cc[piv] = t;
      }
    }
    __syncthreads();
    const T p = col[jj];
    const T inv = p != T(0) ? T(1) / p : T(0);
    for (int i = jj + 1 + tid; i < n; i += kThreads) col[i] *= inv;
    __syncthreads();
    // rank-1 update of the panel's remaining columns, one warp per column
    for (int c = jj + 1 + warp; c < j0 + jb; c += kWarps) {
      T* cc = B + (long long)c * n;
      const T u = cc[jj];
      if (u != T(0))
        for (int i = jj + 1 + lane; i < n; i += 32) cc[i] -= col[i] * u;
    }
    __syncthreads();
  }
}

// The same panel factorisation with the panel's active rows (rows j0..n-1 of
// its jb <= 32 columns) in shared memory for the whole panel, so the column
// steps touch no global memory: in one CTA when they fit, else split over
// the CTAs of a thread-block cluster (gridDim.x CTAs, launched as one
// cluster). Per column every CTA finds the largest entry among its rows and
// publishes it together with that row's jb values, and the CTA that holds
// the diagonal row publishes that row; after one cluster barrier one lane
// per CTA reads the candidates through distributed shared memory, the warp
// picks the pivot (ties to the smaller row, so every CTA picks the same one)
// and reads the winner's published row; the CTAs holding the two rows
// exchange them in their own tiles, and every CTA scales its rows and
// applies the rank-1 update. The published buffers alternate between two
// sets by column parity: a set is rewritten two columns later, after a
// barrier that every reader of its previous contents has passed. All threads
// of all CTAs pass the same barriers (no early exit). A one-CTA launch is a
// cluster of one.
constexpr int kClusterCtas = 8;
constexpr int kPanelThreads = 256;
constexpr int kPanelNB = 32;
constexpr int kPanelLds = kPanelNB + 1;  // padded row stride of the shared tile

template <typename T, bool kCluster, int kThr>
__global__ void __launch_bounds__(kThr)
    lu_panel_smem_kernel(int n, T* B, int j0, int jb, int chunk, int* ipiv) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = kCluster ? (int)cluster.block_rank() : 0;
  const int ncta = kCluster ? (int)cluster.num_blocks() : 1;
  // barrier over every thread of every CTA of the panel
  auto panel_sync = [&]() {
    if constexpr (kCluster) cluster.sync();
    else __syncthreads();
  };
  // shared memory of CTA q (this CTA's own without a cluster)
  auto remote = [&](auto* ptr, int q) {
    if constexpr (kCluster) return cluster.map_shared_rank(ptr, q);
    else return ptr;
  };
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T* tile = reinterpret_cast<T*>(panel_smem);  // [chunk][kPanelLds]
  __shared__ T cand_val[2];
  __shared__ int cand_idx[2];
  __shared__ T cand_row[2][kPanelNB];   // the candidate's row, published
  __shared__ T diag_row[2][kPanelNB];   // the diagonal row, published by its holder
  __shared__ T prow[kPanelNB];          // the pivot row (read)
  __shared__ T r0row[kPanelNB];         // the diagonal row (read by the pivot's holder)
  __shared__ T red_v[kThr / 32];
  __shared__ int red_i[kThr / 32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = j0 + crank * chunk;  // first row of M this CTA holds
  int nrows = n - row0;
  nrows = nrows < 0 ? 0 : (nrows > chunk ? chunk : nrows);
  // consecutive threads take consecutive rows of one column: coalesced loads
  for (int e = tid; e < chunk * jb; e += kThr) {
    const int c = e / chunk, r = e % chunk;
    tile[r * kPanelLds + c] = r < nrows ? B[(long long)(j0 + c) * n + row0 + r] : T(0);
  }
  __syncthreads();
  for (int jj = 0; jj < jb; ++jj) {
    const int par = jj & 1;
    const int rg = j0 + jj;  // row of the diagonal entry
    T best = T(-1);
    int bi = INT_MAX;
    for (int r = tid; r < nrows; r += kThr) {
      const int g = row0 + r;
      if (g >= rg) {
        const T v = fabs(tile[r * kPanelLds + jj]);
        if (v > best || (v == best && g < bi)) { best = v; bi = g; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = lane < kThr / 32 ? red_v[lane] : T(-1);
      bi = lane < kThr / 32 ? red_i[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { cand_val[par] = best; cand_idx[par] = bi; }
      if (lane < jb) {
        cand_row[par][lane] = bi != INT_MAX ? tile[(bi - row0) * kPanelLds + lane] : T(0);
        if (rg >= row0 && rg < row0 + nrows) diag_row[par][lane] = tile[(rg - row0) * kPanelLds + lane];
      }
    }
    panel_sync();  // every CTA's candidate, its row and the diagonal row are visible
    if (warp == 0) {
      T bv = T(-1);
      int bidx = INT_MAX, bq = 0;
      if (lane < ncta) {
        bv = *remote(&cand_val[par], lane);
        bidx = *remote(&cand_idx[par], lane);
        bq = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
        if (oi != INT_MAX && (ov > bv || (ov == bv && oi < bidx) || bidx == INT_MAX)) { bv = ov; bidx = oi; bq = oq; }
      }
      const int p = bidx;
      const int own_r = (rg - j0) / chunk, own_p = (p - j0) / chunk;
      if (lane < jb) {
        prow[lane] = remote(&cand_row[par][0], bq)[lane];
        if (crank == own_p && p != rg) r0row[lane] = remote(&diag_row[par][0], own_r)[lane];
      }
      if (lane == 0) {
        s_piv = p;
        if (crank == 0) ipiv[rg] = p;
      }
      __syncwarp();
      // exchange the two rows in this CTA's own tile
      if (p != rg && lane < jb) {
        if (crank == own_r) tile[(rg - row0) * kPanelLds + lane] = prow[lane];
        if (crank == own_p) tile[(p - row0) * kPanelLds + lane] = r0row[lane];
      }
    }
    __syncthreads();
    const T pv = prow[jj];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    for (int r = tid; r < nrows; r += kThr) {
      if (row0 + r > rg) {
        T* tr = tile + r * kPanelLds;
        const T l = tr[jj] * inv;
        tr[jj] = l;
        for (int c = jj + 1; c < jb; ++c) tr[c] -= l * prow[c];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < chunk * jb; e += kThr) {
    const int c = e / chunk, r = e % chunk;
    if (r < nrows) B[(long long)(j0 + c) * n + row0 + r] = tile[r * kPanelLds + c];
  }
  // no CTA leaves while another might still address its shared memory
  if constexpr (kCluster) cluster.sync();
}

// Row interchanges of the panel and the unit-lower triangular solve with its
// L11 for every column of M outside the panel: one warp per column, L11 in
// shared memory, the 32 unknowns of a column in the warp's lanes. The panel's
// jb interchanges, applied in order, permute at most 2 jb positions; thread 0
// composes them once per CTA (position S[k] receives the entry at src[k]),
// and every warp then gathers and scatters its column's entries in parallel.
template <typename T>
__global__ void __launch_bounds__(256) lu_swap_trsm_warp_kernel(int n, T* B, int j0, int jb, const int* ipiv) {
  __shared__ T L11[kPanelNB][kPanelNB + 1];
  __shared__ int S[2 * kPanelNB], src[2 * kPanelNB];
  __shared__ int s_ns;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < jb * jb; e += blockDim.x) {
    const int t = e / jb, r = e % jb;
    L11[r][t] = B[(long long)(j0 + t) * n + j0 + r];
  }
  if (warp == 0) {
    // warp 0 composes the interchanges: S[0..jb) are the panel rows, further
    // pivot rows are appended once (lane k watches S[jb + k]); a lookup is
    // one ballot over the appended rows
    if (lane < jb) { S[lane] = j0 + lane; src[lane] = j0 + lane; }
    int ns = jb;
    for (int jj = 0; jj < jb; ++jj) {
      const int p = ipiv[j0 + jj];
      if (p >= j0 + jb) {
        const bool hit = jb + lane < ns && S[jb + lane] == p;
        if (__ballot_sync(0xffffffffu, hit) == 0u) {
          if (lane == 0) { S[ns] = p; src[ns] = p; }
          ++ns;
        }
      }
      __syncwarp();
    }
    for (int jj = 0; jj < jb; ++jj) {
      const int p = ipiv[j0 + jj];
      if (p == j0 + jj) continue;  // uniform across the warp
      int kp;
      if (p < j0 + jb) {
        kp = p - j0;
      } else {
        const unsigned m = __ballot_sync(0xffffffffu, jb + lane < ns && S[jb + lane] == p);
        kp = jb + __ffs(m) - 1;
      }
      if (lane == 0) {
        const int t = src[jj];
        src[jj] = src[kp];
        src[kp] = t;
      }
      __syncwarp();
    }
    if (lane == 0) s_ns = ns;
  }
  __syncthreads();
  const int ns = s_ns;
  for (int c = blockIdx.x * nw + warp; c < n - jb; c += gridDim.x * nw) {
    const int col = c < j0 ? c : c + jb;  // skip the panel columns
    T* cc = B + (long long)col * n;
    const T v0 = lane < ns ? cc[src[lane]] : T(0);
    const T v1 = lane + 32 < ns ? cc[src[lane + 32]] : T(0);
    __syncwarp();
    if (lane + 32 < ns) cc[S[lane + 32]] = v1;
    if (col >= j0 + jb) {
      // S[k] = j0 + k for k < jb: lane k holds the permuted entry of row j0 + k
      T x = v0;
      for (int t = 0; t + 1 < jb; ++t) {
        const T xt = __shfl_sync(0xffffffffu, x, t);
        if (lane > t && lane < jb) x -= L11[lane][t] * xt;
      }
      if (lane < ns) cc[S[lane]] = lane < jb ? x : v0;
    } else {
      if (lane < ns) cc[S[lane]] = v0;
    }
  }
}

// Row interchanges of the panel and the unit-lower triangular solve with its
// L11 for every column of M outside the panel, one thread per column.
template <typename T>
__global__ void lu_swap_trsm_kernel(int n, T* B, int j0, int jb, const int* ipiv) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n - jb) return;
  const int col = c < j0 ? c : c + jb;  // skip the panel columns
  T* cc = B + (long long)col * n;
  for (int jj = j0; jj < j0 + jb; ++jj) {
    const int piv = ipiv[jj];
    if (piv != jj) {
      T t = cc[jj];
      cc[jj] = cc[piv];
      cc[piv] = t;
    }
  }
  if (col >= j0 + jb) {
    for (int r = 1; r < jb; ++r) {
      T s = cc[j0 + r];
      for (int t = 0; t < r; ++t) s -= B[(long long)(j0 + t) * n + j0 + r] * cc[j0 + t];
      cc[j0 + r] = s;
    }
  }
}

// Solves A x = b with the factors of M = A^T (P M = L U in the buffer):
// U^T y = b (lower, row i of U^T = column i of U, contiguous), L^T z = y
// (upper with unit diagonal, row i of L^T = column i of L), x = P^T z. Both
// triangular solves go in blocks of 32 rows: the off-block part of a row is a
// warp dot product, the 32 x 32 triangle runs in one warp. x lives in shared
// memory when it fits, else in b itself.
template <typename T>
__global__ void __launch_bounds__(kThreads) lu_apply_kernel(int n, const T* B, const int* ipiv, T* b,
                                                            bool use_smem) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  __shared__ T tri[32][33];
  T* x = use_smem ? reinterpret_cast<T*>(lu_smem) : b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (use_smem)
    for (int i = tid; i < n; i += kThreads) x[i] = b[i];
  __syncthreads();
  // U^T y = b
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = n - i0 < 32 ? n - i0 : 32;
    for (int r = warp; r < ib; r += kWarps) {
      const T* row = B + (long long)(i0 + r) * n;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      int t = lane;
      for (; t + 96 < i0; t += 128) {
        s0 += row[t] * x[t];
        s1 += row[t + 32] * x[t + 32];
        s2 += row[t + 64] * x[t + 64];
        s3 += row[t + 96] * x[t + 96];
      }
      for (; t < i0; t += 32) s0 += row[t] * x[t];
      T s = warp_sum((s0 + s1) + (s2 + s3));
      if (lane == 0) x[i0 + r] -= s;
    }
    // the diagonal block of U^T in shared memory, then column-oriented
    // substitution in warp 0 with the unknowns in its lanes
    for (int e = tid; e < ib * ib; e += kThreads) tri[e / ib][e % ib] = B[(long long)(i0 + e / ib) * n + i0 + e % ib];
    __syncthreads();
    if (warp == 0) {
      T xv = lane < ib ? x[i0 + lane] : T(0);
      for (int t = 0; t < ib; ++t) {
        if (lane == t) xv = tri[t][t] != T(0) ? xv / tri[t][t] : T(0);
        const T xt = __shfl_sync(0xffffffffu, xv, t);
        if (lane > t && lane < ib) xv -= tri[lane][t] * xt;
      }
      if (lane < ib) x[i0 + lane] = xv;
    }
    __syncthreads();
  }
  // L^T z = y
  for (int i1 = n; i1 > 0; i1 -= 32) {
    const int i0 = i1 - 32 > 0 ? i1 - 32 : 0, ib = i1 - i0;
    for (int r = warp; r < ib; r += kWarps) {
      const T* row = B + (long long)(i0 + r) * n;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      int t = i1 + lane;
      for (; t + 96 < n; t += 128) {
        s0 += row[t] * x[t];
        s1 += row[t + 32] * x[t + 32];
        s2 += row[t + 64] * x[t + 64];
        s3 += row[t + 96] * x[t + 96];
      }
      for (; t < n; t += 32) s0 += row[t] * x[t];
      T s = warp_sum((s0 + s1) + (s2 + s3));
      if (lane == 0) x[i0 + r] -= s;
    }
    for (int e = tid; e < ib * ib; e += kThreads) tri[e / ib][e % ib] = B[(long long)(i0 + e / ib) * n + i0 + e % ib];
    __syncthreads();
    if (warp == 0) {
      T xv = lane < ib ? x[i0 + lane] : T(0);
      for (int t = ib - 1; t > 0; --t) {
        const T xt = __shfl_sync(0xffffffffu, xv, t);  // unit diagonal: x_t is final
        if (lane < t) xv -= tri[lane][t] * xt;
      }
      if (lane < ib) x[i0 + lane] = xv;
    }
    __syncthreads();
  }
  // x = P^T z: the interchanges in reverse order
  if (tid == 0)
    for (int j = n - 1; j >= 0; --j) {
      const int p = ipiv[j];
      if (p != j) {
        T t = x[j];
        x[j] = x[p];
        x[p] = t;
      }
    }
  __syncthreads();
  if (use_smem)
    for (int i = tid; i < n; i += kThreads) b[i] = x[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) cholesky_kernel(int n, T* A, int* nonpos) {
  __shared__ T s_d;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T v = A[(long long)j * n + j];
      s_d = v > T(0) ? sqrt(v) : T(0);
      A[(long long)j * n + j] = s_d;
      if (!(v > T(0)) && nonpos) *nonpos = 1;
    }
    __syncthreads();
    T d = s_d;
    T inv = d > T(0) ? T(1) / d : T(0);
    for (int i = j + 1 + threadIdx.x; i < n; i += kThreads) A[(long long)i * n + j] *= inv;
    __syncthreads();
    int rem = n - j - 1;
    long long tot = (long long)rem * rem;
    for (long long e = threadIdx.x; e < tot; e += kThreads) {
      int i = j + 1 + (int)(e / rem), c = j + 1 + (int)(e % rem);
      if (c <= i) A[(long long)i * n + c] -= A[(long long)i * n + j] * A[(long long)c * n + j];
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)n * n; e += kThreads) {
    int i = (int)(e / n), c = (int)(e % n);
    if (c > i) A[e] = T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) tri_inv_kernel(int n, const T* L, T* X) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < n; j += kWarps) {
    for (int i = lane; i < n; i += 32) X[(long long)i * n + j] = T(0);
    __syncwarp();
    if (lane == 0) X[(long long)j * n + j] = T(1) / L[(long long)j * n + j];
    __syncwarp();
    for (int i = j + 1; i < n; ++i) {
      T s = T(0);
      for (int t = j + lane; t < i; t += 32) s += L[(long long)i * n + t] * X[(long long)t * n + j];
      s = warp_sum(s);
      if (lane == 0) X[(long long)i * n + j] = -s / L[(long long)i * n + i];
      __syncwarp();
    }
  }
}

template <typename T>
__global__ void transpose_kernel(int m, int n, const T* in, T* out) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  out[(long long)j * m + i] = in[idx];
}

// out (rows x cols, row-major) <- the view p with out[i][j] = p[i * s0 + j * s1]
template <typename T>
__global__ void transpose_view_kernel(const T* p, long long s1, long long s0, int rows, int cols, T* out) {
  const long long tot = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / cols, j = e % cols;
    out[e] = p[i * s0 + j * s1];
  }
}

template <typename S, typename D>
__global__ void convert_kernel(const S* in, long long n, D* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (D)in[e];
}

// G <- (3 I - G) / 2
__global__ void newton_schulz_rhs_kernel(double* G, int n) {
  const long long tot = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    G[e] = ((i == j ? 3.0 : 0.0) - G[e]) * 0.5;
  }
}

// One step of the first-order Jacobi finish on the Gram matrix G = W^T W of
// nearly orthogonal columns: J = I + K with K_ij = G_ij / (G_jj - G_ii) for
// the pairs that are not yet orthogonal to working precision (the skew K that
// makes J^T G J diagonal to first order); *maxbits receives max |K_ij| as the
// bits of a non-negative double (monotone in the value), infinity when a pair
// is not orthogonal but its diagonal entries are equal.
__global__ void first_order_rotation_kernel(const double* G, int n, double tol, double floor2, double* J,
                                            unsigned long long* maxbits) {
  const long long tot = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double v = 0.0;
    if (i == j) {
      v = 1.0;
    } else {
      const double gii = G[(long long)i * n + i], gjj = G[(long long)j * n + j];
      const double gij = 0.5 * (G[(long long)i * n + j] + G[(long long)j * n + i]);
      const bool orth = (gii <= floor2 && gjj <= floor2) || fabs(gij) <= tol * sqrt(fabs(gii * gjj));
      if (!orth) {
        const double den = gjj - gii;
        v = den != 0.0 ? gij / den : HUGE_VAL;
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(fabs(v)));
      }
      if (!isfinite(v)) v = 0.0;
    }
    J[e] = v;
  }
}

// norms[j] = || column j of W (m x n, row-major) ||
__global__ void column_norms_kernel(const double* W, int m, int n, double* norms) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < m; ++i) a += W[(long long)i * n + j] * W[(long long)i * n + j];
    norms[j] = sqrt(a);
  }
}

// SVD factors from orthogonal columns W = B V (B m x n): S descending by perm,
// the W side (U of B, or Vt of A = B^T when transposed) always, the V side
// when need_v, in the layouts svd_thin returns.
__global__ void finish_svd_kernel(const double* W, const double* V, const double* norms, const int* perm, int m,
                                  int n, bool transposed, bool need_v, double* U, double* S, double* Vt) {
  const long long totw = (long long)m * n, totv = (long long)n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < totw; e += stride) {
    const int i = (int)(e / n), r = (int)(e % n);
    const int c = perm[r];
    const double s = norms[c];
    const double val = s > 0.0 ? W[(long long)i * n + c] / s : 0.0;
    if (!transposed) U[(long long)i * n + r] = val;   // U (m x k)
    else Vt[(long long)r * m + i] = val;               // Vt (k x m)
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; need_v && e < totv; e += stride) {
    const int j = (int)(e / n), r = (int)(e % n);
    const double val = V[(long long)j * n + perm[r]];
    if (!transposed) Vt[(long long)r * n + j] = val;  // Vt (k x n)
    else U[(long long)j * n + r] = val;               // U (n x k)
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) S[e] = norms[perm[e]];
}

// *maxbits <- max |G_ij - delta_ij| as the bits of a non-negative double
__global__ void max_offset_from_identity_kernel(const double* G, int n, unsigned long long* maxbits) {
  const long long tot = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double v = fabs(G[e] - (i == j ? 1.0 : 0.0));
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(isfinite(v) ? v : HUGE_VAL));
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  return (int)(g > 152 * 16 ? 152 * 16 : g);
}

// FP64 Jacobi SVDs with at least this many columns get an FP32 preconditioner
constexpr int kPrecondMinCols = 16;

}  // namespace

// FP64 tall-skinny QR by CholeskyQR2 on all SMs: twice G = A^T A (GEMM),
// G = L L^T (one CTA, n x n), Q = A L^-T (GEMM), R = R2 R1. Returns false,
// leaving Q and R to the Householder kernel, when a Cholesky pivot is not
// positive (rank deficiency at working precision) or Q^T Q is not the
// identity to 1e-12 (condition number beyond what two passes repair).
bool cholesky_qr2(MatView<double> A, double* Q, double* R, cudaStream_t st) {
  const int m = A.m, n = A.n;
  DBuf<double> A64((size_t)m * n), Q1((size_t)m * n), G((size_t)n * n), L((size_t)n * n), R1((size_t)n * n),
      R2((size_t)n * n);
  DBuf<int> nonpos(1);
  DBuf<unsigned long long> maxbits(1);
  transpose_view_kernel<double><<<grid_for((long long)m * n), 256, 0, st>>>(A.p, A.cs, A.rs, m, n, A64.get());
  count_launch();
  auto pass = [&](const double* Ain, double* Qout, double* Rout) -> bool {
    gemm_rm<double>(true, false, n, n, m, 1.0, Ain, n, 0, Ain, n, 0, 0.0, G.get(), n, 0, 1, st);
    TT_CUDA(cudaMemcpyAsync(L.get(), G.get(), sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    TT_CUDA(cudaMemsetAsync(nonpos.get(), 0, sizeof(int), st));
    cholesky_lower<double>(n, L.get(), st, nonpos.get());
    int h = 0;
    TT_CUDA(cudaMemcpyAsync(&h, nonpos.get(), sizeof(int), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    if (h) return false;
    transpose<double>(n, n, L.get(), Rout, st);   // R = L^T
    tri_lower_inverse<double>(n, L.get(), st);     // L <- L^-1
    gemm_rm<double>(false, true, m, n, n, 1.0, Ain, n, 0, L.get(), n, 0, 0.0, Qout, n, 0, 1, st);
    return true;
  };
  if (!pass(A64.get(), Q1.get(), R1.get())) return false;
  if (!pass(Q1.get(), Q, R2.get())) return false;
  gemm_rm<double>(true, false, n, n, m, 1.0, Q, n, 0, Q, n, 0, 0.0, G.get(), n, 0, 1, st);
  TT_CUDA(cudaMemsetAsync(maxbits.get(), 0, sizeof(unsigned long long), st));
  max_offset_from_identity_kernel<<<grid_for((long long)n * n), 256, 0, st>>>(G.get(), n, maxbits.get());
  count_launch();
  unsigned long long hb = 0;
  TT_CUDA(cudaMemcpyAsync(&hb, maxbits.get(), sizeof(hb), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  double off = 0.0;
  std::memcpy(&off, &hb, sizeof(double));
  if (!(off <= 1e-12)) return false;
  gemm_rm<double>(false, false, n, n, n, 1.0, R2.get(), n, 0, R1.get(), n, 0, 0.0, R, n, 0, 1, st);
  check_launch("cholesky_qr2");
  return true;
}

template <typename T>
void qr_thin(MatView<T> A, T* Q, T* R, cudaStream_t st) {
  if (A.m == 0 || A.n == 0) return;
  if constexpr (std::is_same<T, double>::value) {
    if (A.m >= 2 * A.n && A.n >= kPrecondMinCols && cholesky_qr2(A, Q, R, st)) return;
  }
  int k = A.m < A.n ? A.m : A.n;
  DBuf<T> W((size_t)A.m * A.n), tau((size_t)k);
  qr_kernel<T><<<1, kThreads, 0, st>>>(A, W.get(), tau.get(), Q, R);
  count_launch();
  check_launch("qr_kernel");
}

// out = X made orthonormal by two Newton-Schulz steps X <- X (3 I - X^T X) / 2
// (X n x n, out distinct from X). With delta = ||X^T X - I|| one step leaves
// about 1.5 delta^2 and two about 3.4 delta^4: from an FP32-accurate X (delta
// ~ 1e-6) one step would leave ~1e-12, which shows in every reconstruction
// B = W V^T made with it; two reach FP64 rounding.
static void ns_orthonormalise(int n, const double* X, double* out, cudaStream_t st) {
  DBuf<double> G((size_t)n * n), Y((size_t)n * n);
  const double* cur = X;
  for (int step = 0; step < 2; ++step) {
    double* dst = step == 1 ? out : Y.get();
    gemm_rm<double>(true, false, n, n, n, 1.0, cur, n, 0, cur, n, 0, 0.0, G.get(), n, 0, 1, st);
    newton_schulz_rhs_kernel<<<grid_for((long long)n * n), 256, 0, st>>>(G.get(), n);
    count_launch();
    gemm_rm<double>(false, false, n, n, n, 1.0, cur, n, 0, G.get(), n, 0, 0.0, dst, n, 0, 1, st);
    cur = dst;
  }
}

// Finishes the SVD of B from W = B V (V orthonormal, W's columns nearly
// orthogonal) by first-order Jacobi steps computed from the Gram matrix with
// multi-CTA GEMMs: each step rotates by J = orth(I + K) (K from
// first_order_rotation_kernel, one Newton-Schulz step), which squares the
// remaining angles, until every pair is orthogonal to working precision (the
// tolerance of the one-CTA Jacobi kernel). W and V are updated in place.
// Returns false, leaving the sweeps to the Jacobi kernel, when an angle is
// not small (clustered or equal singular values) or three steps do not
// converge.
bool first_order_finish(DBuf<double>& W, DBuf<double>& V, int m, int n, bool transposed, bool need_v, double* U,
                        double* S, double* Vt, cudaStream_t st) {
  constexpr double kMaxAngle = 1e-3;  // first-order steps only from here down
  DBuf<double> G((size_t)n * n), J((size_t)n * n), H((size_t)n * n), W2((size_t)m * n), V2((size_t)n * n);
  DBuf<unsigned long long> maxbits(1);
  const double tol = 4.0 * std::sqrt((double)m) * DBL_EPSILON;
  // the noise floor of the one-CTA kernel: (sqrt(m) eps ||B||_F)^2
  double fro2 = 0.0;
  {
    DBuf<double> nrm((size_t)n);
    column_norms_kernel<<<ceil_div(n, 128), 128, 0, st>>>(W.get(), m, n, nrm.get());
    count_launch();
    std::vector<double> h((size_t)n);
    TT_CUDA(cudaMemcpyAsync(h.data(), nrm.get(), n * sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    for (double v : h) fro2 += v * v;
  }
  const double floor2 = std::max((double)m * DBL_EPSILON * DBL_EPSILON, SvdNoiseFloor::current()) * fro2;
  bool converged = false;
  for (int step = 0; step < 3; ++step) {
    gemm_rm<double>(true, false, n, n, m, 1.0, W.get(), n, 0, W.get(), n, 0, 0.0, G.get(), n, 0, 1, st);
    TT_CUDA(cudaMemsetAsync(maxbits.get(), 0, sizeof(unsigned long long), st));
    first_order_rotation_kernel<<<grid_for((long long)n * n), 256, 0, st>>>(G.get(), n, tol, floor2, J.get(),
                                                                            maxbits.get());
    count_launch();
    unsigned long long hb = 0;
    TT_CUDA(cudaMemcpyAsync(&hb, maxbits.get(), sizeof(hb), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    double maxang = 0.0;
    std::memcpy(&maxang, &hb, sizeof(double));
    if (hb == 0) {
      converged = true;
      break;
    }
    if (!(maxang <= kMaxAngle)) return false;
    // H = J made orthonormal, then W <- W H, V <- V H
    ns_orthonormalise(n, J.get(), H.get(), st);
    gemm_rm<double>(false, false, m, n, n, 1.0, W.get(), n, 0, H.get(), n, 0, 0.0, W2.get(), n, 0, 1, st);
    gemm_rm<double>(false, false, n, n, n, 1.0, V.get(), n, 0, H.get(), n, 0, 0.0, V2.get(), n, 0, 1, st);
    std::swap(W, W2);
    std::swap(V, V2);
  }
  if (!converged) return false;
  // singular values, a stable descending order, the factors
  DBuf<double> norms((size_t)n);
  column_norms_kernel<<<ceil_div(n, 128), 128, 0, st>>>(W.get(), m, n, norms.get());
  count_launch();
  std::vector<double> hs((size_t)n);
  TT_CUDA(cudaMemcpyAsync(hs.data(), norms.get(), n * sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  std::vector<int> perm((size_t)n);
  for (int j = 0; j < n; ++j) perm[(size_t)j] = j;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return hs[(size_t)a] > hs[(size_t)b]; });
  DBuf<int> dperm((size_t)n);
  TT_CUDA(cudaMemcpyAsync(dperm.get(), perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
  finish_svd_kernel<<<grid_for((long long)m * n), 256, 0, st>>>(W.get(), V.get(), norms.get(), dperm.get(), m, n,
                                                                transposed, need_v, U, S, Vt);
  count_launch();
  check_launch("first-order svd finish");
  TT_CUDA(sync_stream(st));  // perm (host memory) is read by the copy above
  return true;
}

template <typename T>
void svd_thin(MatView<T> A, T* U, T* S, T* Vt, cudaStream_t st, SvdSide side) {
  if (A.m == 0 || A.n == 0) return;
  // strongly rectangular: reduce to the square triangular factor first so the
  // Jacobi sweeps run over min(m, n) rows instead of max(m, n)
  if (A.m >= 2 * A.n) {
    const int m = A.m, n = A.n;
    DBuf<T> Q((size_t)m * n), R((size_t)n * n), UR((size_t)n * n);
    qr_thin<T>(A, Q.get(), R.get(), st);
    svd_thin<T>(MatView<T>{R.get(), n, n, n, 1}, UR.get(), S, Vt, st, side);
    if (side != kSvdRight)
      gemm_rm<T>(false, false, m, n, n, T(1), Q.get(), n, 0, UR.get(), n, 0, T(0), U, n, 0, 1, st);
    return;
  }
  if (A.n >= 2 * A.m) {
    // A^T = Q R  =>  A = R^T Q^T ; R^T = U S Vr^T  =>  Vt = Vr^T Q^T
    const int m = A.m, n = A.n;
    DBuf<T> Q((size_t)n * m), R((size_t)m * m), VR((size_t)m * m);
    qr_thin<T>(MatView<T>{A.p, n, m, A.cs, A.rs}, Q.get(), R.get(), st);
    svd_thin<T>(MatView<T>{R.get(), m, m, 1, m}, U, S, VR.get(), st, side);
    if (side != kSvdLeft)
      gemm_rm<T>(false, true, m, n, m, T(1), VR.get(), m, 0, Q.get(), m, 0, T(0), Vt, n, 0, 1, st);
    return;
  }
  bool tr = A.m < A.n;
  int m = tr ? A.n : A.m, n = tr ? A.m : A.n;
  static std::once_flag attr_once;
  cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&]() {
    attr_err = cudaFuncSetAttribute(svd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacobiSmem);
  });
  TT_CUDA(attr_err);
  // the sweeps orthogonalise the columns of B (A, or A^T when A is wide):
  // the side they produce directly is U when A is tall, Vt when A is wide
  const bool need_v = !((side == kSvdLeft && !tr) || (side == kSvdRight && tr));
  const size_t wb = (size_t)m * n * sizeof(T), vb = need_v ? (size_t)n * n * sizeof(T) : 0;
  const bool w_smem = wb <= kJacobiSmem;
  const bool v_smem = need_v && w_smem && wb + vb <= kJacobiSmem;
  const size_t smem = (w_smem ? wb : 0) + (v_smem ? vb : 0);
  DBuf<T> Wc(w_smem ? 0 : (size_t)m * n), Vc((v_smem || !need_v) ? 0 : (size_t)n * n);
  DBuf<int> perm((size_t)n);
  if constexpr (std::is_same<T, double>::value) {
    if (n >= kPrecondMinCols) {
      // FP32 preconditioning: the right singular vectors of an FP32 copy,
      // made orthonormal in FP64, rotate B to nearly orthogonal columns
      // W = B V0; the FP64 sweeps on W then converge in one or two sweeps
      // instead of the six to ten they take from the identity
      DBuf<double> B64((size_t)m * n), V0((size_t)n * n), W((size_t)m * n), G((size_t)n * n), H((size_t)n * n);
      DBuf<float> B32((size_t)m * n), U32((size_t)m * n), S32((size_t)n), Vt32((size_t)n * n);
      // B64 = B row-major (m x n): B = A, or A^T when A is wide
      if (tr) transpose_view_kernel<double><<<grid_for((long long)m * n), 256, 0, st>>>(A.p, A.rs, A.cs, m, n, B64.get());
      else transpose_view_kernel<double><<<grid_for((long long)m * n), 256, 0, st>>>(A.p, A.cs, A.rs, m, n, B64.get());
      count_launch();
      convert_kernel<double, float><<<grid_for((long long)m * n), 256, 0, st>>>(B64.get(), (long long)m * n, B32.get());
      count_launch();
      svd_thin<float>(MatView<float>{B32.get(), m, n, n, 1}, U32.get(), S32.get(), Vt32.get(), st);
      // V0 = Vt32^T in FP64, made orthonormal by Newton-Schulz steps
      transpose<float>(n, n, Vt32.get(), U32.get(), st);
      convert_kernel<float, double><<<grid_for((long long)n * n), 256, 0, st>>>(U32.get(), (long long)n * n, H.get());
      count_launch();
      ns_orthonormalise(n, H.get(), V0.get(), st);
      gemm_rm<double>(false, false, m, n, n, 1.0, B64.get(), n, 0, V0.get(), n, 0, 0.0, W.get(), n, 0, 1, st);
      check_launch("svd preconditioning");
      if (first_order_finish(W, V0, m, n, tr, need_v, U, S, Vt, st)) return;
      MatView<double> wv{W.get(), m, n, n, 1};
      if (!tr) {
        svd_kernel<double><<<1, kThreads, smem, st>>>(wv, false, Wc.get(), Vc.get(), w_smem, v_smem, U, S, Vt,
                                                      perm.get(), V0.get(), need_v, SvdNoiseFloor::current());
        count_launch();
      } else {
        // B = A^T = U_B S Vt_B  =>  A = Vt_B^T S U_B^T
        DBuf<double> UB((size_t)m * n), VtB(need_v ? (size_t)n * n : 0);
        svd_kernel<double><<<1, kThreads, smem, st>>>(wv, false, Wc.get(), Vc.get(), w_smem, v_smem, UB.get(), S,
                                                      VtB.get(), perm.get(), V0.get(), need_v, SvdNoiseFloor::current());
        count_launch();
        if (need_v) transpose<double>(n, n, VtB.get(), U, st);
        transpose<double>(m, n, UB.get(), Vt, st);
      }
      check_launch("svd_kernel");
      return;
    }
  }
  svd_kernel<T><<<1, kThreads, smem, st>>>(A, tr, Wc.get(), Vc.get(), w_smem, v_smem, U, S, Vt, perm.get(),
                                           nullptr, need_v, SvdNoiseFloor::current());
  count_launch();
  check_launch("svd_kernel");
}

// dynamic shared memory of one CTA of the cluster panel (the opt-in limit is 227 KB)
constexpr size_t kPanelSmemMax = 220 * 1024;

template <typename T>
void lu_factor(int n, T* A, int* ipiv, cudaStream_t st) {
  if (n <= 0) return;
  constexpr int nb = kPanelNB;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(lu_panel_smem_kernel<T, false, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kPanelSmemMax);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(lu_panel_smem_kernel<T, true, kPanelThreads>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmemMax);
  });
  TT_CUDA(attr_err);
  for (int j0 = 0; j0 < n; j0 += nb) {
    int jb = n - j0 < nb ? n - j0 : nb;
    // the active rows in one CTA's shared memory when they fit, else over a
    // cluster of kClusterCtas CTAs, else the panel streams through L2. FP64
    // panels of more than 256 rows go to the cluster even when they fit one
    // CTA: their rank-1 updates are FP64 arithmetic, which one SM of GB300
    // issues at about 8 GFLOP/s, so spreading the rows over eight SMs pays
    // for the cluster barriers
    const size_t row_bytes = (size_t)kPanelLds * sizeof(T);
    const bool spread = std::is_same<T, double>::value && n - j0 > 256;
    if (!spread && (size_t)(n - j0) * row_bytes <= kPanelSmemMax) {
      lu_panel_smem_kernel<T, false, 512><<<1, 512, (size_t)(n - j0) * row_bytes, st>>>(n, A, j0, jb, n - j0,
                                                                                       ipiv);
    } else if ((size_t)ceil_div(n - j0, kClusterCtas) * row_bytes <= kPanelSmemMax) {
      const int chunk = ceil_div(n - j0, kClusterCtas);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kClusterCtas, 1, 1);
      cfg.blockDim = dim3(kPanelThreads, 1, 1);
      cfg.dynamicSmemBytes = (size_t)chunk * row_bytes;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kClusterCtas;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      TT_CUDA(cudaLaunchKernelEx(&cfg, lu_panel_smem_kernel<T, true, kPanelThreads>, n, A, j0, jb, chunk, ipiv));
    } else {
      lu_panel_kernel<T><<<1, kThreads, 0, st>>>(n, A, j0, jb, ipiv);
    }
    count_launch();
    int ncols = n - jb;
    if (ncols > 0) {
      const int blocks = std::min(ceil_div(ncols, 8), 152 * 8);
      lu_swap_trsm_warp_kernel<T><<<blocks, 256, 0, st>>>(n, A, j0, jb, ipiv);
      count_launch();
    }
    int rest = n - j0 - jb;
    // M22 -= M21 M12 in M's column-major layout is, on the row-major views of
    // the same buffer, M22^T -= M12^T M21^T
    if (rest > 0)
      gemm_rm<T>(false, false, rest, rest, jb, T(-1), A + (long long)(j0 + jb) * n + j0, n, 0,
                 A + (long long)j0 * n + j0 + jb, n, 0, T(1), A + (long long)(j0 + jb) * n + j0 + jb, n,
                 0, 1, st);
  }
  check_launch("lu_factor");
}

namespace {

// Rows of one step of the cluster triangular solves, and the cluster size.
constexpr int kApplyNB = 64;
constexpr int kApplyCtas = 8;
constexpr int kApplyThreads = 512;

// The inverses of the 64 x 64 diagonal blocks of a factored system in the
// layout lu_apply_kernel reads (block b covers rows and columns b*64 ..
// b*64+63, cut at n): dinv[b] holds the inverse of the block's lower
// triangle (diagonal included) in its lower triangle and the strictly upper
// part of the inverse of its unit upper triangle above the diagonal. One CTA
// per block; thread j computes column j of the lower inverse (forward
// substitution), thread 64 + j column j of the upper one. A zero diagonal
// entry gives zero, as the substitution of lu_apply_kernel does.
template <typename T>
__global__ void __launch_bounds__(2 * kApplyNB) lu_diag_inv_kernel(int n, const T* __restrict__ B,
                                                                   T* __restrict__ dinv) {
  // two padded 64 x 65 tiles in dynamic shared memory (66.5 KB in FP64)
  extern __shared__ __align__(16) unsigned char inv_smem[];
  T(*tri)[kApplyNB + 1] = reinterpret_cast<T(*)[kApplyNB + 1]>(inv_smem);
  T(*out)[kApplyNB + 1] = reinterpret_cast<T(*)[kApplyNB + 1]>(inv_smem + sizeof(T) * kApplyNB * (kApplyNB + 1));
  const int b = blockIdx.x, i0 = b * kApplyNB, ib = n - i0 < kApplyNB ? n - i0 : kApplyNB;
  for (int e = threadIdx.x; e < kApplyNB * kApplyNB; e += blockDim.x) {
    const int r = e / kApplyNB, c = e % kApplyNB;
    tri[r][c] = (r < ib && c < ib) ? B[(long long)(i0 + r) * n + i0 + c] : T(0);
    out[r][c] = T(0);
  }
  __syncthreads();
  const int j = threadIdx.x % kApplyNB;
  if (j < ib) {
    if (threadIdx.x < kApplyNB) {
      // lower with diagonal: x_r = (delta_rj - sum_{j <= t < r} T[r][t] x_t) / T[r][r]
      out[j][j] = tri[j][j] != T(0) ? T(1) / tri[j][j] : T(0);
      for (int r = j + 1; r < ib; ++r) {
        T sum = T(0);
        for (int t = j; t < r; ++t) sum += tri[r][t] * out[t][j];
        out[r][j] = tri[r][r] != T(0) ? -sum / tri[r][r] : T(0);
      }
    } else {
      // unit upper: x_j = 1, x_r = -sum_{r < t <= j} U[r][t] x_t for r < j;
      // the unit diagonal stays implicit (out[j][j] belongs to the lower inverse)
      for (int r = j - 1; r >= 0; --r) {
        T sum = tri[r][j];
        for (int t = r + 1; t < j; ++t) sum += tri[r][t] * out[t][j];
        out[r][j] = -sum;
      }
    }
  }
  __syncthreads();
  T* D = dinv + (size_t)b * kApplyNB * kApplyNB;
  for (int e = threadIdx.x; e < kApplyNB * kApplyNB; e += blockDim.x) D[e] = out[e / kApplyNB][e % kApplyNB];
}

// The solves of lu_apply_kernel spread over a cluster of kApplyCtas CTAs:
// U^T y = b by 64-row blocks from the top, then L^T z = y from the bottom,
// then x[i] = z[perm[i]] (perm null: x = z). In each step every CTA takes
// the block's right-hand side, which the previous steps have completed, and
// multiplies it by the block's precomputed triangle inverse (dinv, from
// lu_diag_inv_kernel; one row per warp), so no step runs a serial chain;
// CTA 0 stores the block's unknowns, and every warp of the cluster subtracts
// their contribution from the rows it owns below (forward) or above
// (backward) the block, one row per warp at a time with the 64 products in
// its lanes. One cluster barrier (hardware, with release / acquire ordering
// of the CTAs' global writes) ends each step, so no step reads a right-hand
// side entry another CTA is still updating. b is the right-hand side on
// entry (updated in place by the forward steps) and x on exit; y and w are
// n-entry scratch vectors. Entries that another CTA wrote are read and
// written at L2 (ld/st.cg), past the SM's L1.
template <typename T>
__global__ void __launch_bounds__(kApplyThreads) lu_apply_cluster_kernel(int n, const T* __restrict__ B,
                                                                         const T* __restrict__ dinv,
                                                                         const int* __restrict__ perm, T* b, T* y,
                                                                         T* w) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  __shared__ T rhs[kApplyNB];
  __shared__ T xb[kApplyNB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarpsPerCta = kApplyThreads / 32;
  const int gwarp = rank * kWarpsPerCta + warp, nwarps = kApplyCtas * kWarpsPerCta;
  const int nblk = (n + kApplyNB - 1) / kApplyNB;
  // forward: U^T y = b (lower triangle of the buffer, diagonal included)
  for (int blk = 0; blk < nblk; ++blk) {
    const int i0 = blk * kApplyNB, ib = n - i0 < kApplyNB ? n - i0 : kApplyNB, i1 = i0 + ib;
    const T* D = dinv + (size_t)blk * kApplyNB * kApplyNB;
    if (tid < ib) rhs[tid] = __ldcg(b + i0 + tid);
    __syncthreads();
    for (int r = warp; r < ib; r += kWarpsPerCta) {
      const T* Dr = D + (size_t)r * kApplyNB;
      T s = (lane <= r ? Dr[lane] * rhs[lane] : T(0)) + (lane + 32 <= r ? Dr[lane + 32] * rhs[lane + 32] : T(0));
      s = warp_sum(s);
      if (lane == 0) xb[r] = s;
    }
    __syncthreads();
    if (rank == 0 && tid < ib) __stcg(y + i0 + tid, xb[tid]);
    for (int row = i1 + gwarp; row < n; row += nwarps) {
      const T* Br = B + (long long)row * n + i0;
      T s = (lane < ib ? Br[lane] * xb[lane] : T(0)) + (lane + 32 < ib ? Br[lane + 32] * xb[lane + 32] : T(0));
      s = warp_sum(s);
      if (lane == 0) __stcg(b + row, __ldcg(b + row) - s);
    }
    cluster.sync();
  }
  // backward: L^T z = y (strict upper triangle of the buffer, unit diagonal)
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int i0 = blk * kApplyNB, ib = n - i0 < kApplyNB ? n - i0 : kApplyNB;
    const T* D = dinv + (size_t)blk * kApplyNB * kApplyNB;
    if (tid < ib) rhs[tid] = __ldcg(y + i0 + tid);
    __syncthreads();
    for (int r = warp; r < ib; r += kWarpsPerCta) {
      const T* Dr = D + (size_t)r * kApplyNB;
      T s = (lane > r && lane < ib ? Dr[lane] * rhs[lane] : T(0)) +
            (lane + 32 > r && lane + 32 < ib ? Dr[lane + 32] * rhs[lane + 32] : T(0));
      s = warp_sum(s);
      if (lane == 0) xb[r] = rhs[r] + s;
    }
    __syncthreads();
    if (rank == 0 && tid < ib) __stcg(w + i0 + tid, xb[tid]);
    for (int row = gwarp; row < i0; row += nwarps) {
      const T* Br = B + (long long)row * n + i0;
      T s = (lane < ib ? Br[lane] * xb[lane] : T(0)) + (lane + 32 < ib ? Br[lane + 32] * xb[lane + 32] : T(0));
      s = warp_sum(s);
      if (lane == 0) __stcg(y + row, __ldcg(y + row) - s);
    }
    cluster.sync();
  }
  // x = P^T z as a gather
  for (int i = rank * kApplyThreads + tid; i < n; i += kApplyCtas * kApplyThreads)
    __stcg(b + i, __ldcg(w + (perm ? perm[i] : i)));
}

// perm[i] = the index the interchanges ipiv of lu_factor (applied in reverse
// order, as lu_apply_kernel applies them) move to position i; one thread
// composes them in shared memory.
__global__ void lu_perm_kernel(int n, const int* __restrict__ ipiv, int* __restrict__ perm) {
  extern __shared__ int perm_smem[];
  int* p = perm_smem;
  int* piv = perm_smem + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    p[i] = i;
    piv[i] = ipiv[i];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = n - 1; j >= 0; --j) {
      const int q = piv[j];
      if (q != j) {
        const int t = p[j];
        p[j] = p[q];
        p[q] = t;
      }
    }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = p[i];
}

}  // namespace

void lu_perm(int n, const int* ipiv, int* perm, cudaStream_t st) {
  if (n <= 0) return;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(lu_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  TT_CUDA(attr_err);
  TT_CHECK((size_t)n * 2 * sizeof(int) <= 200 * 1024, TT_E_INVALID_ARG, "lu_perm: system too large");
  lu_perm_kernel<<<1, 256, (size_t)n * 2 * sizeof(int), st>>>(n, ipiv, perm);
  count_launch();
  check_launch("lu_perm");
}

size_t lu_diag_inv_size(int n) { return (size_t)((n + kApplyNB - 1) / kApplyNB) * kApplyNB * kApplyNB; }

template <typename T>
void lu_diag_inverses(int n, const T* LU, T* dinv, cudaStream_t st) {
  if (n <= 0) return;
  constexpr size_t smem = 2 * sizeof(T) * kApplyNB * (kApplyNB + 1);
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(lu_diag_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  TT_CUDA(attr_err);
  lu_diag_inv_kernel<T><<<(n + kApplyNB - 1) / kApplyNB, 2 * kApplyNB, smem, st>>>(n, LU, dinv);
  count_launch();
  check_launch("lu_diag_inv_kernel");
}

namespace {

// Systems from this size on are solved by the cluster kernel.
constexpr int kApplyClusterMin = 160;

template <typename T>
void lu_apply_cluster(int n, const T* LU, const int* perm, const T* dinv, T* b, cudaStream_t st) {
  DBuf<T> y((size_t)n), w((size_t)n), dtmp;
  if (!dinv) {
    dtmp.alloc(lu_diag_inv_size(n));
    lu_diag_inverses<T>(n, LU, dtmp.get(), st);
    dinv = dtmp.get();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kApplyCtas, 1, 1);
  cfg.blockDim = dim3(kApplyThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kApplyCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TT_CUDA(cudaLaunchKernelEx(&cfg, lu_apply_cluster_kernel<T>, n, LU, dinv, perm, b, y.get(), w.get()));
  count_launch();
  check_launch("lu_apply_cluster_kernel");
}

}  // namespace

template <typename T>
void lu_solve_factored(int n, const T* LU, const int* ipiv, T* b, cudaStream_t st, const int* perm, const T* dinv) {
  if (n <= 0) return;
  if (n >= kApplyClusterMin) {
    if (perm) {
      lu_apply_cluster<T>(n, LU, perm, dinv, b, st);
    } else {
      DBuf<int> p((size_t)n);
      lu_perm(n, ipiv, p.get(), st);
      lu_apply_cluster<T>(n, LU, p.get(), dinv, b, st);
    }
    return;
  }
  // the solution vector in shared memory (opt-in limit, beside the kernel's
  // static 32 x 33 triangle) when it fits
  constexpr size_t kMaxSmem = 160 * 1024;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(lu_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  });
  TT_CUDA(attr_err);
  const bool use_smem = (size_t)n * sizeof(T) <= kMaxSmem;
  lu_apply_kernel<T><<<1, kThreads, use_smem ? (size_t)n * sizeof(T) : 0, st>>>(n, LU, ipiv, b, use_smem);
  count_launch();
  check_launch("lu_apply_kernel");
}

template <typename T>
void lu_solve(int n, T* A, T* b, cudaStream_t st) {
  if (n <= 0) return;
  DBuf<int> ipiv((size_t)n);
  lu_factor<T>(n, A, ipiv.get(), st);
  lu_solve_factored<T>(n, A, ipiv.get(), b, st);
}

template <typename T>
void cholesky_lower(int n, T* A, cudaStream_t st, int* nonpos) {
  if (n <= 0) return;
  cholesky_kernel<T><<<1, kThreads, 0, st>>>(n, A, nonpos);
  count_launch();
  check_launch("cholesky");
}

template <typename T>
void tri_lower_inverse(int n, T* L, cudaStream_t st) {
  if (n <= 0) return;
  DBuf<T> X((size_t)n * n);
  tri_inv_kernel<T><<<1, kThreads, 0, st>>>(n, L, X.get());
  count_launch();
  TT_CUDA(cudaMemcpyAsync(L, X.get(), sizeof(T) * n * n, cudaMemcpyDeviceToDevice, st));
  check_launch("tri_inv");
}

template <typename T>
void transpose(int m, int n, const T* in, T* out, cudaStream_t st) {
  long long tot = (long long)m * n;
  if (tot == 0) return;
  transpose_kernel<T><<<ceil_div(tot, 256), 256, 0, st>>>(m, n, in, out);
  count_launch();
  check_launch("transpose");
}

#define INST(T)                                                                 \
  template void qr_thin<T>(MatView<T>, T*, T*, cudaStream_t);                   \
  template void svd_thin<T>(MatView<T>, T*, T*, T*, cudaStream_t, SvdSide);     \
  template void lu_solve<T>(int, T*, T*, cudaStream_t);                         \
  template void lu_factor<T>(int, T*, int*, cudaStream_t);                      \
  template void lu_solve_factored<T>(int, const T*, const int*, T*, cudaStream_t, const int*, const T*); \
  template void lu_diag_inverses<T>(int, const T*, T*, cudaStream_t);           \
  template void cholesky_lower<T>(int, T*, cudaStream_t, int*);                 \
  template void tri_lower_inverse<T>(int, T*, cudaStream_t);                    \
  template void transpose<T>(int, int, const T*, T*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ttsdp
