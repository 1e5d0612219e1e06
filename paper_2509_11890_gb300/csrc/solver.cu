// Block-AMEn Newton solves, ALS step lengths and the interior-point iteration.
//
// Environments of every (frame, operator, vector) triple are cached on the
// device and updated core by core with the three-stage contractions; the
// reduced projected system (eq. reduced_kkt_system) is assembled from the
// dense local operators and solved by LU; the block index is moved by a
// truncated SVD with a random kick; rounding uses the spectral shift of
// Corollary psdness_rounding.
#include <algorithm>
#include <cmath>
#include <exception>
#include <functional>
#include <limits>
#include <optional>
#include <thread>

#include "contract.cuh"
#include "gemm.cuh"
#include "kkt.cuh"
#include "linalg.cuh"
#include "solver.cuh"
#include "tc_gemm.cuh"

namespace ttsdp {

namespace {

// Runs independent jobs concurrently: job 0 on the calling thread and stream,
// job i > 0 on its own host thread and on side stream i-1, which first waits
// for everything already queued on the calling stream. The calling stream
// then waits for every side stream. The first exception is rethrown after all
// jobs have ended and their streams are drained.
void run_concurrently(std::vector<std::function<void()>>& jobs, std::vector<cudaStream_t>& side) {
  if (jobs.empty()) return;
  if (jobs.size() == 1 || concurrent_solves().load() > 1) {
    // one job, or solves already run concurrently (more host threads would
    // only compete with theirs for the cores): in order, on this thread
    for (auto& j : jobs) j();
    return;
  }
  cudaStream_t main = cur_stream();
  int dev = 0;
  TT_CUDA(cudaGetDevice(&dev));
  while (side.size() + 1 < jobs.size()) {
    cudaStream_t s = nullptr;
    TT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    side.push_back(s);
  }
  cudaEvent_t start = nullptr;
  TT_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  TT_CUDA(cudaEventRecord(start, main));
  const size_t nj = jobs.size();
  std::vector<cudaEvent_t> done(nj, nullptr);
  std::vector<std::exception_ptr> err(nj);
  for (size_t i = 1; i < nj; ++i) TT_CUDA(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
  std::vector<std::thread> th;
  const tt_allocator* al = AllocScope::current();
  for (size_t i = 1; i < nj; ++i) {
    cudaStream_t s = side[i - 1];
    th.emplace_back([&, i, s, al]() {
      try {
        TT_CUDA(cudaSetDevice(dev));
        StreamScope::current() = s;
        AllocScope::current() = al;
        TT_CUDA(cudaStreamWaitEvent(s, start, 0));
        jobs[i]();
        TT_CUDA(cudaEventRecord(done[i], s));
      } catch (...) {
        err[i] = std::current_exception();
        sync_stream(s);
      }
    });
  }
  try {
    jobs[0]();
  } catch (...) {
    err[0] = std::current_exception();
  }
  for (auto& t : th) t.join();
  for (size_t i = 1; i < nj; ++i) {
    cudaStreamWaitEvent(main, done[i], 0);
    cudaEventDestroy(done[i]);
  }
  cudaEventDestroy(start);
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

// Side streams shared by fan_out calls (any thread), handed out and back
// under a lock.
struct StreamPool {
  std::mutex mu;
  std::vector<cudaStream_t> free;
  std::vector<cudaStream_t> take(int n) {
    std::lock_guard<std::mutex> lk(mu);
    std::vector<cudaStream_t> out;
    while ((int)out.size() < n) {
      if (!free.empty()) {
        out.push_back(free.back());
        free.pop_back();
      } else {
        cudaStream_t s = nullptr;
        TT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        out.push_back(s);
      }
    }
    return out;
  }
  void give(const std::vector<cudaStream_t>& v) {
    std::lock_guard<std::mutex> lk(mu);
    free.insert(free.end(), v.begin(), v.end());
  }
};
StreamPool& stream_pool() {
  static StreamPool p;
  return p;
}

constexpr int kFanWidth = 4;

// Enqueues independent jobs on up to kFanWidth side streams from the calling
// thread: job j's launches go to side stream j mod kFanWidth, which first
// waits for everything already queued on the calling stream, and the calling
// stream then waits for every side stream. For jobs that only enqueue work
// (no host synchronisation), their small kernels overlap without host
// threads. Buffers a job allocates are stream-ordered on its side stream and
// are safe to use and free on the calling stream afterwards; with a caller
// allocator in scope (whose frees need not be stream-ordered) the jobs run
// in order on the calling stream instead.
void fan_out(const std::vector<std::function<void()>>& jobs) {
  if (jobs.size() <= 1 || AllocScope::current()) {
    for (auto& j : jobs) j();
    return;
  }
  cudaStream_t main = cur_stream();
  const int width = std::min<int>(kFanWidth, (int)jobs.size());
  std::vector<cudaStream_t> side = stream_pool().take(width);
  cudaEvent_t start = nullptr;
  TT_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  TT_CUDA(cudaEventRecord(start, main));
  for (cudaStream_t s : side) TT_CUDA(cudaStreamWaitEvent(s, start, 0));
  std::exception_ptr err;
  for (size_t j = 0; j < jobs.size(); ++j) {
    StreamScope::current() = side[j % width];
    try {
      jobs[j]();
    } catch (...) {
      if (!err) err = std::current_exception();
    }
  }
  StreamScope::current() = main;
  for (cudaStream_t s : side) {
    cudaEvent_t done = nullptr;
    TT_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    TT_CUDA(cudaEventRecord(done, s));
    TT_CUDA(cudaStreamWaitEvent(main, done, 0));
    TT_CUDA(cudaEventDestroy(done));
  }
  TT_CUDA(cudaEventDestroy(start));
  stream_pool().give(side);
  if (err) std::rethrow_exception(err);
}

// ---------------------------------------------------------------------------
// environments of <W, Op V>
// ---------------------------------------------------------------------------
struct Env {
  DTT op;
  const DTT* vec = nullptr;  // null: the frame itself
  std::vector<DBuf<double>> L, R;

  Env(DTT o, const DTT* v, int d) : op(std::move(o)), vec(v), L(d + 1), R(d + 1) {
    L[0].alloc(1);
    R[d].alloc(1);
    dev_fill(L[0].get(), 1, 1.0, cur_stream());
    dev_fill(R[d].get(), 1, 1.0, cur_stream());
  }
  const DTT& V(const DTT& frame) const { return vec ? *vec : frame; }
  CDims dims(const DTT& frame, int k) const {
    const DTT& v = V(frame);
    return CDims{frame.r[k], frame.r[k + 1], op.r[k], op.r[k + 1], v.r[k], v.r[k + 1], op.m, op.n};
  }
  void push_left(const DTT& frame, int k, int prec) {
    CDims c = dims(frame, k);
    L[k + 1].alloc((size_t)c.rw2 * c.R2 * c.rv2);
    env_left_step(c, L[k].get(), frame.core(k), op.core(k), V(frame).core(k), L[k + 1].get(), prec,
                  cur_stream());
  }
  void push_right(const DTT& frame, int k, int prec) {
    CDims c = dims(frame, k);
    R[k].alloc((size_t)c.rw * c.R * c.rv);
    env_right_step(c, R[k + 1].get(), frame.core(k), op.core(k), V(frame).core(k), R[k].get(), prec,
                   cur_stream());
  }
  // W_{!=k}^T Op vec(V) at core k, written to y (rw * m * rw2)
  void local_rhs(const DTT& frame, int k, double* y, int prec) const {
    CDims c = dims(frame, k);
    local_apply(c, L[k].get(), op.core(k), R[k + 1].get(), vec->core(k), y, prec, cur_stream());
  }
  void local_mat(const DTT& frame, int k, double* out, int prec) const {
    CDims c{frame.r[k], frame.r[k + 1], op.r[k], op.r[k + 1], frame.r[k], frame.r[k + 1], op.m, op.n};
    local_matrix(c, L[k].get(), op.core(k), R[k + 1].get(), out, prec, cur_stream());
  }
};

struct RhsTerm {
  double coef;
  DTT op;
  DTT vec;
};

struct NewtonData {
  DTT A, AT, K;
  std::vector<DTT> LZ, LX;
  std::vector<RhsTerm> rp, rd, rc, rt;
  bool ineq = false;
  DTT TA, AiT;
  std::vector<DTT> DK;
  double sgn = 1.0;
  int nblk() const { return ineq ? 4 : 3; }
};

// Combined multiplier storage (Section 3.5, "Combined Multiplier Storage"):
// with the non-idle masks P_Y = I - K_Y and P_T = I - K_T disjoint, dY and dT
// are one block dLambda (dY = P_Y dLambda, dT = P_T dLambda). The multiplier
// rows become P_Y (p-row) + P_T (t-row):
//   (-P_Y A_eq + sgn P_T T A_ineq) dX + (P_Y K_Y P_Y + P_T (D_ineq + K_T) P_T) dLambda
//       = -(P_Y R_p + P_T R_t),
// the multiplier column of the dZ equation A_eq^T P_Y - sgn A_ineq^T P_T. Every
// operator here is diag_TT of a vector: products are Hadamard products of the
// diagonals, and P D P = P D for 0/1 masks. The system then has the block
// structure of the problem without inequalities (dX, dLambda, dZ).
struct MaskDiagonals {
  const DTT &pY, &pT, &aeq, &ain, &ky;
};

void combine_multipliers(NewtonData& nd, const MaskDiagonals& m) {
  const double sg = nd.sgn;
  DTT row = tt_add(tt_hadamard(m.pY, m.aeq), tt_hadamard(m.pT, tt_op_diag(nd.TA)), 1.0, -sg);
  DTT dk = tt_op_diag(nd.DK[0]);
  for (size_t i = 1; i < nd.DK.size(); ++i) dk = tt_add(dk, tt_op_diag(nd.DK[i]), 1.0, 1.0);
  DTT lam = tt_add(tt_hadamard(m.pY, m.ky), tt_hadamard(m.pT, dk), 1.0, 1.0);
  DTT col = tt_add(tt_hadamard(m.pY, m.aeq), tt_hadamard(m.pT, m.ain), 1.0, -sg);
  std::vector<RhsTerm> rhs;
  for (const RhsTerm& t : nd.rp) rhs.push_back({t.coef, tt_diag(tt_hadamard(m.pY, tt_op_diag(t.op))), t.vec});
  for (const RhsTerm& t : nd.rt) rhs.push_back({t.coef, tt_diag(tt_hadamard(m.pT, tt_op_diag(t.op))), t.vec});
  nd.A = tt_diag(row);
  nd.AT = tt_diag(col);
  nd.K = tt_diag(lam);
  nd.rp = std::move(rhs);
  nd.rt.clear();
  nd.DK.clear();
  nd.ineq = false;
}

DTT op_kron_left(const DTT& m) { return tt_kron(m, tt_identity(m.d, 2)); }   // M kron I: vec(M X)
DTT op_kron_right(const DTT& m) { return tt_kron(tt_identity(m.d, 2), m); }  // I kron M: vec(X M^T)
DTT vecv(const DTT& m) { return m.view(m.m * m.n, 1); }
DTT unvec(const DTT& v) { return v.view(2, 2); }

void sum_local_mats(std::vector<Env>& es, const DTT& frame, int k, double* out, size_t n, int prec) {
  dev_fill(out, n * n, 0.0, cur_stream());
  DBuf<double> tmp(n * n);
  for (Env& e : es) {
    e.local_mat(frame, k, tmp.get(), prec);
    dev_axpy(out, tmp.get(), n * n, 1.0, cur_stream());
  }
}

void sum_local_rhs(std::vector<std::pair<double, Env>>& es, const DTT& frame, int k, double* out, size_t n,
                   int prec) {
  dev_fill(out, n, 0.0, cur_stream());
  DBuf<double> tmp(n);
  for (auto& pe : es) {
    if (pe.first == 0.0) continue;
    pe.second.local_rhs(frame, k, tmp.get(), prec);
    dev_axpy(out, tmp.get(), n, pe.first, cur_stream());
  }
}

double dev_norm(const double* p, size_t n) { return std::sqrt(std::max(0.0, dev_dot(p, p, n, cur_stream()))); }

std::vector<double> host_copy(const double* p, size_t n) {
  std::vector<double> h(n);
  TT_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(double), cudaMemcpyDeviceToHost, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
  return h;
}

void upload(double* dst, const std::vector<double>& h) {
  TT_CUDA(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
}

int truncation_rank_rel(const std::vector<double>& s, double tol_rel, int cap) {
  double nrm2 = 0.0;
  for (double v : s) nrm2 += v * v;
  return truncation_rank(s, tol_rel * std::sqrt(nrm2), cap);
}

// ---------------------------------------------------------------------------
// precision-dispatched dense kernels of the AMEn step
// ---------------------------------------------------------------------------
// Thin SVD of a row-major matrix; the mixed precisions run the Jacobi sweeps
// in FP32 (the block-index move only needs the truncation-level spectrum).
void svd_prec(int prec, MatView<double> A, double* U, double* S, double* Vt, cudaStream_t st,
              SvdSide side = kSvdBoth) {
  if (prec == TT_FP64) {
    svd_thin<double>(A, U, S, Vt, st, side);
    return;
  }
  const int m = A.m, n = A.n, k = m < n ? m : n;
  DBuf<float> a((size_t)m * n), u((size_t)m * k), s(k), vt((size_t)k * n);
  DBuf<double> dense((size_t)m * n);
  dev_copy2d(dense.get(), n, A.p, A.rs, m, n, 1.0, st);  // A is row-major here (cs == 1)
  to_f32(dense.get(), a.get(), (size_t)m * n, st);
  svd_thin<float>(MatView<float>{a.get(), m, n, n, 1}, u.get(), s.get(), vt.get(), st, side);
  if (side != kSvdRight) to_f64(u.get(), U, (size_t)m * k, st);
  to_f64(s.get(), S, k, st);
  if (side != kSvdLeft) to_f64(vt.get(), Vt, (size_t)k * n, st);
}

// FP64 relative residual at which the refinement of a dense local solve stops
// (the accuracy of an FP64 LU of the projected system)
constexpr double kLuRefineTol = 1e-10;

// Block-elimination solves that ran to the end, those of them that used FP32
// factors, and those that fell back to the LU of the whole system (LZ block
// not positive definite, or a residual above the tolerance after the
// corrections).
std::atomic<unsigned long long> g_kkt_block{0}, g_kkt_fp32{0}, g_kkt_fallback{0}, g_kkt_not_pd{0};

// Block elimination with FP64 iterative refinement (factors of type T): x
// from b, *rho the final FP64 relative residual. The corrections stop at
// `target`, after max_corr of them, or once one fails to halve the residual
// (the FP64 residual has reached its rounding floor, or the factors are too
// far from K for the refinement to converge). Returns false, leaving x
// unspecified, when the LZ block does not factor. *flops accumulates the
// algorithmic work.
template <typename T>
bool kkt_refined(int N, int n, const double* K, const double* b, double* x, double* r, double bnorm, double target,
                 int max_corr, int* corrections, double* rho, double* flops, cudaStream_t st) {
  KktFactors<T> f;
  *flops += kkt_factor_flops(N, n);
  if (!kkt_factor<T>(N, n, K, f, st)) {
    g_kkt_not_pd.fetch_add(1, std::memory_order_relaxed);
    return false;
  }
  auto residual = [&]() {
    dev_copy(r, b, N, st);
    gemm_rm<double>(false, false, N, 1, N, -1.0, K, N, 0, x, 1, 0, 1.0, r, 1, 0, 1, st);
    return bnorm > 0 ? dev_norm(r, N) / bnorm : 0.0;
  };
  kkt_apply<T>(f, K, b, x, st);
  *flops += kkt_apply_flops(N, n);
  *rho = residual();
  DBuf<double> dx(N);
  for (int c = 0; c < max_corr && *rho > target; ++c) {
    kkt_apply<T>(f, K, r, dx.get(), st);
    *flops += kkt_apply_flops(N, n);
    dev_axpy(x, dx.get(), N, 1.0, st);
    if (corrections) ++*corrections;
    const double prev = *rho;
    *rho = residual();
    if (*rho > 0.5 * prev) break;
  }
  return true;
}

// FP64 solves by block elimination refine towards this relative residual
// (below what an FP64 LU with partial pivoting leaves on these systems) and
// accept FP32 factors only when the refinement gets to kFp64Accept.
constexpr double kFp64Target = 1e-15;
constexpr double kFp64Accept = 1e-14;

// FP32 LU of the whole system with FP64 iterative refinement: x from b (x
// starts at 0), corrections until `target`, max_corr solves, or a solve that
// fails to halve the residual; *rho the final FP64 relative residual.
void lu_refined_f32(int N, const double* K, const double* b, double* x, double* r, double bnorm, double target,
                    int max_solves, int* corrections, double* rho, double* flops, cudaStream_t st) {
  const size_t nn = (size_t)N * N;
  DBuf<float> kf(nn), rf(N);
  DBuf<int> ipiv(N), perm(N);
  DBuf<double> dx(N);
  dev_fill(x, N, 0.0, st);
  dev_copy(r, b, N, st);
  to_f32(K, kf.get(), nn, st);
  lu_factor<float>(N, kf.get(), ipiv.get(), st);
  lu_perm(N, ipiv.get(), perm.get(), st);
  DBuf<float> dinv(lu_diag_inv_size(N));
  lu_diag_inverses<float>(N, kf.get(), dinv.get(), st);
  *flops += 2.0 / 3.0 * (double)N * N * N;
  double prev = 1.0;
  for (int it = 0; it < max_solves; ++it) {
    to_f32(r, rf.get(), N, st);
    lu_solve_factored<float>(N, kf.get(), ipiv.get(), rf.get(), st, perm.get(), dinv.get());
    *flops += 2.0 * (double)N * N;
    to_f64(rf.get(), dx.get(), N, st);
    dev_axpy(x, dx.get(), N, 1.0, st);
    if (corrections && it > 0) ++*corrections;
    dev_copy(r, b, N, st);
    gemm_rm<double>(false, false, N, 1, N, -1.0, K, N, 0, x, 1, 0, 1.0, r, 1, 0, 1, st);
    *rho = bnorm > 0 ? dev_norm(r, N) / bnorm : 0.0;
    if (*rho <= target || (it > 0 && *rho > 0.5 * prev)) break;
    prev = *rho;
  }
}

// Solves K x = b (K N x N row-major FP64, kept; b becomes x) and returns the
// FP64 relative residual ||b - K x|| / ||b|| of the returned x. Every path
// refines in FP64 against K.
// n_lz > 0: K is a reduced projected system whose last n_lz rows and first
// n_lz columns hold the LZ block; it is solved by block elimination (Cholesky
// of LZ, LU of the multipliers' Schur complement):
//   FP64: FP32 factors first (while *fp32_ok), as in mixed-precision
//   iterative refinement, kept when the FP64 residual gets to kFp64Accept;
//   when that refinement falls short, *fp32_ok becomes false (the rest of
//   the caller's solves go straight to FP64 factors) and FP64 factors,
//   refined towards kFp64Target (at most three corrections), are kept at a
//   residual <= ftol.
//   Reduced precisions: FP32 factors, at most five corrections, kept at a
//   residual <= ftol.
// When LZ is not positive definite (its first Cholesky factorisation, FP32
// or FP64, meets a pivot <= 0), the residual stays above those levels, or
// n_lz = 0, the whole system is solved by LU with partial pivoting:
//   FP64: FP32 factors refined as above while *fp32_ok (kept at
//   kFp64Accept), else FP64 factors of a copy.
//   Reduced precisions: FP32 factors and at most five FP64 refinement
//   solves towards ftol.
double lu_solve_prec(int prec, int N, double* K, double* b, double ftol, int* corrections, int n_lz,
                     bool* fp32_ok) {
  cudaStream_t st = cur_stream();
  // timed as one unit: the factorisations and every triangular-solve pair
  stats_begin(st, 2);
  const size_t nn = (size_t)N * N;
  const double bnorm = dev_norm(b, N);
  DBuf<double> x(N), r(N);
  double rho = 0.0, flops = 0.0;
  const bool try32 = prec != TT_FP64 || (fp32_ok && *fp32_ok);
  auto finish = [&]() {
    dev_copy(b, x.get(), N, st);
    stats_end(st, flops, 2);
    return rho;
  };
  if (n_lz > 0 && n_lz < N) {
    int corr = 0;
    bool ok = false, factored = true;
    if (prec == TT_FP64) {
      if (try32) {
        factored = kkt_refined<float>(N, n_lz, K, b, x.get(), r.get(), bnorm, kFp64Target, 8, &corr, &rho, &flops,
                                      st);
        ok = factored && rho <= kFp64Accept;
        if (factored && !ok) *fp32_ok = false;
        if (ok) g_kkt_fp32.fetch_add(1, std::memory_order_relaxed);
      }
      if (!ok && factored)
        ok = kkt_refined<double>(N, n_lz, K, b, x.get(), r.get(), bnorm, kFp64Target, 3, &corr, &rho, &flops, st) &&
             rho <= ftol;
    } else {
      ok = kkt_refined<float>(N, n_lz, K, b, x.get(), r.get(), bnorm, ftol, 5, &corr, &rho, &flops, st) &&
           rho <= ftol;
      if (ok) g_kkt_fp32.fetch_add(1, std::memory_order_relaxed);
    }
    if (corrections) *corrections += corr;
    if (ok) {
      g_kkt_block.fetch_add(1, std::memory_order_relaxed);
      return finish();
    }
    g_kkt_fallback.fetch_add(1, std::memory_order_relaxed);
  }
  if (try32) {
    const bool fp64 = prec == TT_FP64;
    lu_refined_f32(N, K, b, x.get(), r.get(), bnorm, fp64 ? kFp64Target : ftol, fp64 ? 9 : 5, corrections, &rho,
                   &flops, st);
    if (!fp64 || rho <= kFp64Accept) return finish();
    *fp32_ok = false;
  }
  DBuf<double> Kc(nn);
  dev_copy(Kc.get(), K, nn, st);
  dev_copy(x.get(), b, N, st);
  lu_solve<double>(N, Kc.get(), x.get(), st);
  flops += 2.0 / 3.0 * (double)N * N * N + 2.0 * (double)N * N;
  dev_copy(r.get(), b, N, st);
  gemm_rm<double>(false, false, N, 1, N, -1.0, K, N, 0, x.get(), 1, 0, 1.0, r.get(), 1, 0, 1, st);
  rho = bnorm > 0 ? dev_norm(r.get(), N) / bnorm : 0.0;
  return finish();
}

// ---------------------------------------------------------------------------
// block-AMEn
// ---------------------------------------------------------------------------
BlockTT init_block(int d, int nblk, int rk, Counter& rnd) {
  std::vector<int> r(d + 1, 1);
  for (int k = 1; k < d; ++k) {
    long long cap = 1;
    int e = std::min(k, d - k);
    for (int t = 0; t < e && cap < rk; ++t) cap *= 4;
    r[k] = (int)std::min<long long>(rk, cap);
  }
  DTT c = tt_alloc(d, r, 4, 1);
  for (int k = 0; k < d; ++k) upload(c.core(k), rnd.draw(c.csize(k)));
  BlockTT w;
  w.frame = tt_orth_right(c);
  w.nblk = nblk;
  size_t n0 = w.frame.csize(0);
  w.block = std::make_shared<DBuf<double>>(nblk * n0);
  dev_fill(w.block->get(), nblk * n0, 0.0, cur_stream());
  return w;
}

struct AmenInfo {
  int sweeps = 0;
  double max_change = 0.0;
  long long gmres_iters = 0;
  double forcing = 0.0;        // largest FP64 relative residual of a local solve
  long long corrections = 0;   // correction solves the forcing check asked for
  bool converged = false;      // the sweeps met their tolerance within the budget (in a
                               // reduced precision: max(tol, the precision's floor))
};

// H[i][j] += h[i] for i <= j (H: (m + 1) x m row-major)
__global__ void hess_accum_kernel(double* H, int m, int j, const double* h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= j) H[(size_t)i * m + j] += h[i];
}

// The bookkeeping of Arnoldi step j on the device (one thread): the new
// subdiagonal entry sqrt(*nrm2), the earlier Givens rotations applied to
// column j, the new rotation and the rotated right-hand side g; out[0] =
// |g[j+1]| (the residual norm of the least-squares solution), out[1] = the
// subdiagonal entry, *inv = its inverse (0 when it is 0).
__global__ void arnoldi_step_kernel(double* H, int m, int j, double* cs, double* sn, double* g, const double* nrm2,
                                    double* inv, double* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double hn = sqrt(fmax(*nrm2, 0.0));
  H[(size_t)(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
  }
  const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
  const double rr = hypot(a, c);
  cs[j] = rr > 0 ? a / rr : 1.0;
  sn[j] = rr > 0 ? c / rr : 0.0;
  H[(size_t)j * m + j] = rr;
  H[(size_t)(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  out[0] = fabs(g[j + 1]);
  out[1] = hn;
  *inv = hn > 0.0 ? 1.0 / hn : 0.0;
}

// y = x * (*s) with the scalar read on the device
__global__ void scale_by_dev_kernel(const double* x, long long n, const double* s, double* y) {
  const double v = *s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * v;
}

// Restarted GMRES (Saad & Schultz) on device vectors with classical
// Gram-Schmidt applied twice. The Hessenberg matrix, its Givens rotations and
// the rotated right-hand side stay on the device, so an Arnoldi step reads
// back one pair of scalars (the residual estimate and the subdiagonal entry)
// instead of the projections and the norm; the small triangular solve of a
// cycle runs on the host. Stops at ||b - A x|| <= tol ||b|| or after maxit
// products. Returns the number of operator products.
int gmres(size_t N, const std::function<void(const double*, double*)>& A, const double* b, double* x, double tol,
          int m, int maxit) {
  cudaStream_t st = cur_stream();
  const double bnorm = dev_norm(b, N);
  if (bnorm == 0.0) {
    dev_fill(x, N, 0.0, st);
    return 0;
  }
  DBuf<double> V((size_t)(m + 1) * N), w(N), hdev(m + 1), Hd((size_t)(m + 1) * m), csd(m), snd(m), gd(m + 1),
      scal(2), stat(2);
  std::vector<double> H((size_t)(m + 1) * m), g(m + 1);
  const int grid = (int)std::min<long long>(((long long)N + 255) / 256, 152 * 8);
  int total = 0;
  while (total < maxit) {
    A(x, w.get());
    dev_scale(w.get(), N, -1.0, st);
    dev_axpy(w.get(), b, N, 1.0, st);
    const double beta = dev_norm(w.get(), N);
    if (beta <= tol * bnorm) break;
    dev_copy(V.get(), w.get(), N, st);
    dev_scale(V.get(), N, 1.0 / beta, st);
    dev_fill(Hd.get(), (size_t)(m + 1) * m, 0.0, st);
    dev_fill(gd.get(), m + 1, 0.0, st);
    dev_fill(gd.get(), 1, beta, st);
    int jl = -1;
    bool done = false;
    for (int j = 0; j < m && total < maxit; ++j) {
      A(V.get() + (size_t)j * N, w.get());
      ++total;
      for (int pass = 0; pass < 2; ++pass) {
        dev_multi_dot(V.get(), j + 1, N, w.get(), hdev.get(), st);
        hess_accum_kernel<<<(j + 1 + 127) / 128, 128, 0, st>>>(Hd.get(), m, j, hdev.get());
        count_launch();
        gemm_rm<double>(true, false, (int)N, 1, j + 1, -1.0, V.get(), (int)N, 0, hdev.get(), 1, 0, 1.0, w.get(), 1, 0,
                        1, st);
      }
      dev_dot_async(w.get(), w.get(), N, scal.get(), st);
      arnoldi_step_kernel<<<1, 32, 0, st>>>(Hd.get(), m, j, csd.get(), snd.get(), gd.get(), scal.get(),
                                             scal.get() + 1, stat.get());
      scale_by_dev_kernel<<<grid, 256, 0, st>>>(w.get(), (long long)N, scal.get() + 1, V.get() + (size_t)(j + 1) * N);
      count_launch();
      count_launch();
      check_launch("gmres arnoldi step");
      double hs[2] = {0.0, 0.0};
      TT_CUDA(cudaMemcpyAsync(hs, stat.get(), sizeof(hs), cudaMemcpyDeviceToHost, st));
      TT_CUDA(sync_stream(st));
      jl = j;
      if (hs[0] <= tol * bnorm || hs[1] == 0.0) {
        done = true;
        break;
      }
    }
    if (jl < 0) break;
    TT_CUDA(cudaMemcpyAsync(H.data(), Hd.get(), H.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaMemcpyAsync(g.data(), gd.get(), g.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(sync_stream(st));
    std::vector<double> y(jl + 1, 0.0);
    for (int i = jl; i >= 0; --i) {
      double sum = g[i];
      for (int t2 = i + 1; t2 <= jl; ++t2) sum -= H[(size_t)i * m + t2] * y[t2];
      y[i] = H[(size_t)i * m + i] != 0.0 ? sum / H[(size_t)i * m + i] : 0.0;
    }
    upload(hdev.get(), y);
    gemm_rm<double>(true, false, (int)N, 1, jl + 1, 1.0, V.get(), (int)N, 0, hdev.get(), 1, 0, 1.0, x, 1, 0, 1, st);
    if (done) break;
  }
  return total;
}

// Relative change of the local blocks below which sweeps in a reduced
// precision have converged as far as that precision allows: four unit
// roundoffs of the contraction input format.
double sweep_floor(int prec) {
  switch (prec) {
    case TT_FP32: return 4.0 * 5.96e-8;        // 2^-24
    case TT_MIXED_TF32: return 4.0 * 4.88e-4;  // 2^-11
    case TT_MIXED_BF16: return 4.0 * 3.91e-3;  // 2^-8
    default: return 0.0;
  }
}

// FP64 sweeps that refine a direction found in a reduced precision (default;
// Options::refine_sweeps)
constexpr int kRefineSweeps = 1;

// Relative truncation tolerance of a block move in a sweep of precision
// `prec`: the solve's tolerance, but not below the precision's noise floor.
// Local solutions from reduced-precision contractions carry relative noise
// of a few unit roundoffs; truncating below that level would keep noise
// directions and let the frame ranks grow with them. The closing FP64 sweep
// truncates at the solve's own tolerance.
double move_tol(double tol, int prec) { return std::max(tol, sweep_floor(prec)); }

// Returns the solution with the block index at the core where the last
// sweep ended; *warm receives the same solution moved to core 0 (truncated)
// as the warm start of the next solve.
BlockTT amen_solve(NewtonData& nd, int d, const BlockTT* w0, double tol, int cap, int kick, int max_sweeps,
                   Counter& rnd, int prec_in, int dense_max, int gmres_restart, int gmres_maxit, AmenInfo* info,
                   BlockTT* warm, const std::chrono::steady_clock::time_point* deadline,
                   int refine_sweeps = kRefineSweeps, bool fp32_factors = true) {
  // FP64 dense local solves try FP32 factors until one of them does not
  // refine to the FP64 level; the rest of this solve then factors in FP64
  bool fp32_ok = fp32_factors;
  // sweeps run in prec_in until they stall at its floor (or use the sweep
  // budget), then up to kRefineSweeps FP64 sweeps refine the direction with
  // FP64 environments, local operators and solves
  int prec = prec_in;
  int refine = 0;
  const int nblk = nd.nblk();
  cudaStream_t st = cur_stream();
  BlockTT w = w0 ? *w0 : init_block(d, nblk, kick, rnd);
  DTT frame = w.frame;  // shares cores; replaced core by core below
  frame.c = w.frame.c;
  std::shared_ptr<DBuf<double>> block = w.block;
  // environments
  std::vector<Env> eA, eAT, eK, eLZ, eLX, eTA, eAiT, eDK;
  eA.emplace_back(nd.A, nullptr, d);
  eAT.emplace_back(nd.AT, nullptr, d);
  eK.emplace_back(nd.K, nullptr, d);
  for (auto& o : nd.LZ) eLZ.emplace_back(o, nullptr, d);
  for (auto& o : nd.LX) eLX.emplace_back(o, nullptr, d);
  std::vector<std::pair<double, Env>> rp, rdd, rc, rt;
  for (auto& t : nd.rp) rp.emplace_back(t.coef, Env(t.op, &t.vec, d));
  for (auto& t : nd.rd) rdd.emplace_back(t.coef, Env(t.op, &t.vec, d));
  for (auto& t : nd.rc) rc.emplace_back(t.coef, Env(t.op, &t.vec, d));
  if (nd.ineq) {
    eTA.emplace_back(nd.TA, nullptr, d);
    eAiT.emplace_back(nd.AiT, nullptr, d);
    for (auto& o : nd.DK) eDK.emplace_back(o, nullptr, d);
    for (auto& t : nd.rt) rt.emplace_back(t.coef, Env(t.op, &t.vec, d));
  }
  // every environment's update as one job; the jobs are independent and go
  // out over side streams (fan_out)
  auto for_all = [&](auto fn) {
    std::vector<std::function<void()>> jobs;
    for (auto* v : {&eA, &eAT, &eK, &eLZ, &eLX, &eTA, &eAiT, &eDK})
      for (Env& e : *v) jobs.push_back([&fn, &e]() { fn(e); });
    for (auto* v : {&rp, &rdd, &rc, &rt})
      for (auto& pe : *v) jobs.push_back([&fn, &pe]() { fn(pe.second); });
    fan_out(jobs);
  };
  {
    ProfScope ps("amen.env_init");
    for_all([&](Env& e) {
      for (int k = d - 1; k >= 1; --k) e.push_right(frame, k, prec);
    });
  }

  std::vector<int> blockshape = {frame.r[0], 4, frame.r[1]};
  int sweep = 0;
  double max_change = 0.0;
  const int budget = max_sweeps + (prec_in != TT_FP64 ? refine_sweeps : 0);
  for (sweep = 0; sweep < budget; ++sweep) {
    const bool forward = sweep % 2 == 0;
    max_change = 0.0;
    for (int step = 0; step < d; ++step) {
      TT_CHECK(!deadline || std::chrono::steady_clock::now() < *deadline, TT_E_NO_CONVERGENCE,
               "time limit reached");
      const int k = forward ? step : d - 1 - step;
      const int rl = frame.r[k], rr = frame.r[k + 1];
      const size_t n = (size_t)rl * 4 * rr;
      const int nb = nd.ineq ? 3 : 2;
      const size_t N = nb * n;
      const size_t rc0 = (nb - 1) * n;
      auto nw = std::make_shared<DBuf<double>>(nblk * n);
      if (N > (size_t)dense_max) {
        ProfScope ps("amen.gmres_solve");
        // matrix-free reduced system (eq. reduced_kkt_system) solved by GMRES:
        // each block product inserts the vector into core k and contracts it
        // with the cached environments and the operator core
        int mv_prec = prec;  // precision of the block products (FP64 for the forcing check)
        auto apply_sum = [&](std::vector<Env>& es, const double* x, double* y, double scale, bool acc) {
          DBuf<double> tmp(n);
          if (!acc) dev_fill(y, n, 0.0, st);
          for (Env& e : es) {
            CDims c{rl, rr, e.op.r[k], e.op.r[k + 1], rl, rr, e.op.m, e.op.n};
            local_apply(c, e.L[k].get(), e.op.core(k), e.R[k + 1].get(), x, tmp.get(), mv_prec, st);
            dev_axpy(y, tmp.get(), n, scale, st);
          }
        };
        DBuf<double> r_p(n), r_d(n), r_c(n), b(N), x(N), t(n);
        sum_local_rhs(rp, frame, k, r_p.get(), n, prec);
        sum_local_rhs(rdd, frame, k, r_d.get(), n, prec);
        sum_local_rhs(rc, frame, k, r_c.get(), n, prec);
        dev_copy2d(b.get(), 1, r_p.get(), 1, n, 1, -1.0, st);
        dev_copy2d(b.get() + rc0, 1, r_c.get(), 1, n, 1, -1.0, st);
        apply_sum(eLX, r_d.get(), b.get() + rc0, 1.0, true);
        if (nd.ineq) {
          DBuf<double> r_t(n);
          sum_local_rhs(rt, frame, k, r_t.get(), n, prec);
          dev_copy2d(b.get() + n, 1, r_t.get(), 1, n, 1, -1.0, st);
        }
        auto matvec = [&](const double* xin, double* y) {
          apply_sum(eA, xin, y, -1.0, false);
          apply_sum(eK, xin + n, y, 1.0, true);
          if (nd.ineq) {
            apply_sum(eTA, xin, y + n, nd.sgn, false);
            apply_sum(eDK, xin + 2 * n, y + n, 1.0, true);
          }
          apply_sum(eAT, xin + n, t.get(), 1.0, false);
          if (nd.ineq) apply_sum(eAiT, xin + 2 * n, t.get(), -nd.sgn, true);
          apply_sum(eLZ, xin, y + rc0, 1.0, false);
          apply_sum(eLX, t.get(), y + rc0, 1.0, true);
        };
        // warm start from the block solution of the previous visit of this core
        if (blockshape[0] == rl && blockshape[2] == rr && block) dev_copy(x.get(), block->get(), N, st);
        else dev_fill(x.get(), N, 0.0, st);
        info->gmres_iters += gmres(N, matvec, b.get(), x.get(), 0.1 * tol, gmres_restart, gmres_maxit);
        {
          // forcing check: the residual of the projected system with FP64
          // products; a miss is corrected by GMRES on the FP64 residual
          const double bnorm = dev_norm(b.get(), N);
          DBuf<double> r64(N), dx(N);
          auto true_residual = [&]() {
            mv_prec = TT_FP64;
            matvec(x.get(), r64.get());
            mv_prec = prec;
            dev_scale(r64.get(), N, -1.0, st);
            dev_axpy(r64.get(), b.get(), N, 1.0, st);
            return bnorm > 0 ? dev_norm(r64.get(), N) / bnorm : 0.0;
          };
          double rho = true_residual();
          for (int c = 0; c < 2 && rho > 0.1 * tol && prec != TT_FP64; ++c) {
            dev_fill(dx.get(), N, 0.0, st);
            const double rel = std::min(0.5, 0.1 * tol / rho);
            info->gmres_iters += gmres(N, matvec, r64.get(), dx.get(), rel, gmres_restart, gmres_maxit);
            dev_axpy(x.get(), dx.get(), N, 1.0, st);
            ++info->corrections;
            rho = true_residual();
          }
          info->forcing = std::max(info->forcing, rho);
        }
        dev_copy(nw->get(), x.get(), N, st);
        double* dZ = nw->get() + (nblk - 1) * n;
        apply_sum(eAT, x.get() + n, dZ, 1.0, false);
        if (nd.ineq) apply_sum(eAiT, x.get() + 2 * n, dZ, -nd.sgn, true);
        dev_axpy(dZ, r_d.get(), n, -1.0, st);
      } else {
      ProfScope ps("amen.dense_solve");
      // local operators
      DBuf<double> A(n * n), AT(n * n), Ky(n * n), LZ(n * n), LX(n * n);
      std::optional<ProfScope> ps_part;
      ps_part.emplace("dense.local_mats");
      DBuf<double> r_p(n), r_d(n), r_c(n);
      fan_out({[&]() { eA[0].local_mat(frame, k, A.get(), prec); },
               [&]() { eAT[0].local_mat(frame, k, AT.get(), prec); },
               [&]() { eK[0].local_mat(frame, k, Ky.get(), prec); },
               [&]() { sum_local_mats(eLZ, frame, k, LZ.get(), n, prec); },
               [&]() { sum_local_mats(eLX, frame, k, LX.get(), n, prec); },
               [&]() { sum_local_rhs(rp, frame, k, r_p.get(), n, prec); },
               [&]() { sum_local_rhs(rdd, frame, k, r_d.get(), n, prec); },
               [&]() { sum_local_rhs(rc, frame, k, r_c.get(), n, prec); }});
      ps_part.reset();
      ps_part.emplace("dense.assemble");
      DBuf<double> K(N * N), b(N);
      dev_fill(K.get(), N * N, 0.0, st);
      // row block p: [-A, Ky, 0]
      dev_copy2d(K.get(), N, A.get(), n, n, n, -1.0, st);
      dev_copy2d(K.get() + n, N, Ky.get(), n, n, n, 1.0, st);
      // last row block c: [LZ, LX AT, -sgn LX AiT]
      dev_copy2d(K.get() + rc0 * N, N, LZ.get(), n, n, n, 1.0, st);
      gemm_rm<double>(false, false, n, n, n, 1.0, LX.get(), n, 0, AT.get(), n, 0, 0.0, K.get() + rc0 * N + n,
                      N, 0, 1, st);
      // right-hand sides
      dev_copy2d(b.get(), 1, r_p.get(), 1, n, 1, -1.0, st);
      dev_copy2d(b.get() + rc0, 1, r_c.get(), 1, n, 1, -1.0, st);
      gemm_rm<double>(false, false, n, 1, n, 1.0, LX.get(), n, 0, r_d.get(), 1, 0, 1.0, b.get() + rc0, 1, 0,
                      1, st);
      DBuf<double> AiT;
      if (nd.ineq) {
        DBuf<double> TA(n * n), DK(n * n), r_t(n);
        AiT.alloc(n * n);
        eTA[0].local_mat(frame, k, TA.get(), prec);
        eAiT[0].local_mat(frame, k, AiT.get(), prec);
        sum_local_mats(eDK, frame, k, DK.get(), n, prec);
        sum_local_rhs(rt, frame, k, r_t.get(), n, prec);
        // row block t: [sgn TA, 0, DK]
        dev_copy2d(K.get() + n * N, N, TA.get(), n, n, n, nd.sgn, st);
        dev_copy2d(K.get() + n * N + 2 * n, N, DK.get(), n, n, n, 1.0, st);
        gemm_rm<double>(false, false, n, n, n, -nd.sgn, LX.get(), n, 0, AiT.get(), n, 0, 0.0,
                        K.get() + rc0 * N + 2 * n, N, 0, 1, st);
        dev_copy2d(b.get() + n, 1, r_t.get(), 1, n, 1, -1.0, st);
      }
      {
        ps_part.reset();
        ProfScope ps_lu("dense.lu");
        int corr = 0;
        const double rho = lu_solve_prec(prec, (int)N, K.get(), b.get(), kLuRefineTol, &corr, (int)n, &fp32_ok);
        info->forcing = std::max(info->forcing, rho);
        info->corrections += corr;
      }
      // assemble the new block core [dX, dY, (dT), dZ]
      dev_copy(nw->get(), b.get(), nb * n, st);
      double* dZ = nw->get() + (nblk - 1) * n;
      // dZ = AT dY - sgn AiT dT - r_d
      gemm_rm<double>(false, false, n, 1, n, 1.0, AT.get(), n, 0, b.get() + n, 1, 0, 0.0, dZ, 1, 0, 1, st);
      if (nd.ineq)
        gemm_rm<double>(false, false, n, 1, n, -nd.sgn, AiT.get(), n, 0, b.get() + 2 * n, 1, 0, 1.0, dZ, 1, 0,
                        1, st);
      dev_axpy(dZ, r_d.get(), n, -1.0, st);
      }
      // convergence measure
      double nrm = dev_norm(nw->get(), nblk * n);
      if (blockshape[0] == rl && blockshape[2] == rr && block) {
        DBuf<double> diff(nblk * n);
        dev_copy(diff.get(), nw->get(), nblk * n, st);
        dev_axpy(diff.get(), block->get(), nblk * n, -1.0, st);
        max_change = std::max(max_change, dev_norm(diff.get(), nblk * n) / std::max(nrm, 1e-300));
      } else {
        max_change = std::max(max_change, 1.0);
      }
      const bool last = forward ? (k == d - 1) : (k == 0);
      if (last) {
        block = nw;
        blockshape = {rl, 4, rr};
        auto c0 = std::make_shared<DBuf<double>>(n);
        dev_copy(c0->get(), nw->get(), n, st);
        frame.c[k] = c0;
        break;
      }
      if (forward) {
        ProfScope ps("amen.move_fwd");
        const int rows = rl * 4, cols = nblk * rr;
        DBuf<double> mat((size_t)rows * cols);
        for (int bb = 0; bb < nblk; ++bb)
          dev_copy2d(mat.get() + bb * rr, cols, nw->get() + bb * n, rr, rows, rr, 1.0, st);
        int kk = std::min(rows, cols);
        DBuf<double> U((size_t)rows * kk), S(kk), Vt((size_t)kk * cols);
        // the SVD only chooses the next frame's subspace: it runs in the solve's
        // reduced precision even in the FP64 refinement sweep
        std::optional<ProfScope> ps_svd;
        ps_svd.emplace("move.svd");
        {
          // the move keeps the spectrum above move_tol / sqrt(d): directions
          // 1000 times below it need not be resolved
          const double fl = 1e-3 * move_tol(tol, prec) / std::sqrt((double)d);
          SvdNoiseFloor nf(fl * fl);
          svd_prec(prec_in, MatView<double>{mat.get(), rows, cols, cols, 1}, U.get(), S.get(), Vt.get(), st,
                   kSvdLeft);
        }
        std::vector<double> hs = host_copy(S.get(), kk);
        ps_svd.reset();
        int keep = truncation_rank_rel(hs, move_tol(tol, prec) / std::sqrt((double)d), cap);
        int extra = std::min(kick, std::min(rows - keep, std::max(cap - keep, 0)));
        int nk = keep + std::max(extra, 0);
        DBuf<double> u((size_t)rows * nk);
        dev_copy2d(u.get(), nk, U.get(), kk, rows, keep, 1.0, st);
        // with a kick, or when the SVD ran in FP32, the new frame core is
        // re-orthonormalised in FP64 (the SVD only chooses the subspace)
        if (extra > 0 || prec_in != TT_FP64) {
          if (extra > 0) {
            std::vector<double> rndv = rnd.draw((size_t)rows * extra);
            DBuf<double> rr_((size_t)rows * extra);
            upload(rr_.get(), rndv);
            dev_copy2d(u.get() + keep, nk, rr_.get(), extra, rows, extra, 1.0, st);
          }
          DBuf<double> Q((size_t)rows * nk), Rq((size_t)nk * nk);
          qr_thin<double>(MatView<double>{u.get(), rows, nk, nk, 1}, Q.get(), Rq.get(), st);
          dev_copy(u.get(), Q.get(), (size_t)rows * nk, st);
        }
        DBuf<double> coef((size_t)nk * cols);
        gemm_rm<double>(true, false, nk, cols, rows, 1.0, u.get(), nk, 0, mat.get(), cols, 0, 0.0, coef.get(),
                        cols, 0, 1, st);
        auto fk = std::make_shared<DBuf<double>>((size_t)rows * nk);
        dev_copy(fk->get(), u.get(), (size_t)rows * nk, st);
        frame.c[k] = fk;
        frame.r[k + 1] = nk;
        const int r3 = frame.r[k + 2];
        const size_t nn = (size_t)nk * 4 * r3;
        auto nb2 = std::make_shared<DBuf<double>>(nblk * nn);
        for (int bb = 0; bb < nblk; ++bb)
          gemm_rm<double>(false, false, nk, 4 * r3, rr, 1.0, coef.get() + bb * rr, cols, 0, frame.core(k + 1),
                          4 * r3, 0, 0.0, nb2->get() + bb * nn, 4 * r3, 0, 1, st);
        auto c1 = std::make_shared<DBuf<double>>(nn);
        dev_copy(c1->get(), nb2->get(), nn, st);
        frame.c[k + 1] = c1;
        block = nb2;
        blockshape = {nk, 4, r3};
        ProfScope ps_env("move.env");
        for_all([&](Env& e) { e.push_left(frame, k, prec); });
      } else {
        ProfScope ps("amen.move_bwd");
        const int rows = nblk * rl, cols = 4 * rr;
        int kk = std::min(rows, cols);
        DBuf<double> U((size_t)rows * kk), S(kk), Vt((size_t)kk * cols);
        std::optional<ProfScope> ps_svd;
        ps_svd.emplace("move.svd");
        {
          const double fl = 1e-3 * move_tol(tol, prec) / std::sqrt((double)d);
          SvdNoiseFloor nf(fl * fl);
          svd_prec(prec_in, MatView<double>{nw->get(), rows, cols, cols, 1}, U.get(), S.get(), Vt.get(), st,
                   kSvdRight);
        }
        std::vector<double> hs = host_copy(S.get(), kk);
        ps_svd.reset();
        int keep = truncation_rank_rel(hs, move_tol(tol, prec) / std::sqrt((double)d), cap);
        int extra = std::min(kick, std::min(cols - keep, std::max(cap - keep, 0)));
        int nk = keep + std::max(extra, 0);
        DBuf<double> v((size_t)cols * nk);  // cols x nk
        DBuf<double> vt_keep((size_t)keep * cols);
        dev_copy(vt_keep.get(), Vt.get(), (size_t)keep * cols, st);
        DBuf<double> vk((size_t)cols * keep);
        transpose<double>(keep, cols, vt_keep.get(), vk.get(), st);
        dev_copy2d(v.get(), nk, vk.get(), keep, cols, keep, 1.0, st);
        if (extra > 0 || prec_in != TT_FP64) {
          if (extra > 0) {
            std::vector<double> rndv = rnd.draw((size_t)cols * extra);
            DBuf<double> rr_((size_t)cols * extra);
            upload(rr_.get(), rndv);
            dev_copy2d(v.get() + keep, nk, rr_.get(), extra, cols, extra, 1.0, st);
          }
          DBuf<double> Q((size_t)cols * nk), Rq((size_t)nk * nk);
          qr_thin<double>(MatView<double>{v.get(), cols, nk, nk, 1}, Q.get(), Rq.get(), st);
          dev_copy(v.get(), Q.get(), (size_t)cols * nk, st);
        }
        DBuf<double> coef((size_t)rows * nk);  // (nblk rl) x nk
        gemm_rm<double>(false, false, rows, nk, cols, 1.0, nw->get(), cols, 0, v.get(), nk, 0, 0.0, coef.get(),
                        nk, 0, 1, st);
        auto fk = std::make_shared<DBuf<double>>((size_t)nk * cols);
        transpose<double>(cols, nk, v.get(), fk->get(), st);
        frame.c[k] = fk;
        frame.r[k] = nk;
        const int rp = frame.r[k - 1];
        const size_t nn = (size_t)rp * 4 * nk;
        auto nb2 = std::make_shared<DBuf<double>>(nblk * nn);
        for (int bb = 0; bb < nblk; ++bb)
          gemm_rm<double>(false, false, rp * 4, nk, rl, 1.0, frame.core(k - 1), rl, 0,
                          coef.get() + (size_t)bb * rl * nk, nk, 0, 0.0, nb2->get() + bb * nn, nk, 0, 1, st);
        auto c1 = std::make_shared<DBuf<double>>(nn);
        dev_copy(c1->get(), nb2->get(), nn, st);
        frame.c[k - 1] = c1;
        block = nb2;
        blockshape = {rp, 4, nk};
        ProfScope ps_env("move.env");
        for_all([&](Env& e) { e.push_right(frame, k, prec); });
      }
    }
    if (prec_in == TT_FP64) {
      if (sweep >= 1 && max_change < tol) {
        info->converged = true;
        ++sweep;
        break;
      }
    } else if (prec != TT_FP64) {
      const bool stalled = sweep >= 1 && max_change < std::max(tol, sweep_floor(prec_in));
      if (stalled) info->converged = true;
      if (stalled || sweep + 1 >= max_sweeps) {
        // switch to FP64: rebuild the environments the next sweep reads
        prec = TT_FP64;
        if (forward) {
          for (int k = 0; k + 1 < d; ++k) for_all([&](Env& e) { e.push_left(frame, k, prec); });
        } else {
          for (int k = d - 1; k >= 1; --k) for_all([&](Env& e) { e.push_right(frame, k, prec); });
        }
      }
    } else {
      ++refine;
      if (max_change < tol || refine >= refine_sweeps) {
        ++sweep;
        break;
      }
    }
  }
  info->sweeps = sweep;
  info->max_change = max_change;
  // FP64: the solve met its tolerance when the last sweep's largest block
  // change is below it (a single sweep included, whose changes are measured
  // against the warm start projected onto the new frames)
  if (prec_in == TT_FP64) info->converged = max_change < tol;
  // the solution, exact, with the block index where the last sweep left it
  const bool at_end = (sweep % 2 == 1);
  BlockTT sol;
  sol.frame = frame;
  sol.nblk = nblk;
  sol.block = block;
  sol.pos = at_end ? d - 1 : 0;
  *warm = sol;
  if (at_end) {
    // the warm start of the next solve has its block index at core 0: moving
    // it there is a sweep of block moves truncated like the sweeps' moves
    // (without truncation the frame would grow to nblk times its rank)
    for (int k = d - 1; k >= 1; --k) {
      int rl = frame.r[k], rr = frame.r[k + 1];
      int rows = nblk * rl, cols = 4 * rr;
      int kk = std::min(rows, cols);
      DBuf<double> U((size_t)rows * kk), S(kk), Vt((size_t)kk * cols);
      svd_thin<double>(MatView<double>{block->get(), rows, cols, cols, 1}, U.get(), S.get(), Vt.get(), st);
      std::vector<double> hs = host_copy(S.get(), kk);
      const int keep = truncation_rank_rel(hs, move_tol(tol, prec) / std::sqrt((double)d), cap);
      auto fk = std::make_shared<DBuf<double>>((size_t)keep * cols);
      dev_copy(fk->get(), Vt.get(), (size_t)keep * cols, st);
      frame.c[k] = fk;
      frame.r[k] = keep;
      // coef[b][a][c] = U[(b a)][c] S[c]; new block[b] = frame[k-1] coef[b]
      DBuf<double> coef((size_t)rows * keep);
      dev_copy2d(coef.get(), keep, U.get(), kk, rows, keep, 1.0, st);
      dev_scale_cols(coef.get(), rows, keep, S.get(), st);
      int rp = frame.r[k - 1];
      size_t nn = (size_t)rp * 4 * keep;
      auto nb2 = std::make_shared<DBuf<double>>(nblk * nn);
      for (int bb = 0; bb < nblk; ++bb)
        gemm_rm<double>(false, false, rp * 4, keep, rl, 1.0, frame.core(k - 1), rl, 0,
                        coef.get() + (size_t)bb * rl * keep, keep, 0, 0.0, nb2->get() + bb * nn, keep, 0, 1, st);
      auto c1 = std::make_shared<DBuf<double>>(nn);
      dev_copy(c1->get(), nb2->get(), nn, st);
      frame.c[k - 1] = c1;
      block = nb2;
    }
    warm->frame = frame;
    warm->block = block;
    warm->pos = 0;
  }
  return sol;
}

}  // namespace

double dense_local_solve(int prec, int N, double* K, double* b, int* corrections, int n_lz) {
  // FP32 factors in FP64 mode for the reduced systems only: a general system
  // is factored in FP64
  bool fp32_ok = n_lz > 0;
  return lu_solve_prec(prec, N, K, b, kLuRefineTol, corrections, n_lz, &fp32_ok);
}

void kkt_counts(unsigned long long* block, unsigned long long* fp32, unsigned long long* fallback,
                unsigned long long* not_pd, bool reset) {
  if (block) *block = g_kkt_block.load();
  if (fp32) *fp32 = g_kkt_fp32.load();
  if (fallback) *fallback = g_kkt_fallback.load();
  if (not_pd) *not_pd = g_kkt_not_pd.load();
  if (reset) {
    g_kkt_block = 0;
    g_kkt_fp32 = 0;
    g_kkt_fallback = 0;
    g_kkt_not_pd = 0;
  }
}

DTT BlockTT::component(int b) const {
  DTT t = frame;
  size_t n0 = frame.csize(pos);
  auto c0 = std::make_shared<DBuf<double>>(n0);
  dev_copy(c0->get(), block->get() + b * n0, n0, cur_stream());
  t.c[pos] = c0;
  return t;
}

// ---------------------------------------------------------------------------
// step length: alternating local generalised eigenproblems (Section 3.4)
// ---------------------------------------------------------------------------
static double local_min_eig(int nl, const double* Mk, const double* Dk, double* x) {
  cudaStream_t st = cur_stream();
  size_t nn = (size_t)nl * nl;
  DBuf<double> L(nn), tmp(nn), S(nn);
  // Ms = L L^T and S = Li Ds Li^T (Ms, Ds the symmetric parts) by the
  // bordered Cholesky; Section 3.4: an iterate that is not positive definite
  // shows in its projection; the step length is then undefined and the error
  // is raised
  std::optional<ProfScope> ps_red;
  ps_red.emplace("eig.reduce");
  TT_CHECK(chol_reduce(nl, Mk, Dk, S.get(), L.get(), st), TT_E_NOT_PD,
           "step length: the projected iterate is not positive definite");
  ps_red.reset();
  transpose<double>(nl, nl, S.get(), tmp.get(), st);
  dev_axpy(S.get(), tmp.get(), nn, 1.0, st);
  dev_scale(S.get(), nn, 0.5, st);
  // smallest eigenvector of the symmetric S from an FP32 Jacobi SVD of S + s I
  // (s >= ||S||_F makes every eigenvalue positive, so the smallest singular
  // pair is the smallest eigenpair); its eigenvalue is then the FP64 Rayleigh
  // quotient v^T S v / v^T v, whose error is second order in the FP32 error of v
  double s = dev_norm(S.get(), nn) + 1e-300;
  std::vector<double> diag(nn, 0.0);
  for (int i = 0; i < nl; ++i) diag[(size_t)i * nl + i] = s;
  DBuf<double> Sh(nn), dI(nn);
  upload(dI.get(), diag);
  dev_copy(Sh.get(), S.get(), nn, st);
  dev_axpy(Sh.get(), dI.get(), nn, 1.0, st);
  DBuf<float> Sf(nn), U(nn), Sv(nl), Vt(nn);
  to_f32(Sh.get(), Sf.get(), nn, st);
  {
    ProfScope ps_svd("eig.svd");
    svd_thin<float>(MatView<float>{Sf.get(), nl, nl, nl, 1}, U.get(), Sv.get(), Vt.get(), st, kSvdLeft);
  }
  DBuf<double> v(nl), Sv64(nl);
  transpose<float>(nl, nl, U.get(), Vt.get(), st);  // row nl-1 of U^T = last column of U
  to_f64(Vt.get() + (size_t)(nl - 1) * nl, v.get(), nl, st);
  gemm_rm<double>(false, false, nl, 1, nl, 1.0, S.get(), nl, 0, v.get(), 1, 0, 0.0, Sv64.get(), 1, 0, 1, st);
  const double num = dev_dot(v.get(), Sv64.get(), nl, st), den = dev_dot(v.get(), v.get(), nl, st);
  const double lam = den > 0 ? num / den : 0.0;
  // x = Li^T v
  gemm_rm<double>(true, false, nl, 1, nl, 1.0, L.get(), nl, 0, v.get(), 1, 0, 0.0, x, 1, 0, 1, st);
  return lam;
}

double min_gen_eig(const DTT& M, const DTT& dM, DTT* e_io, bool warm, Counter& rnd, int rank, int sweeps,
                   int prec) {
  const int d = M.d, nmode = M.m;
  cudaStream_t st = cur_stream();
  DTT e;
  if (!warm) {
    std::vector<int> r(d + 1, 1);
    for (int k = 1; k < d; ++k) {
      long long cap = 1;
      int ex = std::min(k, d - k);
      for (int t = 0; t < ex && cap < rank; ++t) cap *= nmode;
      r[k] = (int)std::min<long long>(rank, cap);
    }
    e = tt_alloc(d, r, nmode, 1);
    for (int k = 0; k < d; ++k) upload(e.core(k), rnd.draw(e.csize(k)));
  } else {
    e = tt_copy(*e_io);
  }
  e = tt_orth_right(e);
  Env eM(M, nullptr, d), eD(dM, nullptr, d);
  for (int k = d - 1; k >= 1; --k) {
    eM.push_right(e, k, prec);
    eD.push_right(e, k, prec);
  }
  double lam = std::numeric_limits<double>::infinity();
  for (int sw = 0; sw < sweeps; ++sw) {
    const bool forward = sw % 2 == 0;
    for (int step = 0; step < d; ++step) {
      const int k = forward ? step : d - 1 - step;
      const int rl = e.r[k], rr = e.r[k + 1];
      const int nl = rl * nmode * rr;
      DBuf<double> Mk((size_t)nl * nl), Dk((size_t)nl * nl), x(nl);
      eM.local_mat(e, k, Mk.get(), prec);
      eD.local_mat(e, k, Dk.get(), prec);
      {
        ProfScope ps("eig.local");
        lam = local_min_eig(nl, Mk.get(), Dk.get(), x.get());
      }
      const bool last = forward ? (k == d - 1) : (k == 0);
      if (last) {
        auto c = std::make_shared<DBuf<double>>(nl);
        dev_copy(c->get(), x.get(), nl, st);
        e.c[k] = c;
        break;
      }
      if (forward) {
        int rows = rl * nmode;
        int extra = rank > 1 ? std::max(0, std::min(rank, rows) - 1) : 0;
        int cols = rr + extra;
        DBuf<double> mat((size_t)rows * cols);
        dev_copy2d(mat.get(), cols, x.get(), rr, rows, rr, 1.0, st);
        if (extra > 0) {
          DBuf<double> rr_((size_t)rows * extra);
          upload(rr_.get(), rnd.draw((size_t)rows * extra));
          dev_copy2d(mat.get() + rr, cols, rr_.get(), extra, rows, extra, 1.0, st);
        }
        int kq = std::min(rows, cols);
        DBuf<double> Q((size_t)rows * kq), R((size_t)kq * cols);
        if (cols == rr && rank <= 1) {
          qr_thin<double>(MatView<double>{mat.get(), rows, cols, cols, 1}, Q.get(), R.get(), st);
        } else {
          qr_thin<double>(MatView<double>{mat.get(), rows, cols, cols, 1}, Q.get(), R.get(), st);
        }
        int keep = std::min(kq, rank);
        auto fk = std::make_shared<DBuf<double>>((size_t)rows * keep);
        dev_copy2d(fk->get(), keep, Q.get(), kq, rows, keep, 1.0, st);
        // coef = q^T x_mat (keep x rr); next core = coef core_{k+1}
        DBuf<double> coef((size_t)keep * rr);
        gemm_rm<double>(true, false, keep, rr, rows, 1.0, fk->get(), keep, 0, x.get(), rr, 0, 0.0, coef.get(), rr,
                        0, 1, st);
        int r3 = e.r[k + 2];
        auto nx = std::make_shared<DBuf<double>>((size_t)keep * nmode * r3);
        gemm_rm<double>(false, false, keep, nmode * r3, rr, 1.0, coef.get(), rr, 0, e.core(k + 1), nmode * r3, 0,
                        0.0, nx->get(), nmode * r3, 0, 1, st);
        e.c[k] = fk;
        e.c[k + 1] = nx;
        e.r[k + 1] = keep;
        eM.push_left(e, k, prec);
        eD.push_left(e, k, prec);
      } else {
        int cols0 = nmode * rr;
        int extra = rank > 1 ? std::max(0, std::min(rank, cols0) - 1) : 0;
        int ccount = rl + extra;
        // matT = x^T ((nmode rr) x rl) with random columns appended
        DBuf<double> matT((size_t)cols0 * ccount);
        DBuf<double> xt((size_t)cols0 * rl);
        transpose<double>(rl, cols0, x.get(), xt.get(), st);
        dev_copy2d(matT.get(), ccount, xt.get(), rl, cols0, rl, 1.0, st);
        if (extra > 0) {
          DBuf<double> rr_((size_t)cols0 * extra);
          upload(rr_.get(), rnd.draw((size_t)cols0 * extra));
          dev_copy2d(matT.get() + rl, ccount, rr_.get(), extra, cols0, extra, 1.0, st);
        }
        int kq = std::min(cols0, ccount);
        DBuf<double> Q((size_t)cols0 * kq), R((size_t)kq * ccount);
        qr_thin<double>(MatView<double>{matT.get(), cols0, ccount, ccount, 1}, Q.get(), R.get(), st);
        int keep = std::min(kq, rank);
        DBuf<double> q((size_t)cols0 * keep);
        dev_copy2d(q.get(), keep, Q.get(), kq, cols0, keep, 1.0, st);
        auto fk = std::make_shared<DBuf<double>>((size_t)keep * cols0);
        transpose<double>(cols0, keep, q.get(), fk->get(), st);
        // coef = x_mat q (rl x keep); prev core = core_{k-1} coef
        DBuf<double> coef((size_t)rl * keep);
        gemm_rm<double>(false, false, rl, keep, cols0, 1.0, x.get(), cols0, 0, q.get(), keep, 0, 0.0, coef.get(),
                        keep, 0, 1, st);
        int rp = e.r[k - 1];
        auto px = std::make_shared<DBuf<double>>((size_t)rp * nmode * keep);
        gemm_rm<double>(false, false, rp * nmode, keep, rl, 1.0, e.core(k - 1), rl, 0, coef.get(), keep, 0, 0.0,
                        px->get(), keep, 0, 1, st);
        e.c[k] = fk;
        e.c[k - 1] = px;
        e.r[k] = keep;
        eM.push_right(e, k, prec);
        eD.push_right(e, k, prec);
      }
    }
  }
  if (e_io) *e_io = tt_orth_right(e);
  return lam;
}

// Smallest rank whose discarded tail energy is at most tol^2 of the total, in [1, cap].
static int dmrg_keep(const std::vector<double>& s, double tol, int cap) {
  double tot = 0.0;
  for (double v : s) tot += v * v;
  int keep = (int)s.size();
  double tail = 0.0;
  while (keep > 1 && tail + s[keep - 1] * s[keep - 1] <= tol * tol * tot) {
    tail += s[keep - 1] * s[keep - 1];
    --keep;
  }
  return std::max(1, std::min(keep, cap));
}

// Two-site (DMRG) sweeps for min over e of <e, dM e> / <e, M e> (Section 3.4):
// at bond (k, k+1) the supercore of cores k and k+1 is the local unknown of
// the projected generalised eigenproblem built from the merged operator
// cores; the supercore is split by a truncated SVD (relative tolerance tol,
// at most `rank`), the orthonormal factor is enriched with random columns up
// to `rank` (kick) and re-orthonormalised by QR, and the other factor is the
// projection of the supercore onto it.
double min_gen_eig_dmrg(const DTT& M, const DTT& dM, DTT* e_io, bool warm, Counter& rnd, int rank, int sweeps,
                        int prec, double tol, double stall) {
  const int d = M.d, nmode = M.m;
  if (d < 2) return min_gen_eig(M, dM, e_io, warm, rnd, rank, sweeps, prec);
  cudaStream_t st = cur_stream();
  DTT e;
  if (!warm) {
    std::vector<int> r(d + 1, 1);
    for (int k = 1; k < d; ++k) {
      long long cap = 1;
      int ex = std::min(k, d - k);
      for (int t = 0; t < ex && cap < rank; ++t) cap *= nmode;
      r[k] = (int)std::min<long long>(rank, cap);
    }
    e = tt_alloc(d, r, nmode, 1);
    for (int k = 0; k < d; ++k) upload(e.core(k), rnd.draw(e.csize(k)));
  } else {
    e = tt_copy(*e_io);
  }
  e = tt_orth_right(e);
  Env eM(M, nullptr, d), eD(dM, nullptr, d);
  for (int k = d - 1; k >= 2; --k) {
    eM.push_right(e, k, prec);
    eD.push_right(e, k, prec);
  }
  std::vector<std::shared_ptr<DBuf<double>>> Mm(d - 1), Dm(d - 1);
  for (int k = 0; k + 1 < d; ++k) {
    Mm[k] = tt_merge_cores(M, k);
    Dm[k] = tt_merge_cores(dM, k);
  }
  const int n2 = nmode * nmode;
  double lam = std::numeric_limits<double>::infinity(), lam_prev = lam;
  for (int sw = 0; sw < sweeps; ++sw) {
    // stop once the quotient of a full sweep has stalled (after two sweeps)
    if (sw >= 2 && stall > 0.0 && std::fabs(lam - lam_prev) <= stall * std::fabs(lam)) break;
    lam_prev = lam;
    const bool forward = sw % 2 == 0;
    for (int step = 0; step + 1 < d; ++step) {
      const int k = forward ? step : d - 2 - step;
      const int rl = e.r[k], rr = e.r[k + 2];
      const int nl = rl * n2 * rr;
      DBuf<double> Mk((size_t)nl * nl), Dk((size_t)nl * nl), x(nl);
      CDims cm{rl, rr, M.r[k], M.r[k + 2], rl, rr, n2, n2};
      CDims cd{rl, rr, dM.r[k], dM.r[k + 2], rl, rr, n2, n2};
      local_matrix(cm, eM.L[k].get(), Mm[k]->get(), eM.R[k + 2].get(), Mk.get(), prec, st);
      local_matrix(cd, eD.L[k].get(), Dm[k]->get(), eD.R[k + 2].get(), Dk.get(), prec, st);
      {
        ProfScope ps("eig.local");
        lam = local_min_eig(nl, Mk.get(), Dk.get(), x.get());
      }
      // split the supercore (rl n) x (n rr)
      const int rows = rl * nmode, cols = nmode * rr;
      const int kk = std::min(rows, cols);
      DBuf<double> U((size_t)rows * kk), S(kk), Vt((size_t)kk * cols);
      svd_thin<double>(MatView<double>{x.get(), rows, cols, cols, 1}, U.get(), S.get(), Vt.get(), st,
                       forward ? kSvdLeft : kSvdRight);
      const int keep = dmrg_keep(host_copy(S.get(), kk), tol, rank);
      const int extra = std::max(0, std::min(rank, kk) - keep);
      const int nk = keep + extra;
      if (forward) {
        // left factor: U[:, :keep] with kick columns, orthonormal
        DBuf<double> left((size_t)rows * nk);
        dev_copy2d(left.get(), nk, U.get(), kk, rows, keep, 1.0, st);
        if (extra > 0) {
          DBuf<double> rr_((size_t)rows * extra);
          upload(rr_.get(), rnd.draw((size_t)rows * extra));
          dev_copy2d(left.get() + keep, nk, rr_.get(), extra, rows, extra, 1.0, st);
          DBuf<double> Q((size_t)rows * nk), R((size_t)nk * nk);
          qr_thin<double>(MatView<double>{left.get(), rows, nk, nk, 1}, Q.get(), R.get(), st);
          dev_copy(left.get(), Q.get(), (size_t)rows * nk, st);
        }
        auto ck = std::make_shared<DBuf<double>>((size_t)rows * nk);
        dev_copy(ck->get(), left.get(), (size_t)rows * nk, st);
        auto ck1 = std::make_shared<DBuf<double>>((size_t)nk * cols);
        gemm_rm<double>(true, false, nk, cols, rows, 1.0, left.get(), nk, 0, x.get(), cols, 0, 0.0, ck1->get(), cols,
                        0, 1, st);
        e.c[k] = ck;
        e.c[k + 1] = ck1;
        e.r[k + 1] = nk;
        eM.push_left(e, k, prec);
        eD.push_left(e, k, prec);
      } else {
        // right factor: Vt[:keep]^T with kick columns, orthonormal columns
        DBuf<double> right((size_t)cols * nk), vk((size_t)cols * keep);
        transpose<double>(keep, cols, Vt.get(), vk.get(), st);
        dev_copy2d(right.get(), nk, vk.get(), keep, cols, keep, 1.0, st);
        if (extra > 0) {
          DBuf<double> rr_((size_t)cols * extra);
          upload(rr_.get(), rnd.draw((size_t)cols * extra));
          dev_copy2d(right.get() + keep, nk, rr_.get(), extra, cols, extra, 1.0, st);
          DBuf<double> Q((size_t)cols * nk), R((size_t)nk * nk);
          qr_thin<double>(MatView<double>{right.get(), cols, nk, nk, 1}, Q.get(), R.get(), st);
          dev_copy(right.get(), Q.get(), (size_t)cols * nk, st);
        }
        auto ck1 = std::make_shared<DBuf<double>>((size_t)nk * cols);
        transpose<double>(cols, nk, right.get(), ck1->get(), st);
        auto ck = std::make_shared<DBuf<double>>((size_t)rows * nk);
        gemm_rm<double>(false, false, rows, nk, cols, 1.0, x.get(), cols, 0, right.get(), nk, 0, 0.0, ck->get(), nk,
                        0, 1, st);
        e.c[k] = ck;
        e.c[k + 1] = ck1;
        e.r[k + 1] = nk;
        eM.push_right(e, k + 1, prec);
        eD.push_right(e, k + 1, prec);
      }
    }
  }
  if (e_io) *e_io = tt_orth_right(e);
  return lam;
}


static double step_from_lambda(double lam) {
  return lam >= 0 ? std::numeric_limits<double>::infinity() : -1.0 / lam;
}

// ---------------------------------------------------------------------------
// problem assembly (Section 4)
// ---------------------------------------------------------------------------
static DTT ones_vec(int d) {
  DTT t = tt_alloc(d, std::vector<int>(d + 1, 1), 2, 1);
  for (int k = 0; k < d; ++k) dev_fill(t.core(k), 2, 1.0, cur_stream());
  return t;
}

static DTT unit_first(int d) {
  DTT t = tt_alloc(d, std::vector<int>(d + 1, 1), 2, 2);
  std::vector<double> h = {1.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < d; ++k) upload(t.core(k), h);
  return t;
}

Problem build_maxcut(const DTT& w) {
  const int d = w.d;
  Problem p;
  p.d = d;
  DTT deg = tt_matvec(w, ones_vec(d));  // A_G 1, mode 2
  p.C = tt_add(tt_diag(deg), w, 0.25, -0.25);
  DTT I = tt_identity(d, 2), J = tt_ones_mat(d, 2);
  p.A_eq = tt_diag(vecv(I));
  p.B_eq = vecv(tt_copy(I));
  p.K_y = tt_diag(vecv(tt_add(J, I, 1.0, -1.0)));
  p.lam0 = 1.0;
  return p;
}

Problem build_theta(const DTT& a) {
  const int d = a.d;
  Problem p;
  p.d = d;
  DTT I = tt_identity(d, 2), J = tt_ones_mat(d, 2), E = unit_first(d);
  DTT part1 = tt_diag(vecv(a));
  DTT part2 = tt_kron(vecv(E).view(4, 1), vecv(I).view(1, 4));  // vec_TT(E) vec_TT(I)^T
  p.A_eq = tt_add(part1, part2, 1.0, 1.0);
  p.B_eq = vecv(E);
  p.K_y = tt_diag(vecv(tt_add(tt_add(J, a, 1.0, -1.0), E, 1.0, -1.0)));
  p.C = J;
  p.lam0 = 2.0;
  return p;
}

Problem build_cc(const DTT& cp, const DTT& cm, const DTT& a) {
  const int d = a.d;
  Problem p;
  p.d = d;
  DTT deg = tt_matvec(cm, ones_vec(d));
  p.C = tt_add(tt_add(cp, tt_diag(deg), 1.0, 1.0), cm, 1.0, -1.0);
  DTT I = tt_identity(d, 2), J = tt_ones_mat(d, 2);
  p.A_eq = tt_diag(vecv(I));
  p.B_eq = vecv(tt_copy(I));
  p.K_y = tt_diag(vecv(tt_add(J, I, 1.0, -1.0)));
  p.ineq = true;
  p.A_ineq = tt_diag(vecv(a));
  p.B_ineq = tt_zeros_like_modes(d, 4, 1);
  p.K_t = tt_diag(vecv(tt_add(J, a, 1.0, -1.0)));
  p.ones_t = tt_copy(a);
  p.sgn = 1.0;
  p.q = (long long)std::llround(tt_inner(vecv(a), vecv(J)));
  p.lam0 = 2.0;
  p.lam0_ineq = 1e-3;
  return p;
}

// ---------------------------------------------------------------------------
// the interior-point iteration (Algorithm 1 with the choices of Section 3.5)
// ---------------------------------------------------------------------------
// The step-length eigensolver the options select: two-site DMRG (Section 3.4)
// or one-site ALS, FP64 throughout.
// The eigensolver's random starts and kicks come from a sub-stream of the
// main stream (forked by the caller), so how many sweeps it runs does not
// move the main stream.
static double gen_eig(const Options& o, const DTT& M, const DTT& dM, DTT* e, bool warm, Counter& sub, int rank,
                      int sweeps) {
  if (o.eig_two_site) return min_gen_eig_dmrg(M, dM, e, warm, sub, rank, sweeps, TT_FP64, kDmrgTol, kEigStall);
  return min_gen_eig(M, dM, e, warm, sub, rank, sweeps, TT_FP64);
}

void Solver::set_deadline(double seconds_from_now) {
  has_deadline_ = seconds_from_now > 0.0;
  if (has_deadline_)
    deadline_ = std::chrono::steady_clock::now() +
                std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                    std::chrono::duration<double>(seconds_from_now));
}

Solver::~Solver() {
  for (cudaStream_t s : side_) {
    sync_stream(s);
    cudaStreamDestroy(s);
  }
}

Solver::Solver(Problem p, const Options& o) : p_(std::move(p)), o_(o) {
  rnd_.seed = o.seed;
  rnd_.n = 0;
  const int d = p_.d;
  N_ = 1 << d;
  I_ = tt_identity(d, 2);
  Z_ = tt_scale(I_, p_.lam0);
  Y_ = tt_zeros_like_modes(d, 2, 2);
  if (p_.ineq) {
    DTT e;
    Counter sub = rnd_.fork();
    double lmin = gen_eig(o_, I_, p_.ones_t, &e, false, sub, 2, 6);
    double alpha_p = lmin < 0 ? p_.lam0 * step_from_lambda(lmin) : p_.lam0;
    X_ = tt_add(tt_scale(I_, p_.lam0), p_.ones_t, 1.0, alpha_p / 10.0);
    T_ = tt_scale(p_.ones_t, p_.lam0_ineq);
  } else {
    X_ = tt_scale(I_, p_.lam0);
  }
  eta_ = o.eta0;
  nB_ = tt_norm(p_.B_eq);
  nC_ = tt_norm(vecv(p_.C));
  if (p_.ineq && o.combined_multipliers && tt_is_diag_op(p_.A_eq) && tt_is_diag_op(p_.A_ineq) &&
      tt_is_diag_op(p_.K_y) && tt_is_diag_op(p_.K_t)) {
    DTT one = tt_op_diag(tt_identity(d, 4));
    ky_d_ = tt_op_diag(p_.K_y);
    kt_d_ = tt_op_diag(p_.K_t);
    pY_ = tt_add(one, ky_d_, 1.0, -1.0);
    pT_ = tt_add(one, kt_d_, 1.0, -1.0);
    if (std::fabs(tt_inner(pY_, pT_)) <= 1e-9) {
      combined_ = true;
      aeq_d_ = tt_op_diag(p_.A_eq);
      ain_d_ = tt_op_diag(p_.A_ineq);
    }
  }
}

DTT Solver::slack(const DTT& X) {
  // s = sgn (A_ineq vec X - B_ineq)
  return tt_add(tt_matvec(p_.A_ineq, vecv(X)), p_.B_ineq, p_.sgn, -p_.sgn);
}

Solver::Measures Solver::measures() {
  Measures m;
  DTT rp = tt_add(p_.B_eq, tt_matvec(p_.A_eq, vecv(X_)), 1.0, -1.0);
  DTT rd = tt_add(tt_add(vecv(Z_), vecv(p_.C), 1.0, 1.0), tt_matvec(tt_transpose(p_.A_eq), vecv(Y_)), 1.0, -1.0);
  if (p_.ineq) rd = tt_add(rd, tt_matvec(tt_transpose(p_.A_ineq), vecv(T_)), 1.0, p_.sgn);
  double comp = tt_inner(vecv(Z_), vecv(X_));
  if (p_.ineq) comp += tt_inner(vecv(T_), slack(X_));
  m.pobj = tt_inner(vecv(p_.C), vecv(X_));
  m.dobj = tt_inner(p_.B_eq, vecv(Y_));
  if (p_.ineq) m.dobj -= p_.sgn * tt_inner(p_.B_ineq, vecv(T_));
  m.abs_p = tt_norm(rp);
  m.abs_d = tt_norm(rd);
  m.comp = comp;
  m.rel_p = m.abs_p / (1.0 + nB_);
  m.rel_d = m.abs_d / (1.0 + nC_);
  m.rel_gap = comp / ((N_ + p_.q) * (1.0 + std::fabs(m.pobj)));
  m.mu = comp / (N_ + p_.q);
  return m;
}

void Solver::direction(int dir, double sigma_mu, const DTT* cx, const DTT* cz, const DTT* ct, const DTT* cs,
                       bool zero_p, bool zero_d, DTT& dX, DTT& dY, DTT& dT, DTT& dZ, int* sweeps) {
  const int d = p_.d;
  NewtonData nd;
  DTT vI = vecv(I_);
  DTT idop = tt_identity(d, 4);
  if (dir == 1) {  // AHO
    nd.LZ = {op_kron_right(Z_), op_kron_left(Z_)};
    nd.LX = {op_kron_right(X_), op_kron_left(X_)};
    nd.rc = {{1.0, op_kron_right(Z_), vecv(X_)}, {1.0, op_kron_left(Z_), vecv(X_)}, {-2.0 * sigma_mu, idop, vI}};
  } else {  // XZ
    nd.LZ = {op_kron_left(Z_)};
    nd.LX = {op_kron_right(X_)};
    nd.rc = {{1.0, op_kron_left(Z_), vecv(X_)}, {-sigma_mu, idop, vI}};
  }
  if (cx) {
    if (dir == 1) {
      nd.rc.push_back({1.0, op_kron_right(tt_transpose(*cz)), vecv(*cx)});
      nd.rc.push_back({1.0, op_kron_left(*cz), vecv(*cx)});
    } else {
      nd.rc.push_back({1.0, op_kron_left(*cz), vecv(*cx)});
    }
  }
  if (!zero_p) nd.rp = {{1.0, idop, p_.B_eq}, {-1.0, p_.A_eq, vecv(X_)}};
  else nd.rp = {{0.0, idop, vI}};
  if (!zero_d) {
    nd.rd = {{1.0, idop, vecv(Z_)}, {1.0, idop, vecv(p_.C)}, {-1.0, tt_transpose(p_.A_eq), vecv(Y_)}};
    if (p_.ineq) nd.rd.push_back({p_.sgn, tt_transpose(p_.A_ineq), vecv(T_)});
  } else {
    nd.rd = {{0.0, idop, vI}};
  }
  nd.A = p_.A_eq;
  nd.AT = tt_transpose(p_.A_eq);
  nd.K = p_.K_y;
  if (p_.ineq) {
    nd.ineq = true;
    DTT vT = vecv(T_), vG = vecv(p_.ones_t);
    nd.TA = tt_diag(tt_hadamard(vT, vG));
    DTT s = slack(X_);
    nd.DK = {tt_diag(s), p_.K_t};
    nd.AiT = tt_transpose(p_.A_ineq);
    nd.sgn = p_.sgn;
    nd.rt = {{1.0, tt_diag(vT), s}, {-sigma_mu, idop, vecv(p_.ones_t)}};
    if (ct) nd.rt.push_back({1.0, tt_diag(vecv(*ct)), *cs});
    if (combined_) combine_multipliers(nd, MaskDiagonals{pY_, pT_, aeq_d_, ain_d_, ky_d_});
  }
  AmenInfo info;
  BlockTT warm;
  BlockTT w = amen_solve(nd, d, w_ ? w_.get() : nullptr, eta_, o_.rank_cap, o_.kick, o_.max_sweeps, rnd_,
                         o_.prec, o_.local_dense_max, o_.gmres_restart, o_.gmres_max_iters, &info, &warm,
                         has_deadline_ ? &deadline_ : nullptr, o_.refine_sweeps, o_.fp32_factors != 0);
  gmres_iters_ += info.gmres_iters;
  forcing_it_ = std::max(forcing_it_, info.forcing);
  corrections_ += info.corrections;
  w_ = std::make_unique<BlockTT>(warm);
  *sweeps = info.sweeps;
  amen_ok_ = info.converged;
  dX = unvec(w.component(0));
  if (combined_) {
    const DTT dL = w.component(1);
    dY = unvec(tt_hadamard(dL, pY_));
    dT = unvec(tt_hadamard(dL, pT_));
    dZ = unvec(w.component(2));
  } else if (p_.ineq) {
    dY = unvec(w.component(1));
    dT = unvec(w.component(2));
    dZ = unvec(w.component(3));
  } else {
    dY = unvec(w.component(1));
    dZ = unvec(w.component(2));
  }
  if (dir == 0) {
    dX = tt_sym(dX);
    dY = tt_sym(dY);
    dZ = tt_sym(dZ);
    if (p_.ineq) dT = tt_sym(dT);
  }
}

double Solver::max_step(const DTT& M0, const DTT& dM, DTT* e, Counter* sub) {
  bool warm = (e == &eX_) ? haveX_ : haveZ_;
  // finishing phase: the relaxed cone M + nu I >= 0 (Section 3.5)
  const DTT M = nu_ > 0.0 ? tt_add(M0, I_, 1.0, nu_) : M0;
  Counter own;
  if (!sub) {
    own = rnd_.fork();
    sub = &own;
  }
  double lam = gen_eig(o_, M, tt_sym(dM), e, warm, *sub, o_.eig_rank, o_.eig_sweeps);
  if (e == &eX_) haveX_ = true; else haveZ_ = true;
  return step_from_lambda(lam);
}

double Solver::max_step_diag(const DTT& v, const DTT& dv, DTT* e, Counter* sub) {
  DTT idle = tt_add(vecv(tt_ones_mat(p_.d, 2)), vecv(p_.ones_t), 1.0, -1.0);
  DTT M = tt_diag(tt_add(v, idle, 1.0, 1.0));
  if (nu_ > 0.0) M = tt_add(M, tt_diag(vecv(p_.ones_t)), 1.0, nu_);
  bool warm = (e == &eS_) ? haveS_ : haveT_;
  Counter own;
  if (!sub) {
    own = rnd_.fork();
    sub = &own;
  }
  double lam = gen_eig(o_, M, tt_diag(dv), e, warm, *sub, 1, o_.eig_sweeps);
  if (e == &eS_) haveS_ = true; else haveT_ = true;
  return step_from_lambda(lam);
}

void Solver::steps(const DTT& dX, const DTT& dT, const DTT& dZ, double* ap, double* ad) {
  // The step-length eigensolves of X, Z (and of the slack and T) are
  // independent and run concurrently. Each takes the sub-stream of the main
  // random stream that the order X, Z, s, T gives it, and a failure is
  // reported as that order would report it: the first failing solve's
  // error, with the main stream and the warm starts of the solves after it
  // as if they had not run.
  DTT ds, s;
  if (p_.ineq) {
    ds = tt_matvec(p_.A_ineq, vecv(dX));
    s = slack(X_);
  }
  const int nj = p_.ineq ? 4 : 2;
  Counter sub[4], after[4];
  DTT* warm_e[4] = {&eX_, &eZ_, &eS_, &eT_};
  bool* warm_f[4] = {&haveX_, &haveZ_, &haveS_, &haveT_};
  DTT e_before[4];
  bool f_before[4];
  for (int j = 0; j < nj; ++j) {
    sub[j] = rnd_.fork();
    after[j] = rnd_;
    e_before[j] = *warm_e[j];
    f_before[j] = *warm_f[j];
  }
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  std::exception_ptr err[4];
  std::vector<std::function<void()>> jobs;
  auto guarded_job = [&](int j, std::function<double()> f) {
    jobs.push_back([&, j, f]() {
      try {
        a[j] = f();
      } catch (...) {
        err[j] = std::current_exception();
      }
    });
  };
  guarded_job(0, [&]() { return max_step(X_, dX, &eX_, &sub[0]); });
  guarded_job(1, [&]() { return max_step(Z_, dZ, &eZ_, &sub[1]); });
  if (p_.ineq) {
    guarded_job(2, [&]() { return max_step_diag(s, ds, &eS_, &sub[2]); });
    guarded_job(3, [&]() { return max_step_diag(vecv(T_), vecv(dT), &eT_, &sub[3]); });
  }
  run_concurrently(jobs, side_);
  for (int j = 0; j < nj; ++j) {
    if (!err[j]) continue;
    for (int k = j + 1; k < nj; ++k) {
      *warm_e[k] = e_before[k];
      *warm_f[k] = f_before[k];
    }
    rnd_ = after[j];
    std::rethrow_exception(err[j]);
  }
  double a_p = a[0], a_d = a[1];
  if (p_.ineq) {
    a_p = std::min(a_p, a[2]);
    a_d = std::min(a_d, a[3]);
  }
  *ap = std::min(1.0, o_.damping * a_p);
  *ad = std::min(1.0, o_.damping * a_d);
}

DTT Solver::round_psd(const DTT& Mx, double delta, const DTT* shift, int var_id) {
  double sn = shift ? tt_norm(vecv(*shift)) : 0.0;
  std::vector<int>& prev = prev_[var_id & 3];
  if ((int)prev.size() != p_.d + 1) prev.assign(p_.d + 1, 0);
  std::vector<float>& decay = decay_[var_id & 3];
  if ((int)decay.size() != p_.d + 1) decay.assign(p_.d + 1, 0.f);
  RoundHook hook;
  hook.var_id = var_id;
  hook.mu = mu_now_;
  hook.iter_frac = (double)it_ / (double)std::max(o_.max_iters, 1);
  hook.prev = &prev;
  hook.decay = &decay;
  hook.pred = pred_.get();
  hook.rnd = &rnd_;
  if (trace_) {
    hook.trace_x = &trace_x_;
    hook.trace_y = &trace_y_;
  }
  auto rz = tt_round(vecv(Mx), delta / (1.0 + sn), o_.rank_cap, &hook);
  if (hook.used) pred_used_ += hook.used;
  if (hook.fallbacks) pred_fallbacks_ += hook.fallbacks;
  DTT rounded = unvec(rz.first);
  double zeta = rz.second;
  if (shift && zeta > 0) rounded = tt_add(rounded, *shift, 1.0, zeta);
  if (rounded.maxrank() >= Mx.maxrank() && Mx.maxrank() <= o_.rank_cap) return Mx;
  return rounded;
}

bool Solver::mehrotra(int dir, double mu, bool zp, bool zd, DTT& dX, DTT& dY, DTT& dT, DTT& dZ, double* ap,
                      double* ad, int* sw) {
  DTT dXa, dYa, dTa, dZa;
  direction(dir, 0.0, nullptr, nullptr, nullptr, nullptr, zp, zd, dXa, dYa, dTa, dZa, sw);
  bool ok = amen_ok_;
  double apa, ada;
  {
    ProfScope ps("ipm.steps");
    steps(dXa, dTa, dZa, &apa, &ada);
  }
  DTT Xa = tt_add(X_, dXa, 1.0, apa), Za = tt_add(Z_, dZa, 1.0, ada);
  double mu_aff = tt_inner(vecv(Za), vecv(Xa));
  DTT dsa;
  if (p_.ineq) {
    DTT Ta = tt_add(T_, dTa, 1.0, ada);
    mu_aff += tt_inner(vecv(Ta), slack(Xa));
    dsa = tt_matvec(p_.A_ineq, vecv(dXa));
  }
  mu_aff /= (N_ + p_.q);
  double ratio = std::min(1.0, std::max(0.0, mu_aff / mu));
  double sigma = ratio * ratio * ratio;
  direction(dir, sigma * mu, &dXa, &dZa, p_.ineq ? &dTa : nullptr, p_.ineq ? &dsa : nullptr, zp, zd, dX, dY, dT,
            dZ, sw);
  ok = ok && amen_ok_;
  {
    ProfScope ps("ipm.steps");
    steps(dX, dT, dZ, ap, ad);
  }
  return ok;
}

void Solver::apply_update() {
  ProfScope ps_round("ipm.round");
  const Update& u = last_;
  DTT Xn = tt_add(u.X, u.dX, 1.0, u.ap), Zn = tt_add(u.Z, u.dZ, 1.0, u.ad), Yn = tt_add(u.Y, u.dY, 1.0, u.ad), Tn;
  if (p_.ineq) Tn = tt_add(u.T, u.dT, 1.0, u.ad);
  DTT Xr, Zr, Yr, Tr;
  std::vector<std::function<void()>> jobs;
  jobs.push_back([&]() { Xr = round_psd(Xn, u.tol_p, &I_, 0); });
  jobs.push_back([&]() { Zr = round_psd(Zn, u.tol_d, &I_, 3); });
  jobs.push_back([&]() { Yr = round_psd(Yn, u.tol_d, nullptr, 1); });
  if (p_.ineq) jobs.push_back([&]() { Tr = round_psd(Tn, u.tol_d, &p_.ones_t, 2); });
  if (pred_ || trace_) {
    // the predictor's random sketches and the trace share one stream of
    // draws and one record: keep their order fixed
    for (auto& j : jobs) j();
  } else {
    // the roundings of X, Z, y and t are independent
    run_concurrently(jobs, side_);
  }
  X_ = std::move(Xr);
  Z_ = std::move(Zr);
  Y_ = std::move(Yr);
  if (p_.ineq) T_ = std::move(Tr);
}

bool Solver::redo_update(double alpha_p, double alpha_d) {
  if (!last_.valid) return false;
  if (alpha_p >= 0.0) last_.ap = alpha_p;
  if (alpha_d >= 0.0) last_.ad = alpha_d;
  apply_update();
  return true;
}

IterLog Solver::iterate() {
  // an update that the next step-length solve finds outside the cone is
  // undone and repeated with both step lengths halved (the damp-and-retry
  // safeguard of Section 3.5), at most kMaxRetries times
  for (int attempt = 0;; ++attempt) {
    try {
      IterLog log = iterate_once();
      log.retries = retries_;
      log.fallbacks = fallbacks_;
      return log;
    } catch (const TTError& e) {
      if (e.status != TT_E_NOT_PD || !last_.valid || attempt >= kMaxRetries) throw;
      last_.ap *= 0.5;
      last_.ad *= 0.5;
      apply_update();
      ++retries_;
    }
  }
}

namespace {
// CUDA events of one iteration's device time, released on every path
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    TT_CUDA(cudaEventCreate(&a));
    TT_CUDA(cudaEventCreate(&b));
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

// The finishing phase of Section 3.5 ("Relaxing the Positive Definiteness
// Barrier"): once the relative criteria hold and an absolute tolerance is
// set, iterations take the Mehrotra direction without zeroed residual blocks
// and step lengths for the relaxed cone M + nu I >= 0; an update is kept only
// if it lowers the merit ||R_p||_F + ||R_d||_F + |<X, Z> + <vec T, s>| while
// the relative criteria still hold. Otherwise the previous iterate is kept and
// nu grows tenfold up to nu_max, after which the phase ends.
void Solver::finish_iteration(IterLog& log, const Measures& ms) {
  if (nu_ == 0.0) nu_ = o_.nu0;
  log.finishing = 1;
  log.nu = nu_;
  const double merit = ms.abs_p + ms.abs_d + std::fabs(ms.comp);
  log.merit = merit;
  eta_ = std::max(std::min(eta_, o_.eta_C * ms.mu), o_.eta_floor);
  int dir = it_ < o_.xz_warmup ? 0 : 1;
  DTT dX, dY, dT, dZ;
  double ap = 0.0, ad = 0.0;
  int sw = 0;
  mehrotra(dir, ms.mu, false, false, dX, dY, dT, dZ, &ap, &ad, &sw);
  log.alpha_p = ap;
  log.alpha_d = ad;
  log.direction = dir;
  log.sweeps = sw;
  log.max_rank_W = w_->frame.maxrank();
  const DTT X0 = X_, Y0 = Y_, T0 = T_, Z0 = Z_;
  last_.X = X_;
  last_.Y = Y_;
  last_.T = T_;
  last_.Z = Z_;
  last_.dX = dX;
  last_.dY = dY;
  last_.dT = dT;
  last_.dZ = dZ;
  last_.ap = ap;
  last_.ad = ad;
  last_.tol_p = eta_ * (1.0 + nB_) / 10.0;
  last_.tol_d = eta_ * (1.0 + nC_) / 10.0;
  last_.valid = true;
  apply_update();
  const Measures mn = measures();
  const double eps = 2.0 * o_.eps_gap, eps_c = o_.eps_gap / std::sqrt((double)p_.d);
  const double merit_new = mn.abs_p + mn.abs_d + std::fabs(mn.comp);
  if (mn.rel_p <= eps && mn.rel_d <= eps && mn.rel_gap <= eps_c && merit_new < merit) {
    log.accepted = 1;
  } else {
    log.accepted = 0;
    X_ = X0;
    Y_ = Y0;
    T_ = T0;
    Z_ = Z0;
    last_.valid = false;
    if (nu_ >= o_.nu_max) finish_done_ = true;
    nu_ = std::min(10.0 * nu_, o_.nu_max);
  }
  ++it_;
}

IterLog Solver::iterate_once() {
  cudaStream_t st = cur_stream();
  EventPair ev;
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  TT_CUDA(cudaEventRecord(e0, st));
  IterLog log;
  log.iter = it_;
  forcing_it_ = 0.0;
  Measures ms;
  {
    ProfScope ps("ipm.measures");
    ms = measures();
  }
  log.mu = ms.mu;
  mu_now_ = ms.mu;
  log.rel_p = ms.rel_p;
  log.rel_d = ms.rel_d;
  log.rel_gap = ms.rel_gap;
  log.pobj = ms.pobj;
  log.dobj = ms.dobj;
  const double eps_p = 2.0 * o_.eps_gap, eps_d = 2.0 * o_.eps_gap;
  const double eps_c = o_.eps_gap / std::sqrt((double)p_.d);
  TT_CHECK(std::isfinite(ms.mu) && std::isfinite(ms.rel_p) && std::isfinite(ms.rel_d), TT_E_NUMERIC,
           "non-finite residual");
  const bool rel_ok = ms.rel_p <= eps_p && ms.rel_d <= eps_d && ms.rel_gap <= eps_c;
  const double ft = o_.finish_tol;
  if (rel_ok && ft > 0.0 && !finish_done_ &&
      (ms.abs_p < ft && ms.abs_d < ft && std::fabs(ms.comp) < ft))
    finish_done_ = true;  // the absolute criteria of the finishing phase hold
  if (rel_ok && (ft <= 0.0 || finish_done_)) {
    log.converged = 1;
  } else if (rel_ok) {
    finish_iteration(log, ms);
  } else {
    eta_ = std::max(std::min(eta_, o_.eta_C * ms.mu), o_.eta_floor);
    int dir = it_ < o_.xz_warmup ? 0 : 1;
    const bool zp = ms.rel_p <= eps_p, zd = ms.rel_d <= eps_d;
    DTT dX, dY, dT, dZ;
    double ap = 0.0, ad = 0.0;
    int sw = 0;
    bool ok = mehrotra(dir, ms.mu, zp, zd, dX, dY, dT, dZ, &ap, &ad, &sw);
    if (dir == 1 && (std::min(ap, ad) < kFallbackStep || !ok)) {
      // Section 3.5: an AHO solve that misses its target within the rank and
      // sweep budget, or whose admissible step is nearly zero, is redone with
      // the XZ direction for this iteration
      dir = 0;
      ++fallbacks_;
      mehrotra(dir, ms.mu, zp, zd, dX, dY, dT, dZ, &ap, &ad, &sw);
    }
    log.alpha_p = ap;
    log.alpha_d = ad;
    log.direction = dir;
    log.sweeps = sw;
    log.max_rank_W = w_->frame.maxrank();
    last_.X = X_;
    last_.Y = Y_;
    last_.T = T_;
    last_.Z = Z_;
    last_.dX = dX;
    last_.dY = dY;
    last_.dT = dT;
    last_.dZ = dZ;
    last_.ap = ap;
    last_.ad = ad;
    last_.tol_p = eta_ * (1.0 + nB_) / 10.0;
    last_.tol_d = eta_ * (1.0 + nC_) / 10.0;
    last_.valid = true;
    apply_update();
    ++it_;
  }
  log.max_rank_X = X_.maxrank();
  log.max_rank_Z = Z_.maxrank();
  log.gmres_iters = gmres_iters_;
  log.forcing = forcing_it_;
  log.forcing_corrections = corrections_;
  log.pred_used = pred_used_;
  log.pred_fallbacks = pred_fallbacks_;
  if ((o_.prec == TT_MIXED_TF32 || o_.prec == TT_MIXED_BF16) && tc_check_error(true))
    throw TTError(TT_E_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  TT_CUDA(cudaEventRecord(e1, st));
  TT_CUDA(cudaEventSynchronize(e1));
  float msec = 0.f;
  TT_CUDA(cudaEventElapsedTime(&msec, e0, e1));
  log.seconds = msec * 1e-3;
  return log;
}

}  // namespace ttsdp
