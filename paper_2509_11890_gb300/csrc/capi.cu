// extern "C" boundary: argument checking, stream scoping and the conversion
// of library exceptions into status codes.
#include <cstring>
#include <string>

#include "contract.cuh"
#include "solver.cuh"
#include "tt.cuh"

using namespace ttsdp;

namespace {

thread_local std::string g_last_error;

struct StreamGuard {
  cudaStream_t prev;
  explicit StreamGuard(void* s) : prev(StreamScope::current()) { StreamScope::current() = (cudaStream_t)s; }
  ~StreamGuard() { StreamScope::current() = prev; }
};

// The solver allocates many small scratch buffers stream-ordered; keep freed
// blocks in the device's default pool instead of returning them to the driver
// at every synchronisation (the pool's default release threshold is 0).
void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static thread_local int done_for = -1;
  if (done_for == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    // a block freed on one stream is not handed to another stream behind an
    // inserted wait: with many streams (concurrent solves) such waits chain
    // the streams together; the pool grows instead
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  }
  done_for = dev;
}

template <typename F>
tt_status guarded(void* stream, F&& fn) {
  try {
    StreamGuard g(stream);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      g_last_error = "no CUDA device";
      return TT_E_CUDA;
    }
    keep_pool_memory();
    fn();
    g_last_error.clear();
    return TT_OK;
  } catch (const TTError& e) {
    g_last_error = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return TT_E_NOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return TT_E_INTERNAL;
  }
}

CDims to_cdims(const tt_contract_dims* d) {
  TT_CHECK(d != nullptr, TT_E_INVALID_ARG, "null dims");
  TT_CHECK(d->rw > 0 && d->rw2 > 0 && d->R > 0 && d->R2 > 0 && d->rv > 0 && d->rv2 > 0 && d->m > 0 && d->n > 0,
           TT_E_SHAPE, "dimensions must be positive");
  return CDims{d->rw, d->rw2, d->R, d->R2, d->rv, d->rv2, d->m, d->n};
}

void check_desc(const tt_desc* a) {
  TT_CHECK(a && a->d > 0 && a->ranks && a->cores && a->m > 0 && a->n > 0, TT_E_INVALID_ARG, "bad tt_desc");
}

DTT desc_dev(const tt_desc* a) {
  check_desc(a);
  return tt_from_device(a->d, a->ranks, a->m, a->n, a->cores);
}

DTT desc_host(const tt_desc* a) {
  check_desc(a);
  return tt_from_host(a->d, a->ranks, a->m, a->n, a->cores);
}

Options to_options(const tt_sdp_options* o) {
  Options r;
  if (!o) return r;
  r.eps_gap = o->eps_gap;
  r.rank_cap = o->rank_cap;
  r.xz_warmup = o->xz_warmup;
  r.eta0 = o->eta0;
  r.eta_floor = o->eta_floor;
  r.eta_C = o->eta_C;
  r.damping = o->damping;
  r.prec = o->precision;
  r.max_iters = o->max_iters;
  r.max_sweeps = o->max_sweeps;
  r.kick = o->kick;
  r.eig_rank = o->eig_rank;
  r.eig_sweeps = o->eig_sweeps;
  r.seed = o->seed;
  r.local_dense_max = o->local_dense_max;
  r.gmres_restart = o->gmres_restart;
  r.gmres_max_iters = o->gmres_max_iters;
  r.eig_two_site = o->eig_two_site;
  r.time_limit = o->time_limit;
  r.combined_multipliers = o->combined_multipliers;
  r.finish_tol = o->finish_tol;
  r.nu0 = o->nu0;
  r.nu_max = o->nu_max;
  r.refine_sweeps = o->refine_sweeps;
  r.fp32_factors = o->fp32_factors;
  TT_CHECK(r.fp32_factors == 0 || r.fp32_factors == 1, TT_E_INVALID_ARG, "fp32_factors must be 0 or 1");
  TT_CHECK(r.refine_sweeps >= 1 && r.refine_sweeps <= 8, TT_E_INVALID_ARG, "refine_sweeps must be in 1..8");
  TT_CHECK(r.finish_tol >= 0.0 && r.nu0 > 0.0 && r.nu_max >= r.nu0, TT_E_INVALID_ARG,
           "finishing phase: finish_tol >= 0 and 0 < nu0 <= nu_max");
  TT_CHECK(r.combined_multipliers == 0 || r.combined_multipliers == 1, TT_E_INVALID_ARG,
           "combined_multipliers must be 0 or 1");
  TT_CHECK(r.time_limit >= 0.0, TT_E_INVALID_ARG, "time_limit must be >= 0");
  TT_CHECK(r.eig_two_site == 0 || r.eig_two_site == 1, TT_E_INVALID_ARG, "eig_two_site must be 0 or 1");
  TT_CHECK(r.local_dense_max >= 0 && r.gmres_restart > 0 && r.gmres_max_iters > 0, TT_E_INVALID_ARG,
           "invalid local solver options");
  TT_CHECK(r.rank_cap > 0 && r.max_sweeps > 0 && r.eig_sweeps > 0 && r.eig_rank > 0 && r.kick >= 0,
           TT_E_INVALID_ARG, "invalid options");
  TT_CHECK(r.prec >= TT_FP64 && r.prec <= TT_MIXED_BF16, TT_E_INVALID_ARG, "unknown precision");
  return r;
}

}  // namespace

struct tt_sdp_ctx {
  cudaStream_t stream;
  std::unique_ptr<Solver> solver;
  tt_allocator alloc{nullptr, nullptr, nullptr};
  bool has_alloc = false;
  std::vector<tt_sdp_ctx*> members;  // a batch context owns its instances
  bool batch = false;
  const tt_allocator* allocator() const { return has_alloc ? &alloc : nullptr; }
};

namespace {
// Scope of a call on a context: its stream and its allocator
struct AllocGuard {
  const tt_allocator* prev;
  explicit AllocGuard(const tt_allocator* a) : prev(AllocScope::current()) { AllocScope::current() = a; }
  ~AllocGuard() { AllocScope::current() = prev; }
};

template <typename F>
tt_status ctx_guarded(tt_sdp_ctx* ctx, F&& fn) {
  AllocGuard ag(ctx->allocator());
  return guarded(ctx->stream, std::forward<F>(fn));
}

tt_allocator copy_allocator(const tt_allocator* a) {
  TT_CHECK(!a || (a->alloc && a->free), TT_E_INVALID_ARG, "tt_allocator needs both alloc and free");
  return a ? *a : tt_allocator{nullptr, nullptr, nullptr};
}
}  // namespace

extern "C" {

const char* tt_sdp_status_string(tt_status s) {
  switch (s) {
    case TT_OK: return "ok";
    case TT_E_INVALID_ARG: return "invalid argument";
    case TT_E_SHAPE: return "shape mismatch";
    case TT_E_NOMEM: return "out of memory";
    case TT_E_CUDA: return "CUDA error";
    case TT_E_NOT_PD: return "iterate not positive definite";
    case TT_E_RANK_CAP: return "rank cap bound";
    case TT_E_NO_CONVERGENCE: return "no convergence";
    case TT_E_TIMEOUT: return "device wait timed out";
    case TT_E_NUMERIC: return "non-finite value";
    case TT_E_INTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* tt_last_error(void) { return g_last_error.c_str(); }

uint64_t tt_launch_count(void) { return LaunchCounter::value(); }

void tt_contraction_stats(double* flops, double* seconds) {
  try {
    stats_read(flops, seconds);
  } catch (...) {
    if (flops) *flops = 0;
    if (seconds) *seconds = 0;
  }
}

void tt_contraction_stats_reset(void) {
  try {
    stats_reset();
  } catch (...) {
  }
}

void tt_tc_stats(double* flops, double* seconds, uint64_t* launches) {
  try {
    unsigned long long c = 0;
    stats_read(flops, seconds, 1, &c);
    if (launches) *launches = c;
  } catch (...) {
    if (flops) *flops = 0;
    if (seconds) *seconds = 0;
    if (launches) *launches = 0;
  }
}

void tt_gemm64_stats(double* flops, double* seconds, uint64_t* launches) {
  try {
    unsigned long long c = 0;
    stats_read(flops, seconds, 3, &c);
    if (launches) *launches = c;
  } catch (...) {
    if (flops) *flops = 0;
    if (seconds) *seconds = 0;
    if (launches) *launches = 0;
  }
}

void tt_lu_stats(double* flops, double* seconds, uint64_t* calls) {
  try {
    unsigned long long c = 0;
    stats_read(flops, seconds, 2, &c);
    if (calls) *calls = c;
  } catch (...) {
    if (flops) *flops = 0;
    if (seconds) *seconds = 0;
    if (calls) *calls = 0;
  }
}

size_t tt_core_count(int32_t d, const int32_t* ranks, int32_t m, int32_t n) {
  if (d <= 0 || !ranks) return 0;
  size_t s = 0;
  for (int k = 0; k < d; ++k) s += (size_t)ranks[k] * m * n * ranks[k + 1];
  return s;
}

tt_status tt_env_left_step(const tt_contract_dims* dims, const double* phi, const double* u, const double* op,
                           const double* v, double* out, int32_t precision, void* stream) {
  return guarded(stream, [&] {
    CDims c = to_cdims(dims);
    TT_CHECK(phi && u && op && v && out, TT_E_INVALID_ARG, "null pointer");
    env_left_step(c, phi, u, op, v, out, precision, cur_stream());
  });
}

tt_status tt_env_right_step(const tt_contract_dims* dims, const double* psi, const double* u, const double* op,
                            const double* v, double* out, int32_t precision, void* stream) {
  return guarded(stream, [&] {
    CDims c = to_cdims(dims);
    TT_CHECK(psi && u && op && v && out, TT_E_INVALID_ARG, "null pointer");
    env_right_step(c, psi, u, op, v, out, precision, cur_stream());
  });
}

tt_status tt_local_apply(const tt_contract_dims* dims, const double* phi, const double* op, const double* psi,
                         const double* x, double* y, int32_t precision, void* stream) {
  return guarded(stream, [&] {
    CDims c = to_cdims(dims);
    TT_CHECK(phi && op && psi && x && y, TT_E_INVALID_ARG, "null pointer");
    local_apply(c, phi, op, psi, x, y, precision, cur_stream());
  });
}

tt_status tt_local_matrix(const tt_contract_dims* dims, const double* phi, const double* op, const double* psi,
                          double* out, int32_t precision, void* stream) {
  return guarded(stream, [&] {
    CDims c = to_cdims(dims);
    TT_CHECK(phi && op && psi && out, TT_E_INVALID_ARG, "null pointer");
    local_matrix(c, phi, op, psi, out, precision, cur_stream());
  });
}

tt_status tt_hadamard(const tt_desc* a, const tt_desc* b, double* out, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(out, TT_E_INVALID_ARG, "null output");
    DTT r = tt_hadamard(desc_dev(a), desc_dev(b));
    tt_to_device(r, out);
  });
}

tt_status tt_matvec(const tt_desc* op, const tt_desc* v, double* out, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(out, TT_E_INVALID_ARG, "null output");
    DTT r = tt_matvec(desc_dev(op), desc_dev(v));
    tt_to_device(r, out);
  });
}

tt_status tt_inner(const tt_desc* a, const tt_desc* b, double* out, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(out, TT_E_INVALID_ARG, "null output");
    *out = tt_inner(desc_dev(a), desc_dev(b));
  });
}

tt_status tt_min_gen_eig(const tt_desc* M, const tt_desc* dM, int32_t rank, int32_t sweeps, int32_t two_site,
                         uint64_t seed, double* lambda, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(lambda && rank > 0 && sweeps > 0 && (two_site == 0 || two_site == 1), TT_E_INVALID_ARG,
             "bad tt_min_gen_eig arguments");
    DTT a = desc_dev(M), b = desc_dev(dM);
    TT_CHECK(a.d == b.d && a.m == b.m && a.n == b.n && a.m == a.n, TT_E_SHAPE,
             "tt_min_gen_eig: M and dM must be square TT matrices with equal modes");
    Counter rnd;
    rnd.seed = seed;
    *lambda = two_site ? min_gen_eig_dmrg(a, b, nullptr, false, rnd, rank, sweeps, TT_FP64, kDmrgTol)
                       : min_gen_eig(a, b, nullptr, false, rnd, rank, sweeps, TT_FP64);
  });
}

tt_status tt_round(const tt_desc* in, double delta, int32_t rank_cap, int32_t* ranks_out, double* cores_out,
                   size_t capacity, double* zeta_out, int32_t precision, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(ranks_out && cores_out && zeta_out && delta >= 0.0, TT_E_INVALID_ARG, "bad tt_round arguments");
    TT_CHECK(precision == TT_FP64, TT_E_INVALID_ARG, "rounding runs in FP64");
    DTT a = desc_dev(in);
    auto rz = tt_round(a, delta, rank_cap);
    TT_CHECK(rz.first.count() <= capacity, TT_E_NOMEM, "output capacity too small");
    tt_to_device(rz.first, cores_out);
    for (int k = 0; k <= rz.first.d; ++k) ranks_out[k] = rz.first.r[k];
    *zeta_out = rz.second;
    TT_CUDA(sync_stream(cur_stream()));
  });
}

tt_status tt_lu_solve(int32_t n, const double* K, double* b, int32_t precision, double* rel_residual,
                      void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(n > 0 && K && b && rel_residual, TT_E_INVALID_ARG, "bad tt_lu_solve arguments");
    TT_CHECK(precision >= TT_FP64 && precision <= TT_MIXED_BF16, TT_E_INVALID_ARG, "unknown precision");
    int corr = 0;
    *rel_residual = dense_local_solve(precision, n, const_cast<double*>(K), b, &corr);
    TT_CUDA(sync_stream(cur_stream()));
  });
}

tt_status tt_kkt_solve(int32_t n, int32_t n_lz, const double* K, double* b, int32_t precision,
                       double* rel_residual, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(n > 0 && n_lz > 0 && n_lz < n && K && b && rel_residual, TT_E_INVALID_ARG,
             "bad tt_kkt_solve arguments");
    TT_CHECK(precision >= TT_FP64 && precision <= TT_MIXED_BF16, TT_E_INVALID_ARG, "unknown precision");
    int corr = 0;
    *rel_residual = dense_local_solve(precision, n, const_cast<double*>(K), b, &corr, n_lz);
    TT_CUDA(sync_stream(cur_stream()));
  });
}

void tt_kkt_stats(uint64_t* block_solves, uint64_t* fp32_factor_solves, uint64_t* lu_fallbacks,
                  uint64_t* lz_not_pd, int32_t reset) {
  unsigned long long a = 0, h = 0, f = 0, z = 0;
  kkt_counts(&a, &h, &f, &z, reset != 0);
  if (block_solves) *block_solves = a;
  if (fp32_factor_solves) *fp32_factor_solves = h;
  if (lu_fallbacks) *lu_fallbacks = f;
  if (lz_not_pd) *lz_not_pd = z;
}

tt_status tt_sdp_round(const tt_desc* in, double tol, int32_t rank_cap, int32_t psd_shift, tt_desc* out,
                       double* zeta_out, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(out && out->ranks && zeta_out && tol >= 0.0 && psd_shift >= 0 && psd_shift <= 2, TT_E_INVALID_ARG,
             "bad tt_sdp_round arguments");
    const DTT a = desc_host(in);
    TT_CHECK(psd_shift == 0 || a.m == a.n, TT_E_SHAPE, "a spectral shift needs a square TT matrix");
    // shift S of Corollary psdness_rounding: I for X and Z, J - I for T
    DTT S;
    double sn = 0.0;
    if (psd_shift == 1) S = tt_identity(a.d, a.m);
    if (psd_shift == 2) S = tt_add(tt_ones_mat(a.d, a.m), tt_identity(a.d, a.m), 1.0, -1.0);
    if (psd_shift) sn = tt_norm(S);
    auto rz = tt_round(a.view(a.m * a.n, 1), tol / (1.0 + sn), rank_cap);
    DTT r = rz.first.view(a.m, a.n);
    if (psd_shift && rz.second > 0.0) r = tt_add(r, S, 1.0, rz.second);
    int32_t* ranks = const_cast<int32_t*>(out->ranks);
    for (int k = 0; k <= r.d; ++k) ranks[k] = r.r[k];
    out->d = r.d;
    out->m = r.m;
    out->n = r.n;
    if (out->cores) tt_to_host(r, const_cast<double*>(out->cores));
    *zeta_out = rz.second;
    TT_CUDA(sync_stream(cur_stream()));
  });
}

tt_status tt_from_dense(const double* dense, int32_t d, int32_t n, double eps_rel, int32_t rank_cap,
                        int32_t* ranks_out, double* cores_out, size_t* count, void* stream) {
  return guarded(stream, [&] {
    TT_CHECK(dense && ranks_out && count && d >= 1 && n >= 1 && eps_rel >= 0.0, TT_E_INVALID_ARG,
             "bad tt_from_dense arguments");
    DTT t = tt_from_dense(dense, d, n, eps_rel, rank_cap);
    for (int k = 0; k <= d; ++k) ranks_out[k] = t.r[k];
    size_t need = t.count();
    if (cores_out) {
      TT_CHECK(*count >= need, TT_E_NOMEM, "capacity too small");
      tt_to_host(t, cores_out);
    }
    *count = need;
  });
}

void tt_sdp_default_options(tt_sdp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps_gap = 1e-4;
  o->rank_cap = 16;
  o->xz_warmup = 3;
  o->eta0 = 1e-3;
  o->eta_floor = 1e-4;
  o->eta_C = 2.0;
  o->damping = 0.95;
  o->precision = TT_FP64;
  o->max_iters = 60;
  o->max_sweeps = 4;
  o->kick = 4;
  o->eig_rank = 4;
  o->eig_sweeps = 4;
  o->seed = 1234;
  o->local_dense_max = 8192;
  o->gmres_restart = 40;
  o->gmres_max_iters = 400;
  o->eig_two_site = 1;
  o->time_limit = 0.0;
  o->combined_multipliers = 1;
  o->finish_tol = 0.0;
  o->nu0 = 1e-6;
  o->nu_max = 1e-3;
  o->refine_sweeps = 1;
  o->fp32_factors = 1;
}

}  // extern "C"

// Creates a context whose problem `build` assembles on the device. The
// allocator struct is copied into the context first, so that every buffer
// (the problem's included) refers to the context's own copy.
template <typename B>
static tt_status make_ctx(B&& build, const tt_sdp_options* opts, void* stream, tt_sdp_ctx** out,
                          const tt_allocator* allocator = nullptr) {
  auto* ctx = new tt_sdp_ctx;
  ctx->stream = (cudaStream_t)stream;
  tt_status s = guarded(stream, [&] {
    TT_CHECK(out, TT_E_INVALID_ARG, "null output");
    ctx->alloc = copy_allocator(allocator);
    ctx->has_alloc = allocator != nullptr;
    Options o = to_options(opts);
    AllocGuard ag(ctx->allocator());
    Problem p = build();
    ctx->solver = std::make_unique<Solver>(std::move(p), o);
    *out = ctx;
  });
  if (s != TT_OK) {
    try {
      AllocGuard ag(ctx->allocator());
      StreamGuard g(stream);
      ctx->solver.reset();
    } catch (...) {
    }
    delete ctx;
  }
  return s;
}

// The Problem of a tt_sdp_problem (host cores copied to the device)
static Problem problem_from(const tt_sdp_problem* prob) {
  Problem p;
  {
    TT_CHECK(prob, TT_E_INVALID_ARG, "null problem");
    p.d = prob->C.d;
    p.C = desc_host(&prob->C);
    p.A_eq = desc_host(&prob->A_eq);
    p.B_eq = desc_host(&prob->B_eq);
    p.K_y = desc_host(&prob->K_y);
    TT_CHECK(p.C.m == 2 && p.C.n == 2 && p.A_eq.m == 4 && p.A_eq.n == 4 && p.B_eq.m == 4 && p.K_y.m == 4,
             TT_E_SHAPE, "problem modes");
    TT_CHECK(p.A_eq.d == p.d && p.B_eq.d == p.d && p.K_y.d == p.d, TT_E_SHAPE, "problem orders differ");
    if (prob->A_ineq.d > 0) {
      p.ineq = true;
      p.A_ineq = desc_host(&prob->A_ineq);
      p.B_ineq = desc_host(&prob->B_ineq);
      p.K_t = desc_host(&prob->K_t);
      p.ones_t = desc_host(&prob->ones_t);
      p.sgn = prob->ineq_sign >= 0 ? 1.0 : -1.0;
      p.q = prob->q;
    }
    p.lam0 = prob->lam0 > 0 ? prob->lam0 : 1.0;
    p.lam0_ineq = prob->lam0_ineq > 0 ? prob->lam0_ineq : 1e-3;
  }
  return p;
}

extern "C" {

tt_status tt_sdp_create(const tt_sdp_problem* prob, const tt_sdp_options* opts, const tt_allocator* allocator,
                        void* stream, tt_sdp_ctx** out) {
  return make_ctx([&] { return problem_from(prob); }, opts, stream, out, allocator);
}

tt_status tt_sdp_create_batch(int32_t n, const tt_sdp_problem* probs, const tt_sdp_options* opts,
                              const tt_allocator* allocator, void* stream, tt_sdp_ctx** out) {
  if (n <= 0 || !probs || !out) return TT_E_INVALID_ARG;
  auto* b = new tt_sdp_ctx;
  b->stream = (cudaStream_t)stream;
  b->batch = true;
  for (int i = 0; i < n; ++i) {
    tt_sdp_ctx* c = nullptr;
    tt_status s = tt_sdp_create(&probs[i], opts, allocator, stream, &c);
    if (s != TT_OK) {
      for (tt_sdp_ctx* m : b->members) tt_sdp_destroy(m);
      delete b;
      return s;
    }
    b->members.push_back(c);
  }
  *out = b;
  return TT_OK;
}

int32_t tt_sdp_batch_size(const tt_sdp_ctx* ctx) {
  if (!ctx) return 0;
  return ctx->batch ? (int32_t)ctx->members.size() : 1;
}

tt_sdp_ctx* tt_sdp_batch_member(tt_sdp_ctx* ctx, int32_t i) {
  if (!ctx || !ctx->batch || i < 0 || i >= (int32_t)ctx->members.size()) return nullptr;
  return ctx->members[(size_t)i];
}

tt_status tt_sdp_create_maxcut(const tt_desc* weights, const tt_sdp_options* opts, void* stream, tt_sdp_ctx** out) {
  return make_ctx(
      [&] {
        TT_CHECK(weights && weights->m == 2 && weights->n == 2, TT_E_SHAPE, "weights must have 2 x 2 modes");
        return build_maxcut(desc_host(weights));
      },
      opts, stream, out);
}

tt_status tt_sdp_create_theta(const tt_desc* adjacency, const tt_sdp_options* opts, void* stream,
                              tt_sdp_ctx** out) {
  return make_ctx(
      [&] {
        TT_CHECK(adjacency && adjacency->m == 2 && adjacency->n == 2, TT_E_SHAPE, "adjacency must have 2 x 2 modes");
        return build_theta(desc_host(adjacency));
      },
      opts, stream, out);
}

tt_status tt_sdp_create_cc(const tt_desc* c_plus, const tt_desc* c_minus, const tt_desc* adjacency,
                           const tt_sdp_options* opts, void* stream, tt_sdp_ctx** out) {
  return make_ctx(
      [&] {
        for (const tt_desc* t : {c_plus, c_minus, adjacency})
          TT_CHECK(t && t->m == 2 && t->n == 2, TT_E_SHAPE, "inputs must have 2 x 2 modes");
        return build_cc(desc_host(c_plus), desc_host(c_minus), desc_host(adjacency));
      },
      opts, stream, out);
}

tt_status tt_sdp_newton_step(tt_sdp_ctx* ctx, tt_sdp_iter_info* info) {
  if (!ctx || !info || ctx->batch) return TT_E_INVALID_ARG;
  return ctx_guarded(ctx, [&] {
    IterLog l = ctx->solver->iterate();
    info->iter = l.iter;
    info->converged = l.converged;
    info->mu = l.mu;
    info->rel_p = l.rel_p;
    info->rel_d = l.rel_d;
    info->rel_gap = l.rel_gap;
    info->pobj = l.pobj;
    info->dobj = l.dobj;
    info->alpha_p = l.alpha_p;
    info->alpha_d = l.alpha_d;
    info->max_rank_X = l.max_rank_X;
    info->max_rank_Z = l.max_rank_Z;
    info->max_rank_W = l.max_rank_W;
    info->sweeps = l.sweeps;
    info->direction = l.direction;
    info->seconds = l.seconds;
    info->gmres_iters = l.gmres_iters;
    info->pred_used = l.pred_used;
    info->pred_fallbacks = l.pred_fallbacks;
    info->forcing = l.forcing;
    info->forcing_corrections = l.forcing_corrections;
    info->damped_retries = l.retries;
    info->xz_fallbacks = l.fallbacks;
    info->finishing = l.finishing;
    info->accepted = l.accepted;
    info->nu = l.nu;
    info->merit = l.merit;
  });
}

tt_status tt_sdp_redo_update(tt_sdp_ctx* ctx, double alpha_p, double alpha_d) {
  if (!ctx || ctx->batch) return TT_E_INVALID_ARG;
  return ctx_guarded(ctx, [&] {
    TT_CHECK(ctx->solver->redo_update(alpha_p, alpha_d), TT_E_INVALID_ARG, "no update to redo yet");
  });
}

static tt_status solve_loop(tt_sdp_ctx* ctx, tt_sdp_result* out) {
  tt_sdp_iter_info info;
  double secs = 0.0;
  const int max_iters = ctx->solver->options().max_iters;
  for (int it = 0; it <= max_iters; ++it) {
    tt_status s = tt_sdp_newton_step(ctx, &info);
    if (s != TT_OK) {
      out->status = s;
      return s;
    }
    secs += info.seconds;
    out->iters = info.iter;
    out->pobj = info.pobj;
    out->dobj = info.dobj;
    out->rel_gap = info.rel_gap;
    out->rel_p = info.rel_p;
    out->rel_d = info.rel_d;
    out->seconds = secs;
    if (info.converged) {
      out->status = TT_OK;
      return TT_OK;
    }
  }
  out->status = TT_E_NO_CONVERGENCE;
  return TT_E_NO_CONVERGENCE;
}

tt_status tt_sdp_solve(tt_sdp_ctx* ctx, tt_sdp_result* out) {
  if (!ctx || !out) return TT_E_INVALID_ARG;
  if (ctx->batch) {
    const int32_t n = (int32_t)ctx->members.size();
    std::memset(out, 0, sizeof(*out) * (size_t)n);
    return tt_sdp_solve_batch(n, ctx->members.data(), n < 16 ? n : 16, out);
  }
  std::memset(out, 0, sizeof(*out));
  ctx->solver->set_deadline(ctx->solver->options().time_limit);
  const tt_status s = solve_loop(ctx, out);
  ctx->solver->set_deadline(0.0);
  return s;
}

tt_status tt_sdp_get_iterate(tt_sdp_ctx* ctx, int32_t which, int32_t* ranks, double* cores, size_t* count) {
  if (!ctx || !ranks || !count || ctx->batch) return TT_E_INVALID_ARG;
  return ctx_guarded(ctx, [&] {
    TT_CHECK(which >= 0 && which <= 4, TT_E_INVALID_ARG, "which must be 0..4");
    TT_CHECK(which != 2 || ctx->solver->has_ineq(), TT_E_INVALID_ARG, "no inequality multiplier");
    TT_CHECK(which != 4 || ctx->solver->frame(), TT_E_INVALID_ARG, "no Newton solve has run yet");
    DTT fr;
    if (which == 4) fr = ctx->solver->frame()->component(0);
    const DTT& t = which == 0 ? ctx->solver->X() : which == 1 ? ctx->solver->Y()
                 : which == 2 ? ctx->solver->T() : which == 3 ? ctx->solver->Z() : fr;
    for (int k = 0; k <= t.d; ++k) ranks[k] = t.r[k];
    size_t need = t.count();
    if (cores) {
      TT_CHECK(*count >= need, TT_E_NOMEM, "capacity too small");
      tt_to_host(t, cores);
    }
    *count = need;
  });
}

int32_t tt_sdp_order(const tt_sdp_ctx* ctx) {
  if (!ctx) return 0;
  if (ctx->batch) return ctx->members.empty() ? 0 : ctx->members[0]->solver->order();
  return ctx->solver->order();
}

void tt_sdp_destroy(tt_sdp_ctx* ctx) {
  if (!ctx) return;
  for (tt_sdp_ctx* m : ctx->members) tt_sdp_destroy(m);
  try {
    StreamGuard g(ctx->stream);
    AllocGuard ag(ctx->allocator());
    ctx->solver.reset();
    sync_stream(ctx->stream);
  } catch (...) {
  }
  delete ctx;
}

}  // extern "C"

extern "C" size_t tt_profile_report(char* buf, size_t cap) {
  std::string s;
  for (auto& p : Profiler::table()) s += p.first + " " + std::to_string(p.second) + "\n";
  if (buf && cap) {
    size_t n = s.size() < cap - 1 ? s.size() : cap - 1;
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return s.size();
}

// ---------------------------------------------------------------------------
// learned rank predictor
// ---------------------------------------------------------------------------
#include "rankpred.cuh"

struct tt_rankpred {
  std::shared_ptr<RankPredictor> p;
};

extern "C" {

int32_t tt_rankpred_param_count(void) { return kPredParams; }

tt_status tt_rankpred_create(uint64_t seed, tt_rankpred** out) {
  return guarded(nullptr, [&] {
    TT_CHECK(out, TT_E_INVALID_ARG, "null output");
    auto* r = new tt_rankpred;
    try {
      r->p = std::make_shared<RankPredictor>(seed);
    } catch (...) {
      delete r;
      throw;
    }
    *out = r;
  });
}

void tt_rankpred_destroy(tt_rankpred* p) { delete p; }

tt_status tt_rankpred_get_params(const tt_rankpred* p, float* out) {
  return guarded(nullptr, [&] {
    TT_CHECK(p && out, TT_E_INVALID_ARG, "null argument");
    p->p->get_params(out);
  });
}

tt_status tt_rankpred_set_params(tt_rankpred* p, const float* in) {
  return guarded(nullptr, [&] {
    TT_CHECK(p && in, TT_E_INVALID_ARG, "null argument");
    p->p->set_params(in);
  });
}

tt_status tt_rankpred_grad(tt_rankpred* p, const float* X, const float* t, int32_t n, float* grad, float* loss) {
  return guarded(nullptr, [&] {
    TT_CHECK(p && X && t && grad && loss && n > 0, TT_E_INVALID_ARG, "bad arguments");
    *loss = p->p->grad(X, t, n, grad);
  });
}

tt_status tt_rankpred_train(tt_rankpred* p, const float* X, const float* t, int32_t n, int32_t epochs, int32_t batch,
                            float lr, uint64_t seed, float* loss) {
  return guarded(nullptr, [&] {
    TT_CHECK(p && X && t && loss && n > 0 && epochs > 0 && batch > 0 && lr > 0, TT_E_INVALID_ARG, "bad arguments");
    *loss = p->p->train(X, t, n, epochs, batch, lr, seed);
  });
}

tt_status tt_rankpred_predict(const tt_rankpred* p, const float* X, int32_t n, float* y) {
  return guarded(nullptr, [&] {
    TT_CHECK(p && X && y && n > 0, TT_E_INVALID_ARG, "bad arguments");
    std::vector<float> xs(X, X + (size_t)n * kPredIn);
    std::vector<float> r = p->p->predict(xs, n);
    std::copy(r.begin(), r.end(), y);
  });
}

tt_status tt_sdp_set_rank_predictor(tt_sdp_ctx* ctx, const tt_rankpred* p) {
  if (!ctx) return TT_E_INVALID_ARG;
  return guarded(ctx->stream, [&] {
    if (!p) {
      ctx->solver->set_predictor(nullptr);
      return;
    }
    std::vector<float> params(kPredParams);
    p->p->get_params(params.data());
    auto copy = std::make_shared<RankPredictor>(0);
    copy->set_params(params.data());
    ctx->solver->set_predictor(copy);
  });
}

tt_status tt_sdp_set_trace(tt_sdp_ctx* ctx, int32_t on) {
  if (!ctx) return TT_E_INVALID_ARG;
  ctx->solver->set_trace(on != 0);
  return TT_OK;
}

tt_status tt_sdp_get_trace(tt_sdp_ctx* ctx, float* X, float* t, size_t* n) {
  if (!ctx || !n) return TT_E_INVALID_ARG;
  const auto& tx = ctx->solver->trace_x();
  const auto& ty = ctx->solver->trace_y();
  if (X) {
    if (*n < ty.size() || !t) return TT_E_NOMEM;
    std::copy(tx.begin(), tx.end(), X);
    std::copy(ty.begin(), ty.end(), t);
  }
  *n = ty.size();
  return TT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// concurrent batch of independent solves
// ---------------------------------------------------------------------------
#include <atomic>
#include <chrono>
#include <thread>

extern "C" tt_status tt_sdp_solve_batch(int32_t n, tt_sdp_ctx* const* ctxs, int32_t workers, tt_sdp_result* out) {
  if (n < 0 || (n > 0 && (!ctxs || !out)) || workers <= 0) return TT_E_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return TT_E_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_E_CUDA;
  for (int i = 0; i < n; ++i) sync_stream(ctxs[i]->stream);  // creation work is complete
  std::atomic<int> next{0};
  std::vector<tt_status> st(n, TT_OK);
  std::vector<std::thread> pool;
  const int nw = workers < n ? workers : (n > 0 ? n : 1);
  // while the workers run, waits sleep and each solve stays on one thread
  struct Active {
    int k;
    explicit Active(int k_) : k(k_) { concurrent_solves().fetch_add(k); }
    ~Active() { concurrent_solves().fetch_sub(k); }
  } active(nw);
  for (int w = 0; w < nw; ++w) {
    pool.emplace_back([&]() {
      cudaSetDevice(dev);
      cudaStream_t s = nullptr;
      const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n) break;
        if (!have_stream) {
          st[i] = TT_E_CUDA;
          continue;
        }
        cudaStream_t own = ctxs[i]->stream;
        ctxs[i]->stream = s;
        const auto t0 = std::chrono::steady_clock::now();
        st[i] = tt_sdp_solve(ctxs[i], &out[i]);
        sync_stream(s);
        out[i].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        ctxs[i]->stream = own;
      }
      if (have_stream) {
        sync_stream(s);
        cudaStreamDestroy(s);
      }
    });
  }
  for (auto& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != TT_OK) return st[i];
  return TT_OK;
}
