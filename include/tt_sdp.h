/*
 * tt_sdp.h -- C ABI of the GB300 tensor-train SDP interior-point library.
 *
 * The library implements the inexact tensor-train primal-dual interior-point
 * method for semidefinite programs of Kelbel, Dolgov, Kalise and Russo
 * ("An Inexact Tensor-Train Primal-Dual Interior-Point Method for
 * Semidefinite Programs"): the SDP variables X, Y, [T], Z and the constraint
 * operators are tensor trains with 2 x 2 modes per core (operators on the
 * vec_TT space have 4 x 4 modes), the Newton direction of the tensorised KKT
 * system (Section 3.3, eq. tt-kkt-newton-system) is found by block-AMEn with
 * matrix-free local products, and iterates are kept at moderate rank by TT
 * rounding with a spectral shift (Section 3.4, Corollary psdness_rounding).
 *
 * Conventions shared by every call.
 *  - TT vector cores are row-major [r_k][m][r_{k+1}], TT matrix cores
 *    [r_k][m][n][r_{k+1}], r_0 = r_d = 1, concatenated core after core
 *    (Section 2.3, Definitions "Tensor-Train" and "TT Matrix").
 *  - Multi-indices are big-endian (digit 1 most significant) and vec_TT
 *    interleaves (row digit, column digit) with the row digit more
 *    significant (Section 3.1, Definition "TT Vectorisation" and its
 *    worked example); a 2 x 2 matrix mode (i, j) maps to vector mode 2 i + j.
 *  - All arithmetic on device pointers is ordered on the CUDA stream passed
 *    in (NULL: the legacy default stream). Calls return after their results
 *    are usable on that stream; calls that return host values synchronise it.
 *  - Errors are status codes; nothing else crosses the boundary. A call that
 *    fails leaves its outputs unspecified and the library usable.
 *  - No CPU fallback: without a CUDA device every call returns TT_E_CUDA.
 */
#ifndef TT_SDP_H
#define TT_SDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_E_INVALID_ARG = 1,    /* null pointer, negative size, unknown enum value       */
  TT_E_SHAPE = 2,          /* ranks / modes inconsistent between operands           */
  TT_E_NOMEM = 3,          /* device allocation failed or output capacity too small */
  TT_E_CUDA = 4,           /* CUDA runtime error (message via tt_last_error)        */
  TT_E_NOT_PD = 5,         /* an iterate lost positive definiteness (Section 3.4)   */
  TT_E_RANK_CAP = 6,       /* warning: rank cap bound with truncation error > tol   */
  TT_E_NO_CONVERGENCE = 7, /* iteration or sweep budget exhausted                   */
  TT_E_TIMEOUT = 8,        /* a bounded device wait gave up                         */
  TT_E_NUMERIC = 9,        /* NaN or Inf detected                                   */
  TT_E_INTERNAL = 10
} tt_status;

/* Arithmetic used by the contractions (environments, local products). In the
 * three reduced precisions every AMEn solve closes with one FP64 sweep
 * (FP64 environments, local operators and solves) that refines the direction,
 * and rounding, residuals, norms and step lengths stay FP64. */
typedef enum {
  TT_FP64 = 0,        /* everything in FP64                                          */
  TT_FP32 = 1,        /* FP32 SIMT contractions, FP32 accumulation                   */
  TT_MIXED_TF32 = 2,  /* TF32 tensor-core contractions, FP32 accumulation            */
  TT_MIXED_BF16 = 3   /* BF16 tensor-core contractions, FP32 accumulation            */
} tt_precision;

/* Dimensions of one three-operand contraction step (Section 3.3, the
 * matrix-free local products with cached environments):
 *   frame core   U [rw][m][rw2]
 *   operator core Op [R][m][n][R2]   (TT matrix on the vec_TT space)
 *   vector core  V [rv][n][rv2]
 * A left environment Phi has shape [rw][R][rv], a right one Psi [rw2][R2][rv2]. */
typedef struct {
  int32_t rw, rw2;
  int32_t R, R2;
  int32_t rv, rv2;
  int32_t m, n;
} tt_contract_dims;

/* ---------------------------------------------------------------------------
 * Contraction kernels (rows a6, a7 of the hot path). Device pointers, FP64
 * storage; `precision` selects the arithmetic. Outputs are caller-allocated.
 * ------------------------------------------------------------------------- */

/* Left environment update (Section 3.3, local products with cached
 * environments): out[b'][q][b] = sum U[a'][i][b'] Op[p][i][j][q] V[a][j][b] Phi[a'][p][a].
 * out holds rw2 * R2 * rv2 doubles. */
tt_status tt_env_left_step(const tt_contract_dims* dims, const double* phi, const double* u,
                           const double* op, const double* v, double* out, int32_t precision,
                           void* stream);

/* Right environment update: out[a'][p][a] = sum U[a'][i][b'] Op[p][i][j][q] V[a][j][b] Psi[b'][q][b].
 * out holds rw * R * rv doubles. */
tt_status tt_env_right_step(const tt_contract_dims* dims, const double* psi, const double* u,
                            const double* op, const double* v, double* out, int32_t precision,
                            void* stream);

/* Local matrix-free product (Section 3.3, "inserting the local GMRES vector
 * into the active core"): y[a'][i][b'] = sum Phi[a'][p][a] Op[p][i][j][q] Psi[b'][q][b] x[a][j][b].
 * Here rv = rw-side size of x's left rank and rv2 its right rank;
 * x holds rv * n * rv2 doubles, y holds rw * m * rw2. */
tt_status tt_local_apply(const tt_contract_dims* dims, const double* phi, const double* op,
                         const double* psi, const double* x, double* y, int32_t precision,
                         void* stream);

/* Allocation-free variant of tt_env_left_step (FP64 only). The paper has no
 * counterpart: it exists for callers that cannot allocate device memory while
 * they run, such as a host framework whose own allocator owns the device heap
 * or a latency-critical loop that must not pay for allocation. Instead of
 * stream-ordered scratch, the two intermediate tensors live in one fixed
 * file-scope device array of 4,194,304 doubles (32 MiB) that every GPU loading
 * the library holds until the process exits. Shapes whose intermediates
 * (rw*R*n*rv2 + rw*m*R2*rv2 doubles) exceed it are rejected with TT_E_NOMEM
 * before anything runs. Every call looks up the array's device address with
 * the calling thread's current device (so a reset device is handled); make
 * the first call on a device before any stream capture, since it loads the
 * module there. All calls share the array and it keeps the last call's contents
 * (every element a call reads it has written itself first, so nothing needs
 * clearing); calls that overlap on the GPU, on different streams or devices
 * sharing a context, race on it. Arguments as for tt_env_left_step. */
tt_status tt_env_left_step_noalloc(const tt_contract_dims* dims, const double* phi, const double* u,
                                   const double* op, const double* v, double* out, void* stream);

/* Dense projected operator W^T Op W at one core: out[(a',i,b')][(a,j,b)],
 * (rw*m*rw2) x (rv*n*rv2) row-major doubles. */
tt_status tt_local_matrix(const tt_contract_dims* dims, const double* phi, const double* op,
                          const double* psi, double* out, int32_t precision, void* stream);

/* ---------------------------------------------------------------------------
 * TT-level operations on device cores (rows a3, a8, a9). A tt_desc names
 * device cores here; ranks are host arrays.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t d;              /* number of cores                                    */
  const int32_t* ranks;   /* host array, d + 1 entries, ranks[0] = ranks[d] = 1 */
  int32_t m, n;           /* modes of every core; n = 1 for TT vectors          */
  const double* cores;    /* concatenated cores (device or host, per call)      */
} tt_desc;

/* Number of doubles in the cores of a TT with the given ranks and modes. */
size_t tt_core_count(int32_t d, const int32_t* ranks, int32_t m, int32_t n);

/* Element-wise (Hadamard) product of two TTs with equal modes, the product
 * of the Remark after Definition "TT Diagonalisation" (Section 3.3):
 * core [(a,x)][mode][(b,y)] = A[a][mode][b] B[x][mode][y]; ranks multiply.
 * out holds tt_core_count(d, ra*rb, m, n) doubles. */
tt_status tt_hadamard(const tt_desc* a, const tt_desc* b, double* out, void* stream);

/* TT matrix times TT vector, core [(p,a)][i][(q,b)] = sum_j Op[p][i][j][q] V[a][j][b]
 * (diag_TT operators reduce this to the masked products of Section 3.3). */
tt_status tt_matvec(const tt_desc* op, const tt_desc* v, double* out, void* stream);

/* Inner product <a, b> over all entries (a3): one environment sweep. The
 * result is written to *out (host) and the stream is synchronised. */
tt_status tt_inner(const tt_desc* a, const tt_desc* b, double* out, void* stream);

/* Row a12: the step-length eigenproblem (Section 2.2, Theorem "Optimal Step
 * Size"; Section 3.4): lambda = min over TT vectors e of <e, dM e> / <e, M e>
 * for symmetric TT matrices M (positive definite) and dM with equal square
 * modes, device cores. Runs `sweeps` two-site DMRG sweeps (two_site = 1: at
 * each bond the supercore's projected generalised eigenproblem, then a
 * truncated SVD split with relative tolerance 1e-8 and at most `rank`, plus
 * random kick columns up to `rank`) or one-site ALS sweeps (two_site = 0)
 * from a random start of TT rank `rank` drawn from the SplitMix64 stream
 * `seed`. The largest alpha with M + alpha dM positive semidefinite is
 * -1/lambda when lambda < 0 and unbounded otherwise. FP64; synchronises. */
tt_status tt_min_gen_eig(const tt_desc* M, const tt_desc* dM, int32_t rank, int32_t sweeps, int32_t two_site,
                         uint64_t seed, double* lambda, void* stream);

/* TT rounding (row a9; Oseledets' round_TT as used in Section 2.3):
 * right-to-left Householder QR, then left-to-right truncated SVD. Bond k
 * keeps the smallest rank whose discarded energy is <= (delta/sqrt(d-1))^2,
 * then at most rank_cap (<= 0: no cap). ranks_out (host, d+1), cores_out
 * (device, capacity doubles >= input count). *zeta_out (host) receives
 * ||T - round(T)||_F = sqrt(sum of all discarded sigma^2). The input is a
 * TT vector view (set m to the full mode size, n = 1). */
tt_status tt_round(const tt_desc* in, double delta, int32_t rank_cap, int32_t* ranks_out,
                   double* cores_out, size_t capacity, double* zeta_out, int32_t precision,
                   void* stream);

/* Row a1 helper: TT decomposition (TT-SVD of Oseledets, as Section 4 notes
 * one may do for operators given as matrices) of a dense n^d x n^d matrix,
 * row-major FP64 on the DEVICE, in its vec_TT order: a TT matrix with n x n
 * modes. Bond k keeps the smallest rank whose discarded energy is at most
 * (eps_rel ||M||_F)^2 / (d-1), then at most rank_cap (<= 0: none).
 * ranks_out (host, d+1), cores_out (host, capacity doubles; NULL = size query:
 * *count receives the number of doubles). FP64 throughout. */
tt_status tt_from_dense(const double* dense, int32_t d, int32_t n, double eps_rel, int32_t rank_cap,
                        int32_t* ranks_out, double* cores_out, size_t* count, void* stream);

/* ---------------------------------------------------------------------------
 * The solver (rows a1-a5, a10-a12): a context holds one SDP in TT form and
 * its iterates on the device.
 * ------------------------------------------------------------------------- */

/* Tensorised SDP of Section 3.1:
 *   max <C, X>  s.t.  A_eq vec_TT(X) = B_eq,  A_ineq vec_TT(X) >= / <= B_ineq,  X psd,
 * with the idle-multiplier masks K_y, K_t of Section 3.3. All descriptors
 * name HOST cores; they are copied at create. Operators have m = n = 4,
 * right-hand sides m = 4, n = 1, C and ones_t m = n = 2. Absent parts have d = 0. */
typedef struct {
  tt_desc C;
  tt_desc A_eq;
  tt_desc B_eq;
  tt_desc K_y;
  tt_desc A_ineq;
  tt_desc B_ineq;
  tt_desc K_t;
  tt_desc ones_t;      /* 1_T: ones on the non-idle inequality positions            */
  int32_t ineq_sign;   /* +1: s = A_ineq x - B_ineq >= 0 (Section 4.3); -1: <=       */
  int64_t q;           /* number of inequality entries in mirrored storage          */
  double lam0;         /* initial scale lambda* (Section 5.1)                        */
  double lam0_ineq;    /* lambda*_ineq                                               */
} tt_sdp_problem;

typedef struct {
  double eps_gap;      /* target; eps_p = eps_d = 2 eps_gap, eps_c = eps_gap / sqrt(d) */
  int32_t rank_cap;    /* cap on iterate and direction TT ranks                        */
  int32_t xz_warmup;   /* iterations with the XZ direction before AHO (3)              */
  double eta0;         /* initial forcing term (1e-3)                                  */
  double eta_floor;    /* delta of the forcing schedule (1e-4)                         */
  double eta_C;        /* C of eta <- max(min(eta, C mu), delta) (2)                   */
  double damping;      /* step damping factor (0.95)                                   */
  int32_t precision;   /* tt_precision of the contractions                             */
  int32_t max_iters;
  int32_t max_sweeps;  /* AMEn sweeps per Newton solve (reduced precisions: plus the
                          closing FP64 sweep)                                        */
  int32_t kick;        /* AMEn random enrichment columns                               */
  int32_t eig_rank;    /* TT rank of the step-length eigenvector                       */
  int32_t eig_sweeps;
  uint64_t seed;       /* SplitMix64 counter stream seed                               */
  int32_t local_dense_max; /* reduced local systems up to this size (8192) are formed
                              and solved by block elimination (or LU), larger ones
                              matrix-free by restarted GMRES                       */
  int32_t gmres_restart;
  int32_t gmres_max_iters; /* operator products per local solve                       */
  int32_t eig_two_site;    /* step lengths (Section 3.4): 1 two-site DMRG sweeps with
                              SVD rank adaptation and random kicks, 0 one-site ALS    */
  double time_limit;       /* tt_sdp_solve / tt_sdp_solve_batch: wall-clock seconds per
                              solve (0: none). When it passes, the iteration in
                              progress is abandoned at its next core step, the
                              context keeps the last completed iterate and the solve
                              returns TT_E_NO_CONVERGENCE                          */
  int32_t combined_multipliers; /* 1 (default): with inequalities whose non-idle mask
                              I - K_T is disjoint from that of Y, I - K_Y, and all of
                              A_eq, A_ineq, K_Y, K_T diagonal, dY and dT are one block
                              dLambda of the AMEn solve (Section 3.5, "Combined
                              Multiplier Storage"); 0: separate blocks            */
  double finish_tol;       /* finishing phase (Section 3.5, "Relaxing the Positive
                              Definiteness Barrier"), 0 (default): off. When > 0, once
                              the relative criteria hold the solve goes on until
                              ||R_p||_F, ||R_d||_F and |<X,Z> + <vec T, s>| are all
                              below finish_tol, with step lengths for the relaxed
                              cone M + nu I >= 0 and updates kept only when they
                              lower the merit ||R_p|| + ||R_d|| + |gap| while the
                              relative criteria still hold; a rejected update keeps
                              the iterate and multiplies nu by 10, up to nu_max,
                              after which the phase ends                          */
  double nu0, nu_max;      /* first and largest relaxation nu (1e-6, 1e-3)            */
  int32_t refine_sweeps;   /* reduced precisions: FP64 sweeps that close every AMEn
                              solve (1 by default; 1..8)                           */
  int32_t fp32_factors;    /* TT_FP64: 1 (default) lets the dense local solves factor
                              in FP32 and refine in FP64 (mixed-precision iterative
                              refinement), keeping the result only when its FP64
                              relative residual reaches 1e-14; after the first miss
                              in an AMEn solve its remaining solves factor in FP64.
                              0: FP64 factors only                                  */
} tt_sdp_options;

typedef struct tt_sdp_ctx tt_sdp_ctx;

typedef struct {
  int32_t iter;
  int32_t converged;   /* 1 when the stopping rules of Section 3.5 hold              */
  double mu, rel_p, rel_d, rel_gap, pobj, dobj, alpha_p, alpha_d;
  int32_t max_rank_X, max_rank_Z, max_rank_W, sweeps;
  int32_t direction;   /* 0 XZ, 1 AHO                                                 */
  double seconds;      /* device time of the iteration (CUDA events)                 */
  int64_t gmres_iters; /* local GMRES operator products so far                       */
  int64_t pred_used;      /* bonds rounded by the predicted-rank range finder so far   */
  int64_t pred_fallbacks; /* predicted bonds that fell back to the adaptive SVD        */
  /* Forcing check (Section 3.3, eq. forcing-condition, applied to the projected
   * systems the AMEn sweep solves): the largest FP64 relative residual
   * ||b - K x|| / ||b|| of a local solve in this iteration, K the projected
   * operator with FP64 products, and the correction solves run so far because a
   * residual exceeded the local tolerance (GMRES: eta/10, LU: 1e-10).        */
  double forcing;
  int64_t forcing_corrections;
  /* Damp-and-retry (Section 3.5): updates redone with halved step lengths so
   * far, because the next step-length solve found the iterate outside the
   * cone (at most 4 per iteration; then TT_E_NOT_PD is returned).            */
  int64_t damped_retries;
  /* AHO -> XZ fallback (Section 3.5): AHO iterations redone with the XZ
   * direction so far, because an AMEn solve missed its tolerance within the
   * sweep budget or the admissible step was below 1e-3.                      */
  int64_t xz_fallbacks;
  /* Finishing phase (Section 3.5): 1 when this iteration belonged to it, then
   * whether its update was kept, the relaxation nu of its step lengths and the
   * merit of the iterate it started from.                                    */
  int32_t finishing, accepted;
  double nu, merit;
} tt_sdp_iter_info;

typedef struct {
  tt_status status;
  int32_t iters;
  double pobj, dobj, rel_gap, rel_p, rel_d, seconds;
} tt_sdp_result;

/* Defaults of Section 5.1 (eps_gap 1e-4, 3 XZ warm-up iterations, eta0 1e-3,
 * eta floor 1e-4, C = 2) and of this library (damping 0.95, kick 4, ...). */
void tt_sdp_default_options(tt_sdp_options* opts);

/* Device memory hook. Every device buffer a context allocates (iterates,
 * environments, scratch of the sweeps) comes from `alloc` and goes back
 * through `free`, with the CUDA stream the library works on at that moment
 * (all earlier work that touches the block is ordered before that point on
 * it) and the caller's `user` pointer; a framework that owns the device heap
 * (a caching allocator) passes its own pair here. `alloc` returns NULL when
 * it cannot satisfy the request (the call then fails with TT_E_NOMEM); sizes
 * are bytes and blocks must be 256-byte aligned. The struct is copied at
 * create; the functions must stay callable until the context is destroyed
 * and may be called from library worker threads. NULL selects the device's
 * default stream-ordered memory pool (cudaMallocAsync). The
 * step-length and rounding calls outside a context always use the pool. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, void* stream, void* user);
  void* user;
} tt_allocator;

/* Copies the problem to the device and sets the initial point of Section 5.1:
 * X = Z = lam0 I, Y = 0 (with inequalities X = lam0 I + (alpha_p/10) 1_T,
 * T = lam0_ineq 1_T). `allocator` may be NULL (default pool). */
tt_status tt_sdp_create(const tt_sdp_problem* prob, const tt_sdp_options* opts, const tt_allocator* allocator,
                        void* stream, tt_sdp_ctx** out);

/* A batch of n independent SDPs (the many-instance workload; each instance as
 * for tt_sdp_create, same options). tt_sdp_solve on the returned context
 * solves every instance concurrently (one host worker thread and one CUDA
 * stream per concurrently running instance, at most 16) and writes n results;
 * tt_sdp_newton_step and tt_sdp_get_iterate reject a batch context (read an
 * instance through tt_sdp_batch_member). tt_sdp_destroy frees every
 * instance. */
tt_status tt_sdp_create_batch(int32_t n, const tt_sdp_problem* probs, const tt_sdp_options* opts,
                              const tt_allocator* allocator, void* stream, tt_sdp_ctx** out);
/* Number of instances of a batch context (1 for a single context). */
int32_t tt_sdp_batch_size(const tt_sdp_ctx* ctx);
/* Instance i of a batch context, owned by the batch (NULL when out of range). */
tt_sdp_ctx* tt_sdp_batch_member(tt_sdp_ctx* ctx, int32_t i);

/* Row a5, the dense local solve of one AMEn core step (Section 3.3: the
 * reduced projected system eq. reduced_kkt_system when it is small enough to
 * be formed): K x = b with K n x n row-major FP64 on the DEVICE (not
 * modified) and b (n doubles, device) overwritten by x. TT_FP64: LU with
 * partial pivoting in FP64. Reduced precisions: one FP32 factorisation
 * refined in FP64 until ||b - K x|| <= 1e-10 ||b|| (at most five
 * corrections). *rel_residual (host) receives the FP64 relative residual of
 * the returned x. Synchronises the stream. */
tt_status tt_lu_solve(int32_t n, const double* K, double* b, int32_t precision, double* rel_residual,
                      void* stream);

/* Row a5 as the AMEn sweeps run it: the reduced projected system of
 * Section 3.3 (eq. reduced_kkt_system) solved by the block elimination that
 * follows it there. K is n x n row-major FP64 on the DEVICE (not modified),
 * unknowns [dX; multipliers] with dX the first n_lz, equations [multiplier
 * rows; complementarity rows] with the complementarity rows the last n_lz,
 * so that the bottom-left n_lz x n_lz block is the projected L_Z (symmetric
 * positive definite while Z is; only its symmetric part is factored). With
 * L_Z = U^T U (Cholesky), the multipliers solve the Schur complement system
 * (F - E L_Z^-1 G) dl = b_m - E L_Z^-1 b_c by LU with partial pivoting
 * (F, E, G the remaining blocks), and dX = L_Z^-1 (b_c - G dl). Every
 * solve is refined in FP64 against K; refinement stops at the target, after
 * the step budget, or once a step fails to halve the residual. TT_FP64: FP32
 * factors first (mixed-precision iterative refinement, at most eight steps
 * towards 1e-15), kept when the relative residual reaches 1e-14; otherwise
 * FP64 factors (at most three steps towards 1e-15). Reduced precisions: FP32
 * factors and at most five steps towards 1e-10. When L_Z is not numerically
 * positive definite, or the residual stays above 1e-10, the whole system is
 * solved by LU with partial pivoting: FP32 factors refined in FP64 (kept in
 * TT_FP64 only at a residual of 1e-14), else, in TT_FP64, FP64 factors. b (n doubles, device) is overwritten by x; *rel_residual
 * (host) receives the FP64 relative residual. 0 < n_lz < n is required.
 * Synchronises the stream. */
tt_status tt_kkt_solve(int32_t n, int32_t n_lz, const double* K, double* b, int32_t precision,
                       double* rel_residual, void* stream);
/* Block-elimination solves of tt_kkt_solve and of the AMEn sweeps completed,
 * those of them that kept FP32 factors, those that fell back to the LU of
 * the whole system, and the Cholesky factorisations (FP32 or FP64) that met
 * a pivot of L_Z that was not positive, since the last reset (reset != 0
 * clears all four after reading; any pointer may be NULL). */
void tt_kkt_stats(uint64_t* block_solves, uint64_t* fp32_factor_solves, uint64_t* lu_fallbacks,
                  uint64_t* lz_not_pd, int32_t reset);

/* Row a9 on host data: TT rounding (Section 2.3, round_TT) followed by the
 * spectral shift of Section 3.4, Corollary psdness_rounding. `in` names HOST
 * cores of a TT matrix (m = n) or vector (n = 1). The input is rounded as a
 * vector (m * n per core): bond k keeps the smallest rank whose discarded
 * energy is <= (delta / sqrt(d-1))^2, then at most rank_cap (<= 0: no cap);
 * zeta = sqrt(sum of all discarded sigma^2) = ||in - round(in)||_F.
 *   psd_shift 0: out = round(in) at delta = tol.
 *   psd_shift 1: out = round(in) + zeta I (X and Z of the SDP), rounded at
 *                delta = tol / (1 + ||I||_F) so that ||in - out||_F <= tol.
 *   psd_shift 2: out = round(in) + zeta (J - I), the inequality mask 1_T of
 *                the complete-graph constraints of Section 4.3 (the
 *                multiplier T), rounded at tol / (1 + ||J - I||_F).
 * Shifts need a square TT matrix (m = n). `out` is caller-owned: out->ranks
 * points to a writable array of d + 1 ints that receives the ranks and
 * out->cores to a writable host buffer (the const qualifiers of tt_desc
 * describe inputs); out->d, m, n are set from `in`. With out->cores == NULL
 * only the ranks are written (size query: the buffer needs
 * tt_core_count(d, ranks, m, n) doubles); the rounding is deterministic, so a
 * second call with the buffer writes cores of exactly those ranks.
 * *zeta_out receives zeta. FP64 on the device; synchronises the stream. */
tt_status tt_sdp_round(const tt_desc* in, double tol, int32_t rank_cap, int32_t psd_shift, tt_desc* out,
                       double* zeta_out, void* stream);

/* Row a1: assemble the Section 4 formulations on the device from the graph
 * adjacency given as a host TT matrix (2 x 2 modes, zero diagonal) and create
 * the context. Max-Cut (Section 4.1) uses `weights` (the weighted adjacency;
 * pass the adjacency for unit weights); theta (Section 4.2) the adjacency;
 * correlation clustering (Section 4.3) C+ and C- and the adjacency. */
tt_status tt_sdp_create_maxcut(const tt_desc* weights, const tt_sdp_options* opts, void* stream,
                               tt_sdp_ctx** out);
tt_status tt_sdp_create_theta(const tt_desc* adjacency, const tt_sdp_options* opts, void* stream,
                              tt_sdp_ctx** out);
tt_status tt_sdp_create_cc(const tt_desc* c_plus, const tt_desc* c_minus, const tt_desc* adjacency,
                           const tt_sdp_options* opts, void* stream, tt_sdp_ctx** out);

/* One iteration of Algorithm 1 (residuals, mu, Mehrotra predictor and
 * corrector Newton solves, step lengths, update and rounding). Returns
 * TT_OK with info->converged = 1 when the stopping rules already hold. */
tt_status tt_sdp_newton_step(tt_sdp_ctx* ctx, tt_sdp_iter_info* info);

/* Undoes the last update of Algorithm 1 and redoes it from the stored iterate
 * and direction with step lengths alpha_p (X) and alpha_d (Y, T, Z); a
 * negative value keeps that step length. The result is rounded like every
 * update (Corollary psdness_rounding). Meant for exercising the safeguards of
 * Section 3.5: an update planted past the boundary of the cone is found by
 * the next step-length solve and repaired by damp-and-retry. Returns
 * TT_E_INVALID_ARG before the first update. */
tt_status tt_sdp_redo_update(tt_sdp_ctx* ctx, double alpha_p, double alpha_d);

/* Iterates until the stopping rules hold or max_iters. For a batch context
 * (tt_sdp_create_batch) `out` is an array of tt_sdp_batch_size(ctx) results
 * and the status is that of tt_sdp_solve_batch. */
tt_status tt_sdp_solve(tt_sdp_ctx* ctx, tt_sdp_result* out);

/* Solves n independent contexts concurrently: `workers` host threads, each
 * with its own non-blocking CUDA stream on the current device, take contexts
 * from a shared queue and run tt_sdp_solve on them (a context's own stream is
 * replaced by the worker's for the duration). out[i] receives context i's
 * result; out[i].seconds is its wall time from start to finish on its stream.
 * The contexts must be distinct. A rank predictor may be attached to several
 * of them (prediction only reads its parameters) but must not be trained
 * while the batch runs. The tensor-core fault flag is one per device, so a
 * fault in one context's kernel is reported by every context that reads it
 * during the batch. Returns TT_OK when every context converged, else the
 * status of the first context (by index) that did not. */
tt_status tt_sdp_solve_batch(int32_t n, tt_sdp_ctx* const* ctxs, int32_t workers, tt_sdp_result* out);

/* Copies iterate `which` (0 X, 1 Y, 2 T, 3 Z; TT matrices with 2 x 2 modes)
 * to the host. which = 4 gives the block-AMEn frame kept as the warm start of
 * the next Newton solve (Section 3.5), a TT vector with mode 4 whose core 0
 * carries block 0 (dX); its ranks are the frame's bond ranks. With
 * cores == NULL only ranks (d+1 ints) and *count are set. */
tt_status tt_sdp_get_iterate(tt_sdp_ctx* ctx, int32_t which, int32_t* ranks, double* cores,
                             size_t* count);

/* Number of cores d of the context's problem. */
int32_t tt_sdp_order(const tt_sdp_ctx* ctx);

void tt_sdp_destroy(tt_sdp_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Learned per-bond rank predictor (row a9, learned variant). The paper picks
 * every rank by the adaptive SVD; this library adds a small network that
 * predicts the rank the adaptive SVD would choose, so that a rounding can use
 * a fixed-rank randomised range finder (Halko, Martinsson and Tropp) whose
 * sketch product runs on the TF32 tensor cores. The exact FP64 truncation
 * error of the sketched bond is checked against the bond tolerance; when it
 * exceeds it (or the rank cap would bind) the bond falls back to the
 * adaptive SVD, which has the final word. Network: 10 features -> 64 -> 64 -> 64
 * -> 1, tanh hidden layers, sigmoid output = rank / cap, trained on the GPU
 * (mean squared error, Adam) by the library's own kernels. Features of a
 * bond: one-hot variable (X, Y, T, Z), bond position k/(d-2), log10(mu)/10,
 * input rank / cap, previous rank of that bond / cap, iteration / max_iters,
 * and the singular-value decay seen at that bond in the variable's previous
 * rounding (log10(sigma_kept_last / sigma_1) / 16, 0 before the first), which
 * costs no extra decomposition.
 * All arrays below are HOST arrays.
 * ------------------------------------------------------------------------- */
typedef struct tt_rankpred tt_rankpred;

/* Number of float parameters (9153). */
int32_t tt_rankpred_param_count(void);
/* Xavier-initialised network from the SplitMix64 stream `seed`. */
tt_status tt_rankpred_create(uint64_t seed, tt_rankpred** out);
void tt_rankpred_destroy(tt_rankpred* p);
tt_status tt_rankpred_get_params(const tt_rankpred* p, float* out);
tt_status tt_rankpred_set_params(tt_rankpred* p, const float* in);
/* Mean squared error on (X: n x 10, t: n) and its gradient (param_count floats). */
tt_status tt_rankpred_grad(tt_rankpred* p, const float* X, const float* t, int32_t n, float* grad, float* loss);
/* Adam (beta 0.9 / 0.999) on shuffled mini-batches; *loss = final full-data loss. */
tt_status tt_rankpred_train(tt_rankpred* p, const float* X, const float* t, int32_t n, int32_t epochs,
                            int32_t batch, float lr, uint64_t seed, float* loss);
/* y (n values in (0, 1)) for the feature rows X (n x 10). */
tt_status tt_rankpred_predict(const tt_rankpred* p, const float* X, int32_t n, float* y);
/* Attach a copy of the predictor to a context (NULL detaches). */
tt_status tt_sdp_set_rank_predictor(tt_sdp_ctx* ctx, const tt_rankpred* p);
/* Record (features, adaptive-SVD rank / cap) of every bond rounded by the adaptive SVD. */
tt_status tt_sdp_set_trace(tt_sdp_ctx* ctx, int32_t on);
/* Copy the recorded trace: X (n x 10 floats) and t (n floats); with X == NULL only *n is set. */
tt_status tt_sdp_get_trace(tt_sdp_ctx* ctx, float* X, float* t, size_t* n);

/* ---------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------- */
const char* tt_sdp_status_string(tt_status s);
/* Message of the last failure on the calling thread (empty if none). */
const char* tt_last_error(void);
/* Kernels launched by the library since load (monotone counter). */
uint64_t tt_launch_count(void);
/* Device time spent in the contraction kernels since the last reset, and
 * their algorithmic flop count (for the contraction TFLOP/s metric). */
void tt_contraction_stats(double* flops, double* seconds);
void tt_contraction_stats_reset(void);
/* Tensor-core GEMM launches of the TF32 / BF16 contractions since the last
 * reset: algorithmic flops (2 M N K with the unpadded K), device seconds from
 * CUDA events around each launch, and the launch count. */
void tt_tc_stats(double* flops, double* seconds, uint64_t* launches);
/* Dense local solves of the AMEn sweeps since the last reset: algorithmic
 * flops, device seconds from CUDA events and the number of local systems.
 * Block elimination (N unknowns, n of them dX, m = N - n): n^3 / 3 + 2 n^2 m
 * + 2 n m^2 + 2 m^3 / 3 per factorisation plus 4 n^2 + 2 m^2 + 4 n m per
 * solve; LU of the whole system (the fallback, and tt_lu_solve): 2 N^3 / 3
 * per factorisation plus 2 N^2 per triangular-solve pair (the time of a
 * fallback includes the block attempt). Reset with
 * tt_contraction_stats_reset. */
void tt_lu_stats(double* flops, double* seconds, uint64_t* calls);
/* FP64 launches of the strided SIMT GEMM (gemm_nd_kernel: every FP64
 * contraction stage, local operator, block move and trailing update) since
 * the last reset, sampled: every eighth launch of each host thread is timed
 * with CUDA events (its split-K reduction included); flops (2 M N K),
 * seconds and the count are those of the timed launches (about an eighth of
 * all). Reset with tt_contraction_stats_reset. */
void tt_gemm64_stats(double* flops, double* seconds, uint64_t* launches);
/* Per-phase host wall time accumulated while the environment variable
 * TTSDP_PROFILE=1 is set (each phase then synchronises the stream): one
 * "name seconds" line per phase, written NUL-terminated into buf (at most cap
 * bytes); returns the full text length. */
size_t tt_profile_report(char* buf, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* TT_SDP_H */
