// The TT interior-point solver: problem assembly (Section 4), block-AMEn
// Newton solves (Section 3.3), step lengths (Section 3.4) and Algorithm 1.
#pragma once

#include <chrono>

#include <memory>
#include <string>
#include <vector>

#include "tt.cuh"

namespace ttsdp {

struct Problem {
  int d = 0;
  DTT C, A_eq, B_eq, K_y;                 // C: 2x2 modes; operators 4x4; B_eq mode 4
  bool ineq = false;
  DTT A_ineq, B_ineq, K_t, ones_t;
  double sgn = 1.0;
  long long q = 0;
  double lam0 = 1.0, lam0_ineq = 1e-3;
};

Problem build_maxcut(const DTT& weights);
Problem build_theta(const DTT& adjacency);
Problem build_cc(const DTT& c_plus, const DTT& c_minus, const DTT& adjacency);

// Block TT (Definition "Block Tensor-Train") with the block index at core 0.
struct BlockTT {
  DTT frame;                              // vector TT (mode 4); core pos = block 0
  int nblk = 0;
  int pos = 0;                            // core that carries the block index
  std::shared_ptr<DBuf<double>> block;    // nblk x r_pos x 4 x r_pos+1
  DTT component(int b) const;
};

struct Options {
  double eps_gap = 1e-4;
  int rank_cap = 16;
  int xz_warmup = 3;
  double eta0 = 1e-3, eta_floor = 1e-4, eta_C = 2.0, damping = 0.95;
  int prec = 0;
  int max_iters = 60, max_sweeps = 4, kick = 4, eig_rank = 4, eig_sweeps = 4;
  int eig_two_site = 1;  // step lengths by two-site DMRG sweeps; 0: one-site ALS
  double time_limit = 0.0;  // seconds per solve (0: none)
  uint64_t seed = 1234;
  int local_dense_max = 8192, gmres_restart = 40, gmres_max_iters = 400;
  int combined_multipliers = 1;  // one block dLambda for dY, dT when their masks are disjoint
  // finishing phase (Section 3.5): absolute tolerance (0: off) and the barrier relaxation range
  double finish_tol = 0.0, nu0 = 1e-6, nu_max = 1e-3;
  int refine_sweeps = 1;  // closing FP64 sweeps of a reduced-precision AMEn solve
  int fp32_factors = 1;   // FP64: dense local solves may use FP32 factors refined in FP64
};

struct IterLog {
  int iter = 0, converged = 0, direction = 0, sweeps = 0;
  double mu = 0, rel_p = 0, rel_d = 0, rel_gap = 0, pobj = 0, dobj = 0, alpha_p = 0, alpha_d = 0;
  int max_rank_X = 0, max_rank_Z = 0, max_rank_W = 0;
  double seconds = 0;
  long long gmres_iters = 0;
  long long pred_used = 0, pred_fallbacks = 0;
  double forcing = 0;               // largest FP64 relative residual of a local solve this iteration
  long long forcing_corrections = 0;
  long long retries = 0;            // damped retries of updates that left the cone, so far
  long long fallbacks = 0;          // AHO iterations redone with the XZ direction, so far
  int finishing = 0, accepted = 1;  // finishing-phase iteration; its update was kept
  double nu = 0.0, merit = 0.0;     // its barrier relaxation; merit of the iterate it started from
};

class RankPredictor;

class Solver {
 public:
  Solver(Problem p, const Options& o);
  ~Solver();
  Solver(const Solver&) = delete;
  Solver& operator=(const Solver&) = delete;
  IterLog iterate();        // one iteration of Algorithm 1
  // redo the last update from its stored iterate and direction with other
  // step lengths (negative: keep that one); false when no update exists yet
  bool redo_update(double alpha_p, double alpha_d);
  // wall-clock deadline checked between the core steps of the AMEn sweeps;
  // past it the iteration in progress throws TT_E_NO_CONVERGENCE
  void set_deadline(double seconds_from_now);
  const DTT& X() const { return X_; }
  const DTT& Y() const { return Y_; }
  const DTT& T() const { return T_; }
  const DTT& Z() const { return Z_; }
  // frame of the last Newton solve's warm start (block index at core 0); null before the first
  const BlockTT* frame() const { return w_.get(); }
  bool has_ineq() const { return p_.ineq; }
  int order() const { return p_.d; }
  int iter() const { return it_; }
  const Options& options() const { return o_; }
  // learned rank predictor for the roundings (null: adaptive SVD only)
  void set_predictor(std::shared_ptr<RankPredictor> p) { pred_ = std::move(p); }
  // record (features, adaptive-SVD rank / cap) of every rounded bond
  void set_trace(bool on) { trace_ = on; }
  const std::vector<float>& trace_x() const { return trace_x_; }
  const std::vector<float>& trace_y() const { return trace_y_; }

 private:
  struct Measures {
    double rel_p, rel_d, rel_gap, pobj, dobj, mu;
    double abs_p, abs_d, comp;  // ||R_p||_F, ||R_d||_F, <X, Z> + <vec T, s>
  };
  Measures measures();
  DTT slack(const DTT& X);
  void direction(int dir, double sigma_mu, const DTT* cx, const DTT* cz, const DTT* ct, const DTT* cs,
                 bool zero_p, bool zero_d, DTT& dX, DTT& dY, DTT& dT, DTT& dZ, int* sweeps);
  void steps(const DTT& dX, const DTT& dT, const DTT& dZ, double* ap, double* ad);
  // sub: the random sub-stream of the eigensolve (null: forked from the main stream here)
  double max_step(const DTT& M, const DTT& dM, DTT* e, Counter* sub = nullptr);
  double max_step_diag(const DTT& v, const DTT& dv, DTT* e, Counter* sub = nullptr);
  DTT round_psd(const DTT& M, double delta, const DTT* shift, int var_id);
  IterLog iterate_once();
  // one iteration of the finishing phase (Section 3.5); fills log
  void finish_iteration(IterLog& log, const Measures& ms);
  double nu_ = 0.0;          // relaxation M + nu I >= 0 of the step lengths
  bool finish_done_ = false;
  // Mehrotra predictor and corrector solves with their step lengths; returns
  // whether both AMEn solves met their tolerance
  bool mehrotra(int dir, double mu, bool zp, bool zd, DTT& dX, DTT& dY, DTT& dT, DTT& dZ, double* ap, double* ad,
                int* sw);
  static constexpr double kFallbackStep = 1e-3;
  bool amen_ok_ = true;
  long long fallbacks_ = 0;
  void apply_update();  // X, Y, T, Z <- rounded (last_ iterate + step lengths x direction)

  // the last update of Algorithm 1, kept so that it can be damped and redone
  struct Update {
    DTT X, Y, T, Z, dX, dY, dT, dZ;
    double ap = 0.0, ad = 0.0, tol_p = 0.0, tol_d = 0.0;
    bool valid = false;
  };
  static constexpr int kMaxRetries = 4;
  Update last_;
  long long retries_ = 0;

  Problem p_;
  Options o_;
  Counter rnd_;
  DTT I_, X_, Y_, T_, Z_;
  double eta_, nB_, nC_;
  int it_ = 0, N_;
  long long gmres_iters_ = 0;
  double mu_now_ = 1.0;
  std::shared_ptr<RankPredictor> pred_;
  bool trace_ = false;
  std::vector<float> trace_x_, trace_y_;
  std::vector<int> prev_[4];
  std::vector<float> decay_[4];
  long long pred_used_ = 0, pred_fallbacks_ = 0;
  double forcing_it_ = 0.0;
  long long corrections_ = 0;
  std::unique_ptr<BlockTT> w_;
  DTT eX_, eZ_, eT_, eS_;
  bool haveX_ = false, haveZ_ = false, haveT_ = false, haveS_ = false;
  std::vector<cudaStream_t> side_;  // streams of the concurrent roundings
  // combined multiplier storage: diagonals of the non-idle masks P_Y, P_T and
  // of A_eq, A_ineq, K_Y, K_T (set when every one of them is diagonal and the
  // masks are disjoint)
  bool combined_ = false;
  DTT pY_, pT_, aeq_d_, ain_d_, ky_d_, kt_d_;
  bool has_deadline_ = false;
  std::chrono::steady_clock::time_point deadline_;
};

// Solves K x = b (N x N row-major FP64 on the device, kept; b becomes x) as the
// dense local solves of the AMEn sweep do. n_lz > 0: K is a reduced projected
// system whose last n_lz rows and first n_lz columns hold the symmetric
// positive definite LZ block, solved by block elimination (Cholesky of LZ, LU
// of the multipliers' Schur complement) with FP64 refinement; otherwise, or
// when LZ does not factor, LU with partial pivoting in FP64, or one FP32
// factorisation refined in FP64 for the reduced precisions. Returns the FP64
// relative residual; *corrections counts the refinement solves.
double dense_local_solve(int prec, int N, double* K, double* b, int* corrections, int n_lz = 0);

// Block-elimination solves completed, those of them with FP32 factors, those
// that fell back to the LU of the whole system, and the factorisations that
// stopped at a pivot of L_Z that was not positive, since the last reset.
void kkt_counts(unsigned long long* block, unsigned long long* fp32, unsigned long long* fallback,
                unsigned long long* not_pd, bool reset);

// min over e of <e, dM e>/<e, M e> (M positive definite): one-site ALS and
// two-site DMRG sweeps (relative SVD truncation tolerance tol at each split).
double min_gen_eig(const DTT& M, const DTT& dM, DTT* e, bool warm, Counter& rnd, int rank, int sweeps,
                   int prec);
// two-site sweeps stop once a full sweep changes the quotient by at most
// stall times its size (after two sweeps; 0: run every sweep)
double min_gen_eig_dmrg(const DTT& M, const DTT& dM, DTT* e, bool warm, Counter& rnd, int rank, int sweeps,
                        int prec, double tol, double stall = 0.0);
constexpr double kDmrgTol = 1e-8;
constexpr double kEigStall = 1e-9;

}  // namespace ttsdp
