// Learned per-bond rank predictor for TT rounding (an addition of this
// library; the paper chooses every rank by the adaptive SVD): a 9 -> 64 -> 64
// -> 64 -> 1 MLP (tanh hidden layers, sigmoid output) trained on the GPU by
// the library's own forward / backward / Adam kernels on rounding traces that
// the solver records, predicting (chosen rank) / (rank cap).
#pragma once

#include <vector>

#include "common.cuh"

namespace ttsdp {

constexpr int kPredIn = 10, kPredHidden = 64;
constexpr int kPredParams = kPredHidden * kPredIn + kPredHidden + 2 * (kPredHidden * kPredHidden + kPredHidden) +
                            kPredHidden + 1;

class RankPredictor {
 public:
  explicit RankPredictor(uint64_t seed);
  void set_params(const float* host);
  void get_params(float* host) const;
  // y[i] in (0, 1) for the n feature rows of X (row-major n x 9, device)
  void predict_dev(const float* X, int n, float* y) const;
  std::vector<float> predict(const std::vector<float>& X, int n) const;
  // mean squared error and its gradient (host outputs) on one batch
  float grad(const float* Xh, const float* th, int n, float* gh);
  // Adam on mini-batches; returns the final full-data loss
  float train(const float* Xh, const float* th, int n, int epochs, int batch, float lr, uint64_t seed);

 private:
  float loss_grad_dev(const float* X, const float* t, int n, float* g);
  DBuf<float> p_, m_, v_;
  long long step_ = 0;
};

}  // namespace ttsdp
