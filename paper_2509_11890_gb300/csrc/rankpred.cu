// MLP kernels of the learned rank predictor: dense layers as strided GEMMs,
// fused bias + tanh, sigmoid / squared-error head, tanh backward, column sums
// for bias gradients and an Adam update, all in FP32 on the device.
#include <cmath>

#include "gemm.cuh"
#include "rankpred.cuh"
#include "tt.cuh"

namespace ttsdp {

namespace {

constexpr int NI = kPredIn, NH = kPredHidden;
// offsets of the parameter blocks in the flat vector
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH * NH,
              OW4 = OB3 + NH, OB4 = OW4 + NH;

int g1(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

#define LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void bias_tanh_kernel(float* H, const float* b, int n, int w) {
  LOOP(e, (long long)n * w) H[e] = tanhf(H[e] + b[e % w]);
}

// y = sigmoid(z + b4); dz = 2 (y - t) / n * y (1 - y); per-sample squared error
__global__ void head_kernel(const float* z, const float* b4, const float* t, int n, float* y, float* dz, float* err) {
  LOOP(i, n) {
    const float yi = 1.f / (1.f + expf(-(z[i] + b4[0])));
    y[i] = yi;
    if (t) {
      const float r = yi - t[i];
      dz[i] = 2.f * r / n * yi * (1.f - yi);
      err[i] = r * r;
    }
  }
}

// D[i][j] = dz[i] * w[j] * (1 - H[i][j]^2)
__global__ void outer_tanh_back_kernel(const float* dz, const float* w, const float* H, int n, int wdt, float* D) {
  LOOP(e, (long long)n * wdt) {
    const long long i = e / wdt, j = e % wdt;
    const float h = H[e];
    D[e] = dz[i] * w[j] * (1.f - h * h);
  }
}

__global__ void tanh_back_kernel(float* D, const float* H, long long n) {
  LOOP(e, n) {
    const float h = H[e];
    D[e] *= (1.f - h * h);
  }
}

// out[j] = sum_i D[i][j]
__global__ void colsum_kernel(const float* D, int n, int w, float* out) {
  const int j = blockIdx.x;
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += D[(long long)i * w + j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  LOOP(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void fill_f_kernel(float* p, int n, float v) { LOOP(i, n) p[i] = v; }

// dense layer: H (n x wo) = X (n x wi) W^T (W: wo x wi, row-major)
void dense(const float* X, int n, int wi, const float* W, int wo, float* H, cudaStream_t st) {
  gemm_rm<float>(false, true, n, wo, wi, 1.f, X, wi, 0, W, wi, 0, 0.f, H, wo, 0, 1, st);
}

}  // namespace

RankPredictor::RankPredictor(uint64_t seed) : p_(kPredParams), m_(kPredParams), v_(kPredParams) {
  // Xavier-uniform weights from the SplitMix64 counter stream, zero biases
  Counter c;
  c.seed = seed;
  std::vector<double> u = c.draw(kPredParams);
  std::vector<float> h(kPredParams, 0.f);
  auto init = [&](int off, int fan_in, int fan_out, int count) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < count; ++i) h[off + i] = (float)(a * u[off + i]);
  };
  init(OW1, NI, NH, NH * NI);
  init(OW2, NH, NH, NH * NH);
  init(OW3, NH, NH, NH * NH);
  init(OW4, NH, 1, NH);
  set_params(h.data());
  cudaStream_t st = cur_stream();
  fill_f_kernel<<<g1(kPredParams), 256, 0, st>>>(m_.get(), kPredParams, 0.f);
  fill_f_kernel<<<g1(kPredParams), 256, 0, st>>>(v_.get(), kPredParams, 0.f);
  count_launch();
  count_launch();
  check_launch("rankpred init");
}

void RankPredictor::set_params(const float* host) {
  TT_CUDA(cudaMemcpyAsync(p_.get(), host, kPredParams * sizeof(float), cudaMemcpyHostToDevice, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
}

void RankPredictor::get_params(float* host) const {
  TT_CUDA(cudaMemcpyAsync(host, p_.get(), kPredParams * sizeof(float), cudaMemcpyDeviceToHost, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
}

void RankPredictor::predict_dev(const float* X, int n, float* y) const {
  cudaStream_t st = cur_stream();
  const float* p = p_.get();
  DBuf<float> H1((size_t)n * NH), H2((size_t)n * NH), H3((size_t)n * NH), z(n);
  dense(X, n, NI, p + OW1, NH, H1.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H1.get(), p + OB1, n, NH);
  dense(H1.get(), n, NH, p + OW2, NH, H2.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H2.get(), p + OB2, n, NH);
  dense(H2.get(), n, NH, p + OW3, NH, H3.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H3.get(), p + OB3, n, NH);
  dense(H3.get(), n, NH, p + OW4, 1, z.get(), st);
  head_kernel<<<g1(n), 256, 0, st>>>(z.get(), p + OB4, nullptr, n, y, nullptr, nullptr);
  for (int i = 0; i < 4; ++i) count_launch();
  check_launch("rankpred forward");
}

std::vector<float> RankPredictor::predict(const std::vector<float>& Xh, int n) const {
  if (n <= 0) return {};
  DBuf<float> X((size_t)n * NI), y(n);
  TT_CUDA(cudaMemcpyAsync(X.get(), Xh.data(), (size_t)n * NI * sizeof(float), cudaMemcpyHostToDevice, cur_stream()));
  predict_dev(X.get(), n, y.get());
  std::vector<float> out(n);
  TT_CUDA(cudaMemcpyAsync(out.data(), y.get(), n * sizeof(float), cudaMemcpyDeviceToHost, cur_stream()));
  TT_CUDA(sync_stream(cur_stream()));
  return out;
}

float RankPredictor::loss_grad_dev(const float* X, const float* t, int n, float* g) {
  cudaStream_t st = cur_stream();
  const float* p = p_.get();
  DBuf<float> H1((size_t)n * NH), H2((size_t)n * NH), H3((size_t)n * NH), z(n), y(n), dz(n), err(n);
  DBuf<float> D3((size_t)n * NH), D2((size_t)n * NH), D1((size_t)n * NH);
  // forward
  dense(X, n, NI, p + OW1, NH, H1.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H1.get(), p + OB1, n, NH);
  dense(H1.get(), n, NH, p + OW2, NH, H2.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H2.get(), p + OB2, n, NH);
  dense(H2.get(), n, NH, p + OW3, NH, H3.get(), st);
  bias_tanh_kernel<<<g1((long long)n * NH), 256, 0, st>>>(H3.get(), p + OB3, n, NH);
  dense(H3.get(), n, NH, p + OW4, 1, z.get(), st);
  head_kernel<<<g1(n), 256, 0, st>>>(z.get(), p + OB4, t, n, y.get(), dz.get(), err.get());
  // backward: output layer
  gemm_rm<float>(true, false, NH, 1, n, 1.f, H3.get(), NH, 0, dz.get(), 1, 0, 0.f, g + OW4, 1, 0, 1, st);
  colsum_kernel<<<1, 256, 0, st>>>(dz.get(), n, 1, g + OB4);
  // layer 3
  outer_tanh_back_kernel<<<g1((long long)n * NH), 256, 0, st>>>(dz.get(), p + OW4, H3.get(), n, NH, D3.get());
  gemm_rm<float>(true, false, NH, NH, n, 1.f, D3.get(), NH, 0, H2.get(), NH, 0, 0.f, g + OW3, NH, 0, 1, st);
  colsum_kernel<<<NH, 256, 0, st>>>(D3.get(), n, NH, g + OB3);
  // layer 2
  gemm_rm<float>(false, false, n, NH, NH, 1.f, D3.get(), NH, 0, p + OW3, NH, 0, 0.f, D2.get(), NH, 0, 1, st);
  tanh_back_kernel<<<g1((long long)n * NH), 256, 0, st>>>(D2.get(), H2.get(), (long long)n * NH);
  gemm_rm<float>(true, false, NH, NH, n, 1.f, D2.get(), NH, 0, H1.get(), NH, 0, 0.f, g + OW2, NH, 0, 1, st);
  colsum_kernel<<<NH, 256, 0, st>>>(D2.get(), n, NH, g + OB2);
  // layer 1
  gemm_rm<float>(false, false, n, NH, NH, 1.f, D2.get(), NH, 0, p + OW2, NH, 0, 0.f, D1.get(), NH, 0, 1, st);
  tanh_back_kernel<<<g1((long long)n * NH), 256, 0, st>>>(D1.get(), H1.get(), (long long)n * NH);
  gemm_rm<float>(true, false, NH, NI, n, 1.f, D1.get(), NH, 0, X, NI, 0, 0.f, g + OW1, NI, 0, 1, st);
  colsum_kernel<<<NH, 256, 0, st>>>(D1.get(), n, NH, g + OB1);
  for (int i = 0; i < 12; ++i) count_launch();
  check_launch("rankpred backward");
  // mean squared error
  DBuf<float> s(1);
  colsum_kernel<<<1, 256, 0, st>>>(err.get(), n, 1, s.get());
  count_launch();
  float h = 0.f;
  TT_CUDA(cudaMemcpyAsync(&h, s.get(), sizeof(float), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  return h / n;
}

float RankPredictor::grad(const float* Xh, const float* th, int n, float* gh) {
  TT_CHECK(n > 0, TT_E_INVALID_ARG, "empty batch");
  cudaStream_t st = cur_stream();
  DBuf<float> X((size_t)n * NI), t(n), g(kPredParams);
  TT_CUDA(cudaMemcpyAsync(X.get(), Xh, (size_t)n * NI * sizeof(float), cudaMemcpyHostToDevice, st));
  TT_CUDA(cudaMemcpyAsync(t.get(), th, n * sizeof(float), cudaMemcpyHostToDevice, st));
  float loss = loss_grad_dev(X.get(), t.get(), n, g.get());
  TT_CUDA(cudaMemcpyAsync(gh, g.get(), kPredParams * sizeof(float), cudaMemcpyDeviceToHost, st));
  TT_CUDA(sync_stream(st));
  return loss;
}

float RankPredictor::train(const float* Xh, const float* th, int n, int epochs, int batch, float lr, uint64_t seed) {
  TT_CHECK(n > 0 && epochs > 0 && batch > 0, TT_E_INVALID_ARG, "bad training arguments");
  cudaStream_t st = cur_stream();
  // shuffle once per epoch on the host (SplitMix64), upload each epoch's permuted copy
  DBuf<float> X((size_t)n * NI), t(n), g(kPredParams);
  std::vector<float> xs((size_t)n * NI), ts(n);
  std::vector<int> perm(n);
  Counter c;
  c.seed = seed;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::vector<double> u = c.draw(n);
    for (int i = n - 1; i > 0; --i) {  // Fisher-Yates
      int j = (int)((u[i] * 0.5 + 0.5) * (i + 1));
      if (j > i) j = i;
      std::swap(perm[i], perm[j]);
    }
    for (int i = 0; i < n; ++i) {
      for (int f = 0; f < NI; ++f) xs[(size_t)i * NI + f] = Xh[(size_t)perm[i] * NI + f];
      ts[i] = th[perm[i]];
    }
    TT_CUDA(cudaMemcpyAsync(X.get(), xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    TT_CUDA(cudaMemcpyAsync(t.get(), ts.data(), ts.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    for (int b0 = 0; b0 < n; b0 += batch) {
      const int nb = std::min(batch, n - b0);
      loss_grad_dev(X.get() + (size_t)b0 * NI, t.get() + b0, nb, g.get());
      ++step_;
      const float c1 = 1.f - std::pow(b1, (float)step_), c2 = 1.f - std::pow(b2, (float)step_);
      adam_kernel<<<g1(kPredParams), 256, 0, st>>>(p_.get(), m_.get(), v_.get(), g.get(), kPredParams, lr, b1, b2, c1,
                                                   c2, eps);
      count_launch();
    }
  }
  check_launch("rankpred train");
  TT_CUDA(cudaMemcpyAsync(X.get(), Xh, (size_t)n * NI * sizeof(float), cudaMemcpyHostToDevice, st));
  TT_CUDA(cudaMemcpyAsync(t.get(), th, n * sizeof(float), cudaMemcpyHostToDevice, st));
  return loss_grad_dev(X.get(), t.get(), n, g.get());
}

}  // namespace ttsdp
