// Learned plan selector: the MLP cost model of mlp.cu applied to planning.
//
// For a product the network predicts the log2-time (seconds) of each of the
// COSMA_MLP_OUT plan candidates (planner.cpp: tile class x k split x
// assignment order).  The analytic plan (Alg. 1's FindSeqSchedule + FitRanks
// with the cost model) stays the choice unless it is one of the candidates and
// the network predicts another applicable candidate faster by at least the
// dtype's margin (log2 seconds; 0.05, about 3.5 %, unless set -- the autotuner
// calibrates one per dtype on shapes kept out of training); an analytic plan
// outside the candidate set is kept.  Sizes outside the range the network was trained on, a missing
// network, or a call that may not synchronise (stream capture) also keep the
// analytic plan.  Choices are cached per (m, n, k, dtype).
#include <cuda_runtime.h>
#include <math.h>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace cosma {

namespace {

struct Selector {
  bool ready = false;
  std::vector<float> host;
  float* dev = nullptr;  // device parameters
  double lo = 0.0, hi = 0.0;
  unsigned dtype_mask = ~0u;  // dtypes the network was trained on
  float margin[8] = {0.05f, 0.05f, 0.05f, 0.05f, 0.05f, 0.05f, 0.05f, 0.05f};  // log2 s
  std::map<std::tuple<int64_t, int64_t, int64_t, int>, int> cache;
  cudaStream_t stream = nullptr;
  float* dX = nullptr;
  float* dY = nullptr;
  int cap = 0;
};

std::mutex g_sel_mu;
Selector g_sel[16];


bool same_plan(const cosma_plan& a, const cosma_plan& b) {
  return a.tile_m == b.tile_m && a.tile_n == b.tile_n && a.k_block == b.k_block &&
         a.pk == b.pk && a.order == b.order && a.ctas == b.ctas && a.pm == b.pm && a.pn == b.pn;
}

int features(int64_t m, int64_t n, int64_t k, int dtype, float* x) {
  if (m < 1 || n < 1 || k < 1 || !x) return COSMA_ERR_INVALID_ARG;
  if (dtype < COSMA_F64 || dtype > COSMA_F64_EMU_BF16) return COSMA_ERR_INVALID_ARG;
  x[0] = (float)(log2((double)m) / 16.0);
  x[1] = (float)(log2((double)n) / 16.0);
  x[2] = (float)(log2((double)k) / 16.0);
  for (int i = 3; i < COSMA_MLP_IN; ++i) x[i] = 0.f;
  x[3 + dtype] = 1.f;
  return COSMA_OK;
}

// Forward pass for `count` shapes and the best applicable candidate of each.
int predict_locked(Selector& s, int count, const int64_t* mnk, int dtype, int* best, float* pred,
                   const DeviceInfo& dev, const cosma_config& cfg) {
  if (!s.stream && cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess)
    return COSMA_ERR_CUDA;
  if (s.cap < count) {
    if (s.dX) cudaFree(s.dX);
    if (s.dY) cudaFree(s.dY);
    s.dX = s.dY = nullptr;
    s.cap = 0;
    if (cudaMalloc(&s.dX, (size_t)count * COSMA_MLP_IN * 4) != cudaSuccess ||
        cudaMalloc(&s.dY, (size_t)count * COSMA_MLP_OUT * 4) != cudaSuccess) {
      cudaGetLastError();
      return COSMA_ERR_NO_WORKSPACE;
    }
    s.cap = count;
  }
  std::vector<float> X((size_t)count * COSMA_MLP_IN), Y((size_t)count * COSMA_MLP_OUT);
  for (int i = 0; i < count; ++i) {
    const int rc = features(mnk[3 * i], mnk[3 * i + 1], mnk[3 * i + 2], dtype, &X[(size_t)i * COSMA_MLP_IN]);
    if (rc != COSMA_OK) return rc;
  }
  if (cudaMemcpyAsync(s.dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
    return COSMA_ERR_CUDA;
  if (mlp_forward(count, s.dX, s.dev, s.dY, s.stream) != 0) return COSMA_ERR_CUDA;
  if (cudaMemcpyAsync(Y.data(), s.dY, Y.size() * 4, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
      cudaStreamSynchronize(s.stream) != cudaSuccess)
    return COSMA_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    cosma_plan pa;
    const bool have_a =
        plan_gemm(m, n, k, dtype, COSMA_SELECT_ANALYTIC, dev, cfg, &pa, false) == COSMA_OK;
    int b = -1, ca = -1;
    float bv = 0.f;
    for (int c = 0; c < COSMA_MLP_OUT; ++c) {
      cosma_plan p;
      if (plan_candidate(m, n, k, dtype, c, dev, cfg, &p) != COSMA_OK) continue;
      if (have_a && ca < 0 && same_plan(p, pa)) ca = c;
      const float v = Y[(size_t)i * COSMA_MLP_OUT + c];
      if (b < 0 || v < bv) { b = c; bv = v; }
    }
    // -1: the analytic plan, kept (see the file header)
    int choice = -1;
    if (!have_a) choice = b;
    else if (ca >= 0) choice = (b >= 0 && bv < Y[(size_t)i * COSMA_MLP_OUT + ca] - s.margin[dtype & 7])
                                   ? b : ca;
    if (best) best[i] = choice;
  }
  if (pred) memcpy(pred, Y.data(), Y.size() * 4);
  return COSMA_OK;
}

int device_index() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 16) {
    cudaGetLastError();
    return -1;
  }
  return d;
}

}  // namespace

int learned_plan(int64_t m, int64_t n, int64_t k, int dtype, const DeviceInfo& dev,
                 const cosma_config& cfg, cosma_plan* out, bool may_sync) {
  if (m < 1 || n < 1 || k < 1) return COSMA_ERR_UNSUPPORTED;
  const int d = dev.device >= 0 ? dev.device : device_index();
  if (d < 0) return COSMA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_sel_mu);
  Selector& s = g_sel[d];
  if (!s.ready) return COSMA_ERR_UNSUPPORTED;
  if (dtype < 0 || dtype >= 32 || !((s.dtype_mask >> dtype) & 1u)) return COSMA_ERR_UNSUPPORTED;
  const double lm = log2((double)m), ln = log2((double)n), lk = log2((double)k);
  if (lm < s.lo || lm > s.hi || ln < s.lo || ln > s.hi || lk < s.lo || lk > s.hi)
    return COSMA_ERR_UNSUPPORTED;
  const auto key = std::make_tuple(m, n, k, dtype);
  auto it = s.cache.find(key);
  int c;
  if (it != s.cache.end()) {
    c = it->second;
  } else {
    if (!may_sync) return COSMA_ERR_UNSUPPORTED;
    const int64_t mnk[3] = {m, n, k};
    int rc = predict_locked(s, 1, mnk, dtype, &c, nullptr, dev, cfg);
    if (rc != COSMA_OK) return COSMA_ERR_UNSUPPORTED;
    s.cache[key] = c;
  }
  if (c < 0) return COSMA_ERR_UNSUPPORTED;  // the analytic plan is kept
  return plan_candidate(m, n, k, dtype, c, dev, cfg, out);
}

}  // namespace cosma

using namespace cosma;

namespace {
DeviceInfo info_or_default() {
  DeviceInfo info;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0 && current_info(&info) == COSMA_OK)
    return info;
  cudaGetLastError();
  DeviceInfo d;
  d.sms = 148;
  return d;
}
}  // namespace

extern "C" {

int cosma_plan_candidate(int64_t m, int64_t n, int64_t k, int dtype, int c, cosma_plan* out) {
  cosma_config cfg;
  cosma_get_config(&cfg);
  const DeviceInfo info = info_or_default();
  return plan_candidate(m, n, k, dtype, c, info, cfg, out);
}

int cosma_selector_features(int64_t m, int64_t n, int64_t k, int dtype, float* x) {
  return features(m, n, k, dtype, x);
}

int cosma_mlp_forward(int batch, const float* X, const float* params, float* Y, void* stream) {
  if (batch < 0 || (batch > 0 && (!X || !params || !Y))) return COSMA_ERR_INVALID_ARG;
  return mlp_forward(batch, X, params, Y, (cudaStream_t)stream) == 0 ? COSMA_OK : COSMA_ERR_CUDA;
}

int cosma_mlp_loss_grad(int batch, const float* X, const int* cand, const float* target,
                        const float* params, float* grad, float* loss, void* stream) {
  if (batch < 1 || !X || !cand || !target || !params || !grad) return COSMA_ERR_INVALID_ARG;
  void* scratch = nullptr;
  const int rc = lib_scratch(mlp_partial_bytes(batch), (cudaStream_t)stream, &scratch);
  if (rc != COSMA_OK) return rc;
  return mlp_loss_grad(batch, X, cand, target, params, grad, loss, static_cast<float*>(scratch),
                       (cudaStream_t)stream) == 0
             ? COSMA_OK
             : COSMA_ERR_CUDA;
}

int cosma_mlp_adam(int n, float* params, const float* grad, float* m, float* v, int step,
                   float lr, float beta1, float beta2, float eps, void* stream) {
  if (n < 1 || !params || !grad || !m || !v || step < 1) return COSMA_ERR_INVALID_ARG;
  return mlp_adam(n, params, grad, m, v, step, lr, beta1, beta2, eps, (cudaStream_t)stream) == 0
             ? COSMA_OK
             : COSMA_ERR_CUDA;
}

int cosma_selector_set(const float* params, double log2_lo, double log2_hi) {
  const int d = device_index();
  if (d < 0) return COSMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_sel_mu);
  Selector& s = g_sel[d];
  s.cache.clear();
  if (!params) {
    s.ready = false;
    return COSMA_OK;
  }
  if (!(log2_lo <= log2_hi)) return COSMA_ERR_INVALID_ARG;
  if (!s.dev && cudaMalloc(&s.dev, COSMA_MLP_PARAMS * 4) != cudaSuccess) {
    cudaGetLastError();
    return COSMA_ERR_NO_WORKSPACE;
  }
  s.host.assign(params, params + COSMA_MLP_PARAMS);
  if (cudaMemcpy(s.dev, params, COSMA_MLP_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return COSMA_ERR_CUDA;
  s.lo = log2_lo;
  s.hi = log2_hi;
  s.dtype_mask = ~0u;
  s.ready = true;
  return COSMA_OK;
}

int cosma_selector_margin(int dtype, float log2_margin) {
  if (dtype < COSMA_F64 || dtype > COSMA_F32_EMU_TF32 || !(log2_margin >= 0.f))
    return COSMA_ERR_INVALID_ARG;
  const int d = device_index();
  if (d < 0) return COSMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_sel_mu);
  Selector& s = g_sel[d];
  s.margin[dtype] = log2_margin;
  s.cache.clear();
  return COSMA_OK;
}

int cosma_selector_restrict(unsigned dtype_mask) {
  const int d = device_index();
  if (d < 0) return COSMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_sel_mu);
  Selector& s = g_sel[d];
  if (!s.ready) return COSMA_ERR_UNSUPPORTED;
  s.dtype_mask = dtype_mask;
  s.cache.clear();
  return COSMA_OK;
}

int cosma_selector_predict(int count, const int64_t* mnk, int dtype, int* best, float* pred) {
  if (count < 0 || (count > 0 && (!mnk || !best))) return COSMA_ERR_INVALID_ARG;
  if (count == 0) return COSMA_OK;
  cosma_config cfg;
  cosma_get_config(&cfg);
  const DeviceInfo info = info_or_default();
  const int d = device_index();
  if (d < 0) return COSMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_sel_mu);
  Selector& s = g_sel[d];
  if (!s.ready) return COSMA_ERR_UNSUPPORTED;
  return predict_locked(s, count, mnk, dtype, best, pred, info, cfg);
}

}  // extern "C"
