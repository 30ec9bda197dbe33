// K-MLP-FWD / K-MLP-BWD / K-MLP-ADAM: the selector's cost model (learned
// pattern; not in the paper).  A 3-layer FP32 network IN -> 64 -> 64 -> OUT
// with ReLU predicts the log-time of each plan candidate from the log sizes
// and the dtype of a product.
//
// Each block keeps all weights in shared memory and walks rows of the batch;
// thread j owns hidden unit j.  The backward pass accumulates a block's
// gradients in registers (thread j: column j of dW2 and dW3, row j of dW1)
// and writes one partial per block; a second kernel sums the partials in a
// fixed order, so gradients do not depend on scheduling.  Parameter layout:
// W1 (64 x IN), b1, W2 (64 x 64), b2, W3 (OUT x 64), b3.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace cosma {

namespace {

constexpr int IN = COSMA_MLP_IN, HID = COSMA_MLP_HIDDEN, OUT = COSMA_MLP_OUT;
constexpr int O_W1 = 0, O_B1 = O_W1 + HID * IN, O_W2 = O_B1 + HID, O_B2 = O_W2 + HID * HID,
              O_W3 = O_B2 + HID, O_B3 = O_W3 + OUT * HID, NP = O_B3 + OUT;
static_assert(NP == COSMA_MLP_PARAMS, "parameter count");
constexpr int GRAD_BLOCKS = 64;

__device__ __forceinline__ void load_params(const float* __restrict__ p, float* sp) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sp[i] = p[i];
  __syncthreads();
}

__global__ void __launch_bounds__(HID) mlp_forward_kernel(int batch, const float* __restrict__ X,
                                                          const float* __restrict__ p,
                                                          float* __restrict__ Y) {
  __shared__ float sp[NP];
  __shared__ float x[IN], h1[HID], h2[HID];
  load_params(p, sp);
  const int j = threadIdx.x;
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    if (j < IN) x[j] = X[(int64_t)b * IN + j];
    __syncthreads();
    float z = sp[O_B1 + j];
#pragma unroll
    for (int i = 0; i < IN; ++i) z += sp[O_W1 + j * IN + i] * x[i];
    h1[j] = fmaxf(z, 0.f);
    __syncthreads();
    z = sp[O_B2 + j];
    for (int i = 0; i < HID; ++i) z += sp[O_W2 + j * HID + i] * h1[i];
    h2[j] = fmaxf(z, 0.f);
    __syncthreads();
    if (j < OUT) {
      float y = sp[O_B3 + j];
      for (int i = 0; i < HID; ++i) y += sp[O_W3 + j * HID + i] * h2[i];
      Y[(int64_t)b * OUT + j] = y;
    }
    __syncthreads();
  }
}

// Per-block partial gradients of L = (1/B) sum_b (y_b[c_b] - t_b)^2.
__global__ void __launch_bounds__(HID) mlp_grad_kernel(int batch, const float* __restrict__ X,
                                                       const int* __restrict__ cand,
                                                       const float* __restrict__ target,
                                                       const float* __restrict__ p,
                                                       float* __restrict__ partial) {
  __shared__ float sp[NP];
  __shared__ float x[IN], h1[HID], h2[HID], dz2[HID];
  __shared__ float s_dy, s_loss;
  __shared__ int s_c;
  load_params(p, sp);
  const int j = threadIdx.x;
  float gW1[IN], gW2[HID], gW3[OUT];
  float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int i = 0; i < IN; ++i) gW1[i] = 0.f;
#pragma unroll
  for (int i = 0; i < HID; ++i) gW2[i] = 0.f;
#pragma unroll
  for (int i = 0; i < OUT; ++i) gW3[i] = 0.f;
  if (j == 0) s_loss = 0.f;
  const float inv_b = 1.0f / (float)batch;
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    if (j < IN) x[j] = X[(int64_t)b * IN + j];
    if (j == 0) s_c = cand[b];
    __syncthreads();
    if (s_c < 0 || s_c >= OUT) {  // not a candidate index: the row contributes nothing
      __syncthreads();
      continue;
    }
    float z1 = sp[O_B1 + j];
#pragma unroll
    for (int i = 0; i < IN; ++i) z1 += sp[O_W1 + j * IN + i] * x[i];
    h1[j] = fmaxf(z1, 0.f);
    __syncthreads();
    float z2 = sp[O_B2 + j];
    for (int i = 0; i < HID; ++i) z2 += sp[O_W2 + j * HID + i] * h1[i];
    h2[j] = fmaxf(z2, 0.f);
    __syncthreads();
    const int c = s_c;
    if (j == 0) {
      float y = sp[O_B3 + c];
      for (int i = 0; i < HID; ++i) y += sp[O_W3 + c * HID + i] * h2[i];
      const float r = y - target[b];
      s_loss += r * r;
      s_dy = 2.0f * r * inv_b;
    }
    __syncthreads();
    const float dy = s_dy;
    // layer 3
#pragma unroll
    for (int o = 0; o < OUT; ++o)
      if (o == c) gW3[o] += dy * h2[j];
    if (j == c) gb3 += dy;
    const float d2 = (z2 > 0.f) ? sp[O_W3 + c * HID + j] * dy : 0.f;
    dz2[j] = d2;
    __syncthreads();
    // layer 2: thread j owns column j of dW2
#pragma unroll
    for (int i = 0; i < HID; ++i) gW2[i] += dz2[i] * h1[j];
    gb2 += d2;
    float dh1 = 0.f;
    for (int i = 0; i < HID; ++i) dh1 += sp[O_W2 + i * HID + j] * dz2[i];
    const float d1 = (z1 > 0.f) ? dh1 : 0.f;
#pragma unroll
    for (int i = 0; i < IN; ++i) gW1[i] += d1 * x[i];
    gb1 += d1;
    __syncthreads();
  }
  float* out = partial + (int64_t)blockIdx.x * (NP + 1);
#pragma unroll
  for (int i = 0; i < IN; ++i) out[O_W1 + j * IN + i] = gW1[i];
  out[O_B1 + j] = gb1;
#pragma unroll
  for (int i = 0; i < HID; ++i) out[O_W2 + i * HID + j] = gW2[i];
  out[O_B2 + j] = gb2;
#pragma unroll
  for (int o = 0; o < OUT; ++o) out[O_W3 + o * HID + j] = gW3[o];
  // thread j accumulated db3[j] over the rows whose observed candidate is j
  if (j < OUT) out[O_B3 + j] = gb3;
  if (j == 0) out[NP] = s_loss * inv_b;
}

// grad[i] = sum over blocks (in block order) of partial[block][i]; loss likewise.
__global__ void mlp_reduce_kernel(int blocks, const float* __restrict__ partial,
                                  float* __restrict__ grad, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > NP) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += partial[(int64_t)b * (NP + 1) + i];
  if (i < NP) grad[i] = s;
  else if (loss) *loss = s;
}

__global__ void mlp_adam_kernel(int n, float* __restrict__ p, const float* __restrict__ g,
                                float* __restrict__ m, float* __restrict__ v, float lr,
                                float beta1, float beta2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

int mlp_forward(int batch, const float* X, const float* params, float* Y, cudaStream_t st) {
  if (batch <= 0) return 0;
  const int blocks = batch < 152 * 8 ? batch : 152 * 8;
  mlp_forward_kernel<<<blocks, HID, 0, st>>>(batch, X, params, Y);
  count_launch();
  return (int)cudaGetLastError();
}

int mlp_loss_grad(int batch, const float* X, const int* cand, const float* target,
                  const float* params, float* grad, float* loss, float* partial,
                  cudaStream_t st) {
  const int blocks = batch < GRAD_BLOCKS ? batch : GRAD_BLOCKS;
  mlp_grad_kernel<<<blocks, HID, 0, st>>>(batch, X, cand, target, params, partial);
  count_launch();
  mlp_reduce_kernel<<<(NP + 1 + 255) / 256, 256, 0, st>>>(blocks, partial, grad, loss);
  count_launch();
  return (int)cudaGetLastError();
}

long long mlp_partial_bytes(int batch) {
  const int blocks = batch < GRAD_BLOCKS ? batch : GRAD_BLOCKS;
  return (long long)blocks * (NP + 1) * 4;
}

int mlp_adam(int n, float* params, const float* grad, float* m, float* v, int step, float lr,
             float beta1, float beta2, float eps, cudaStream_t st) {
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  mlp_adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, params, grad, m, v, lr, beta1, beta2, eps,
                                                   c1, c2);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace cosma
