// Library-internal declarations shared by the host runtime and the kernel
// translation units.  Not part of the ABI.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/cosma.h"
#include "schedule.h"

namespace cosma {

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;      // max dynamic shared memory per block (bytes)
  int smem_per_sm = 0;
  int regs_per_sm = 0;
  int l2_bytes = 0;
  int cc_major = 0, cc_minor = 0;
};

// Per-kernel-family constants used by the planner's cost model.
struct KernelDesc {
  int kernel;
  int tile_m, tile_n, k_block, stages;
  int w_in, w_acc, w_out;     // bytes per input element / accumulator / output
  double fast_bytes;          // S in bytes for this kernel on one SM
  double flops_per_clk_sm;    // pipe peak per SM (dense)
  double efficiency;          // fraction of the pipe peak the main loop sustains
};

// Planner (planner.cpp).
int plan_gemm(int64_t m, int64_t n, int64_t k, int dtype, int selector, const DeviceInfo& dev,
              const cosma_config& cfg, cosma_plan* out, bool may_sync = true);
int plan_candidate(int64_t m, int64_t n, int64_t k, int dtype, int c, const DeviceInfo& dev,
                   const cosma_config& cfg, cosma_plan* out);
int validate_plan(int64_t m, int64_t n, int64_t k, int dtype, const DeviceInfo& dev,
                  const cosma_plan& p);
Sched sched_from_plan(int64_t m, int64_t n, int64_t k, const cosma_plan& p);
int find_seq_schedule(long long S, int* a, int* b);
int fit_ranks_weighted(int64_t m, int64_t n, int64_t k, int p, double delta, double wa, double wb,
                       double wc, int grid[3]);
int learned_plan(int64_t m, int64_t n, int64_t k, int dtype, const DeviceInfo& dev,
                 const cosma_config& cfg, cosma_plan* out, bool may_sync);  // selector.cu
// MLP kernels (mlp.cu)
int mlp_forward(int batch, const float* X, const float* params, float* Y, cudaStream_t st);
int mlp_loss_grad(int batch, const float* X, const int* cand, const float* target,
                  const float* params, float* grad, float* loss, float* partial, cudaStream_t st);
long long mlp_partial_bytes(int batch);
int mlp_adam(int n, float* params, const float* grad, float* m, float* v, int step, float lr,
             float beta1, float beta2, float eps, cudaStream_t st);
// Library workspace for internal users (api.cu); grows outside capture only.
int lib_scratch(long long bytes, cudaStream_t st, void** out);
// Device info of the current device (api.cu).
int current_info(DeviceInfo* out);

// Kernel launchers (return cudaError_t values).
struct GemmArgs {
  int64_t m, n, k;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  void* C; int64_t ldc;
};
int launch_simt(int dtype, const GemmArgs& g, const Sched& s, void* partial, int* status,
                cudaStream_t st);
int launch_reduce(int dtype, const GemmArgs& g, int pk, const void* partial, cudaStream_t st);

// Launch accounting (api.cu): every kernel launch the library makes calls this.
void count_launch(int n = 1);
// Event pair around the dominant kernel of a call when profiling is enabled.
void prof_mark(cudaStream_t st, bool begin);

// Bytes of workspace a plan needs (split-k partials, operand copies, slices).
long long workspace_bytes(int64_t m, int64_t n, int64_t k, int dtype, const cosma_plan& p);

}  // namespace cosma
