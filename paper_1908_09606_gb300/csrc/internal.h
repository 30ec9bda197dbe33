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
// What a launcher outside api.cu needs of the current device (api.cu).
struct LibContext {
  DeviceInfo info;
  cosma_config cfg;
  int* status;           // device status word
  long long wait_limit;  // clock cycles before a device wait gives up
};
int lib_context(LibContext* out);
// cosma_gemm on device operands, planned by the configured selector (api.cu).
int run_device(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
               int64_t ldb, void* C, int64_t ldc, int dtype, void* stream);
// cosma_gemm_ex on device operands (api.cu).
int run_device_ex(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
                  int64_t ldb, void* C, int64_t ldc, int dtype, double alpha, double beta,
                  int trans_a, int trans_b, void* stream);

// Kernel launchers (return cudaError_t values).
struct GemmArgs {
  int64_t m, n, k;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  void* C; int64_t ldc;
  double alpha = 1.0, beta = 0.0;  // C = alpha A B + beta C (beta == 0: C is not read)
  // 1: the operand is stored transposed (A as k x m with lda >= m, B as n x k with
  // ldb >= k).  Only the bf16 and emulated launchers take transposed operands.
  int trans_a = 0, trans_b = 0;
};
int launch_simt(int dtype, const GemmArgs& g, const Sched& s, void* partial, int* status,
                cudaStream_t st);
int launch_reduce(int dtype, const GemmArgs& g, int pk, const void* partial, cudaStream_t st);
// C = beta C (beta == 0: C = 0 without reading it), for k == 0 or alpha == 0.
int launch_scale(int dtype, const GemmArgs& g, cudaStream_t st);
// dst (cols x rows, ld_dst) = transpose of src (rows x cols, ld_src), 4- or 8-byte elements.
int launch_transpose(int elem_bytes, const void* src, int64_t rows, int64_t cols,
                     int64_t ld_src, void* dst, int64_t ld_dst, cudaStream_t st);

// Emulated FP64 (emu.cu): workspace layout and the three phases of a product.
struct EmuWorkspace {
  int* eA;                 // row exponents of A [m]
  int* eB;                 // column exponents of B [n]
  void* SA;                // bf16 slices of A, k-blocked: [s][k panels][m][row_pitch]
  void* SB;                // bf16 slices of B^T, k-blocked: [s][k panels][n][row_pitch]
  long long* T;            // running totals of the kernels (one region per CTA)
  int64_t t_bytes;         // bytes at T
  long long* X;            // k-split plans: the product's exact fixed-point total [m][n]
                           // (null when the workspace was sized without a split)
  unsigned int* lockstep;  // one counter for lock-step rounds
  int64_t row_pitch;       // elements per row of one k panel (a row block starts at
                           // row * row_pitch)
};
// sms: the SM count of the plans the workspace serves (cosma_plan::sms);
// split_elems: elements of the exact total a k-split plan sums into (m n for a
// plan with pk > 1, else 0).
long long emu_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_config& cfg, int sms,
                              int64_t split_elems);
// k rounded up to whole panels of the k-blocked slice layout.
int64_t emu_padded_k(int64_t k);
// COSMA_OK when the element format's operand preparation covers this k, else
// COSMA_ERR_UNSUPPORTED (api.cu); checked before anything is sized or allocated.
int k_supported(int dtype, int64_t k);
EmuWorkspace emu_carve(void* ws, int64_t m, int64_t n, int64_t k, const cosma_config& cfg,
                       int sms, int64_t split_elems);
int emu_check_config(const cosma_config& cfg);
// Exponents and slices of rows [0, m) of A into eA[0..m) and SA (slice_rows
// rows between slices); of columns [0, n) of B likewise.
// trans = 1: the operand is stored transposed (A as k x m, B as n x k).
int emu_prepare_a(const double* A, int64_t m, int64_t k, int64_t lda, int trans, int* eA,
                  void* SA, int64_t slice_rows, int* status, const cosma_config& cfg,
                  cudaStream_t st);
int emu_prepare_b(const double* B, int64_t k, int64_t n, int64_t ldb, int trans, int* eB,
                  void* SB, int64_t slice_rows, int* status, const cosma_config& cfg,
                  cudaStream_t st);
// C[m x n] = alpha (product of the prepared slices) + beta C, under plan p (an
// F64_EMU_BF16 plan for m x n x k).  T: t_bytes of running-total scratch (one
// region per CTA of the launch; COSMA_ERR_INVALID_ARG when too small).  X: at
// least m n int64 when p.pk > 1 (the k slices' exact totals are summed there),
// else unused.
int emu_multiply(int64_t m, int64_t n, int64_t k, const cosma_plan& p, const cosma_config& cfg,
                 const int* eA, const void* SA, int64_t a_slice_rows, const int* eB,
                 const void* SB, int64_t b_slice_rows, double* C, int64_t ldc, double alpha,
                 double beta, long long* T, int64_t t_bytes, long long* X,
                 unsigned int* lockstep, int* status, long long wait_limit, cudaStream_t st);
int launch_emu_bf16(const GemmArgs& g, const cosma_plan& p, const cosma_config& cfg, void* ws,
                    long long ws_bytes, int* status, long long wait_limit, cudaStream_t st);

// Launch accounting (api.cu): every kernel launch the library makes calls this.
void count_launch(int n = 1);
// Event pair around the dominant kernel of a call when profiling is enabled.
void prof_mark(cudaStream_t st, bool begin);
// Whether cosma_profile_enable is on (api.cu).
bool prof_enabled();

// Bytes of workspace a plan needs (split-k partials, operand copies, slices).
long long workspace_bytes(int64_t m, int64_t n, int64_t k, int dtype, const cosma_plan& p);

}  // namespace cosma
