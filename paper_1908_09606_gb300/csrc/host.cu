// Host-resident operands (cosma_gemm_host): C = A B with A, B, C in host
// memory, the copies pipelined against the kernels.
//
// The product is cut into Rm x Rn blocks (rows of A x columns of B, Rm, Rn <= 2).
// Three queues run concurrently:
//   copy-in  (library stream): A_0, B_0, B_1, ..., A_1, ...  host -> device
//   compute  (caller's stream): block (i, j) in row-major order, each after its
//            A_i and B_j have landed; emulated FP64 prepares the exponents and
//            slices of A_i and B_j once, then multiplies every block from them
//   copy-out (library stream): C block (i, j) as soon as its kernels are done
// so only the first A and B blocks and the last C block are exposed.  The two
// copy streams fork from the caller's stream (an event recorded there first:
// the previous call's work on the staging buffers is finished) and join back
// to it (the caller's stream waits for the last copy-out), so the call is
// stream-ordered and may be captured into a CUDA graph.
#include <cuda_runtime.h>
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cosma {

namespace {

constexpr int kMaxDevices = 16;
constexpr int kMaxR = 2;
constexpr int kEvents = 2 + 2 * kMaxR + kMaxR * kMaxR;
constexpr int64_t kSplitMin = 8192;  // a dimension is cut in two from this length

struct HostState {
  bool ready = false;
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t ev[kEvents] = {};
  void* stage = nullptr;
  size_t stage_bytes = 0;
  bool captured = false;       // stage is recorded in a captured graph
  std::vector<void*> retired;  // captured stages given up on growth; freed at finalize
};

std::mutex g_host_mu;
HostState g_host[kMaxDevices];

// Phase events of the last cosma_gemm_host call made while profiling was on
// (cosma_profile_enable) and not under stream capture.
struct HostPhases {
  bool ready = false, valid = false;
  cudaEvent_t start = nullptr, in_done = nullptr, end = nullptr;
  cudaEvent_t pb[kMaxR * kMaxR] = {}, pe[kMaxR * kMaxR] = {};
  int nblocks = 0;
};
HostPhases g_phases[kMaxDevices];

int phases_init(HostPhases& p) {
  if (p.ready) return COSMA_OK;
  cudaEvent_t* all[3] = {&p.start, &p.in_done, &p.end};
  for (cudaEvent_t* e : all)
    if (cudaEventCreate(e) != cudaSuccess) return COSMA_ERR_CUDA;
  for (int i = 0; i < kMaxR * kMaxR; ++i)
    if (cudaEventCreate(&p.pb[i]) != cudaSuccess || cudaEventCreate(&p.pe[i]) != cudaSuccess)
      return COSMA_ERR_CUDA;
  p.ready = true;
  return COSMA_OK;
}

inline int64_t rup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

int init_state(HostState& h) {
  if (h.ready) return COSMA_OK;
  if (cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking) != cudaSuccess)
    return COSMA_ERR_CUDA;
  for (int i = 0; i < kEvents; ++i)
    if (cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming) != cudaSuccess)
      return COSMA_ERR_CUDA;
  h.ready = true;
  return COSMA_OK;
}

int staging(HostState& h, size_t bytes, cudaStream_t st, uint8_t** out) {
  const bool cap = capturing(st);
  if (h.stage_bytes < bytes) {
    if (cap) return COSMA_ERR_NO_WORKSPACE;
    if (h.stage) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return COSMA_ERR_CUDA;
      if (h.captured) h.retired.push_back(h.stage);  // a graph may still read it
      else cudaFree(h.stage);
      h.stage = nullptr;
      h.stage_bytes = 0;
      h.captured = false;
    }
    const size_t want = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    if (cudaMalloc(&h.stage, want) != cudaSuccess) {
      cudaGetLastError();
      return COSMA_ERR_NO_WORKSPACE;
    }
    h.stage_bytes = want;
  }
  if (cap) h.captured = true;
  *out = static_cast<uint8_t*>(h.stage);
  return COSMA_OK;
}

int in_bytes(int dtype) {
  return dtype == COSMA_F32 || dtype == COSMA_F32_EMU_TF32 ? 4 : dtype == COSMA_BF16 ? 2 : 8;
}
int out_bytes(int dtype) {
  return dtype == COSMA_F32 || dtype == COSMA_BF16 || dtype == COSMA_F32_EMU_TF32 ? 4 : 8;
}

// Block boundaries along a dimension: 1 block, or 2 split at a multiple of 256.
int blocks_of(int64_t len, int64_t cut[kMaxR + 1]) {
  const int r = len >= kSplitMin ? 2 : 1;
  cut[0] = 0;
  if (r == 2) cut[1] = rup((len + 1) / 2, 256);
  cut[r] = len;
  return r;
}

int ok(cudaError_t e) { return e == cudaSuccess ? COSMA_OK : COSMA_ERR_CUDA; }

}  // namespace

void host_release(int dev) {
  std::lock_guard<std::mutex> lock(g_host_mu);
  if (dev < 0 || dev >= kMaxDevices) return;
  HostState& h = g_host[dev];
  if (!h.ready) return;
  if (h.stage) cudaFree(h.stage);
  for (void* p : h.retired) cudaFree(p);
  for (int i = 0; i < kEvents; ++i)
    if (h.ev[i]) cudaEventDestroy(h.ev[i]);
  if (h.in) cudaStreamDestroy(h.in);
  if (h.out) cudaStreamDestroy(h.out);
  h = HostState{};
  HostPhases& p = g_phases[dev];
  if (p.ready) {
    cudaEvent_t all[3] = {p.start, p.in_done, p.end};
    for (cudaEvent_t e : all) cudaEventDestroy(e);
    for (int i = 0; i < kMaxR * kMaxR; ++i) {
      cudaEventDestroy(p.pb[i]);
      cudaEventDestroy(p.pe[i]);
    }
  }
  p = HostPhases{};
}

}  // namespace cosma

using namespace cosma;

extern "C" int cosma_gemm_host(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                               const void* B, int64_t ldb, void* C, int64_t ldc, int dtype,
                               void* stream) {
  if (dtype < COSMA_F64 || dtype > COSMA_F32_EMU_TF32) return COSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return COSMA_ERR_INVALID_ARG;
  if (lda < (k > 1 ? k : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1))
    return COSMA_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return COSMA_OK;
  if (!C || !is_host_ptr(C)) return COSMA_ERR_INVALID_ARG;
  if (k > 0 && (!A || !B || !is_host_ptr(A) || !is_host_ptr(B))) return COSMA_ERR_INVALID_ARG;
  if (dtype == COSMA_F64_EMU_INT8) return COSMA_ERR_UNSUPPORTED;
  if (k_supported(dtype, k) != COSMA_OK) return COSMA_ERR_UNSUPPORTED;

  LibContext ctx;
  int rc = lib_context(&ctx);
  if (rc != COSMA_OK) return rc;
  const int dev = ctx.info.device;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_host_mu);
  HostState& h = g_host[dev];
  rc = init_state(h);
  if (rc != COSMA_OK) return rc;

  const int ei = in_bytes(dtype), eo = out_bytes(dtype);
  const int64_t lda_d = rup(k > 0 ? k : 1, 8), ldb_d = rup(n, 8), ldc_d = rup(n, 8);
  const size_t a_bytes = (size_t)rup(m * lda_d * ei, 256);
  const size_t b_bytes = (size_t)rup((k > 0 ? k : 1) * ldb_d * ei, 256);
  const size_t c_bytes = (size_t)rup(m * ldc_d * eo, 256);
  uint8_t* base = nullptr;
  rc = staging(h, a_bytes + b_bytes + c_bytes, st, &base);
  if (rc != COSMA_OK) return rc;
  uint8_t* Ad = base;
  uint8_t* Bd = base + a_bytes;
  uint8_t* Cd = base + a_bytes + b_bytes;

  int64_t rcut[kMaxR + 1], ccut[kMaxR + 1];
  const int Rm = blocks_of(m, rcut), Rn = blocks_of(n, ccut);

  // Emulated FP64: the blocks are planned first, so that the workspace holds the
  // exact total of the largest block whose plan splits k (the blocks run one
  // after another on `stream` and share it).
  const bool emu = dtype == COSMA_F64_EMU_BF16 && k > 0;
  EmuWorkspace ew{};
  cosma_plan bplan[kMaxR * kMaxR];
  if (emu) {
    rc = emu_check_config(ctx.cfg);
    if (rc != COSMA_OK) return rc;
    int64_t split = 0;
    for (int i = 0; i < Rm; ++i)
      for (int j = 0; j < Rn; ++j) {
        const int64_t mb = rcut[i + 1] - rcut[i], nb = ccut[j + 1] - ccut[j];
        rc = plan_gemm(mb, nb, k, dtype, ctx.cfg.selector, ctx.info, ctx.cfg, &bplan[i * Rn + j],
                       !capturing(st));
        if (rc != COSMA_OK) return rc;
        if (bplan[i * Rn + j].pk > 1) split = std::max(split, mb * nb);
      }
    void* ws = nullptr;
    rc = lib_scratch(emu_workspace_bytes(m, n, k, ctx.cfg, ctx.info.sms, split), st, &ws);
    if (rc != COSMA_OK) return rc;
    ew = emu_carve(ws, m, n, k, ctx.cfg, ctx.info.sms, split);
  }
  cudaEvent_t ev_start = h.ev[0], ev_done = h.ev[1];
  cudaEvent_t* ev_a = h.ev + 2;
  cudaEvent_t* ev_b = h.ev + 2 + kMaxR;
  cudaEvent_t* ev_c = h.ev + 2 + 2 * kMaxR;

  HostPhases& ph = g_phases[dev];
  const bool prof = prof_enabled() && !capturing(st) && phases_init(ph) == COSMA_OK;
  if (prof) {
    ph.valid = false;
    if ((rc = ok(cudaEventRecord(ph.start, st))) != COSMA_OK) return rc;
  }
  // fork: the copy streams start after everything already queued on `stream`
  if ((rc = ok(cudaEventRecord(ev_start, st))) != COSMA_OK) return rc;
  if ((rc = ok(cudaStreamWaitEvent(h.in, ev_start, 0))) != COSMA_OK) return rc;
  if ((rc = ok(cudaStreamWaitEvent(h.out, ev_start, 0))) != COSMA_OK) return rc;

  // Everything between the fork and the join; on an error the streams are
  // still joined, so a capture in progress stays well formed.
  auto body = [&]() -> int {
    // copy-in, in the order compute consumes it
    auto copy_a = [&](int i) -> int {
      const int64_t r0 = rcut[i], r1 = rcut[i + 1];
      if (k > 0) {
        const cudaError_t e = cudaMemcpy2DAsync(
            Ad + (size_t)r0 * lda_d * ei, (size_t)lda_d * ei,
            static_cast<const uint8_t*>(A) + (size_t)r0 * lda * ei, (size_t)lda * ei,
            (size_t)k * ei, (size_t)(r1 - r0), cudaMemcpyHostToDevice, h.in);
        if (e != cudaSuccess) return COSMA_ERR_CUDA;
      }
      return ok(cudaEventRecord(ev_a[i], h.in));
    };
    auto copy_b = [&](int j) -> int {
      const int64_t c0 = ccut[j], c1 = ccut[j + 1];
      if (k > 0) {
        const cudaError_t e = cudaMemcpy2DAsync(
            Bd + (size_t)c0 * ei, (size_t)ldb_d * ei, static_cast<const uint8_t*>(B) + (size_t)c0 * ei,
            (size_t)ldb * ei, (size_t)(c1 - c0) * ei, (size_t)k, cudaMemcpyHostToDevice, h.in);
        if (e != cudaSuccess) return COSMA_ERR_CUDA;
      }
      return ok(cudaEventRecord(ev_b[j], h.in));
    };
    if ((rc = copy_a(0)) != COSMA_OK) return rc;
    for (int j = 0; j < Rn; ++j)
      if ((rc = copy_b(j)) != COSMA_OK) return rc;
    for (int i = 1; i < Rm; ++i)
      if ((rc = copy_a(i)) != COSMA_OK) return rc;

    // compute and copy-out, block by block
    for (int i = 0; i < Rm; ++i) {
      const int64_t r0 = rcut[i], r1 = rcut[i + 1];
      if ((rc = ok(cudaStreamWaitEvent(st, ev_a[i], 0))) != COSMA_OK) return rc;
      if (emu) {
        rc = emu_prepare_a(reinterpret_cast<const double*>(Ad) + r0 * lda_d, r1 - r0, k, lda_d,
                           0, ew.eA + r0, static_cast<uint8_t*>(ew.SA) + (size_t)r0 * ew.row_pitch * 2,
                           m, ctx.status, ctx.cfg, st);
        if (rc > 0) return COSMA_ERR_CUDA;
        if (rc < 0) return rc;
      }
      for (int j = 0; j < Rn; ++j) {
        const int64_t c0 = ccut[j], c1 = ccut[j + 1];
        const int64_t mb = r1 - r0, nb = c1 - c0;
        if (i == 0) {
          if ((rc = ok(cudaStreamWaitEvent(st, ev_b[j], 0))) != COSMA_OK) return rc;
          if (emu) {
            rc = emu_prepare_b(reinterpret_cast<const double*>(Bd) + c0, k, nb, ldb_d, 0,
                               ew.eB + c0, static_cast<uint8_t*>(ew.SB) + (size_t)c0 * ew.row_pitch * 2,
                               n, ctx.status, ctx.cfg, st);
            if (rc > 0) return COSMA_ERR_CUDA;
            if (rc < 0) return rc;
          }
        }
        uint8_t* Cblk = Cd + ((size_t)r0 * ldc_d + c0) * eo;
        if (prof && (rc = ok(cudaEventRecord(ph.pb[i * Rn + j], st))) != COSMA_OK) return rc;
        if (emu) {
          rc = emu_multiply(mb, nb, k, bplan[i * Rn + j], ctx.cfg, ew.eA + r0,
                            static_cast<uint8_t*>(ew.SA) + (size_t)r0 * ew.row_pitch * 2, m, ew.eB + c0,
                            static_cast<uint8_t*>(ew.SB) + (size_t)c0 * ew.row_pitch * 2, n,
                            reinterpret_cast<double*>(Cblk), ldc_d, 1.0, 0.0, ew.T, ew.t_bytes, ew.X,
                            ew.lockstep,
                            ctx.status, ctx.wait_limit, st);
          if (rc > 0) return COSMA_ERR_CUDA;
          if (rc < 0) return rc;
        } else {
          rc = run_device(mb, nb, k, Ad + (size_t)r0 * lda_d * ei, lda_d, Bd + (size_t)c0 * ei, ldb_d,
                          Cblk, ldc_d, dtype, st);
          if (rc != COSMA_OK) return rc;
        }
        if (prof && (rc = ok(cudaEventRecord(ph.pe[i * Rn + j], st))) != COSMA_OK) return rc;
        cudaEvent_t evc = ev_c[i * Rn + j];
        if ((rc = ok(cudaEventRecord(evc, st))) != COSMA_OK) return rc;
        if ((rc = ok(cudaStreamWaitEvent(h.out, evc, 0))) != COSMA_OK) return rc;
        const cudaError_t e = cudaMemcpy2DAsync(
            static_cast<uint8_t*>(C) + ((size_t)r0 * ldc + c0) * eo, (size_t)ldc * eo, Cblk,
            (size_t)ldc_d * eo, (size_t)nb * eo, (size_t)mb, cudaMemcpyDeviceToHost, h.out);
        if (e != cudaSuccess) return COSMA_ERR_CUDA;
      }
    }
    return COSMA_OK;
  };
  const int brc = body();
  // join: `stream` continues after the last copy-in and the last copy-out
  if (prof && brc == COSMA_OK) cudaEventRecord(ph.in_done, h.in);
  rc = ok(cudaEventRecord(ev_start, h.in));
  if (rc == COSMA_OK) rc = ok(cudaStreamWaitEvent(h.out, ev_start, 0));
  if (rc == COSMA_OK) rc = ok(cudaEventRecord(ev_done, h.out));
  if (rc == COSMA_OK) rc = ok(cudaStreamWaitEvent(st, ev_done, 0));
  if (prof && brc == COSMA_OK && rc == COSMA_OK && cudaEventRecord(ph.end, st) == cudaSuccess) {
    ph.nblocks = Rm * Rn;
    ph.valid = true;
  }
  return brc != COSMA_OK ? brc : rc;
}

extern "C" int cosma_profile_host(double* phases, int count) {
  if (!phases || count < 1) return COSMA_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return COSMA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_host_mu);
  const HostPhases& p = g_phases[dev];
  if (!p.valid) return COSMA_ERR_INVALID_ARG;
  if (cudaEventSynchronize(p.end) != cudaSuccess) return COSMA_ERR_CUDA;
  auto span = [](cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : -1.0;
  };
  double products = 0.0;
  for (int i = 0; i < p.nblocks; ++i) products += span(p.pb[i], p.pe[i]);
  const double v[6] = {span(p.start, p.end), span(p.start, p.pb[0]), products,
                       span(p.pe[p.nblocks - 1], p.end), span(p.start, p.in_done),
                       (double)p.nblocks};
  const int n = count < 6 ? count : 6;
  for (int i = 0; i < n; ++i) phases[i] = v[i];
  return n;
}
