// Host runtime behind include/cosma.h: argument checks, plans, workspace,
// dispatch to the kernels, device status word.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cosma {

int launch_tc_bf16(const GemmArgs& g, const Sched& s, const cosma_plan& p, void* ws,
                   long long ws_bytes, int* status, long long wait_limit, cudaStream_t st);
long long tc_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_plan& p, const void* A,
                             int64_t lda, int trans_a, const void* B, int64_t ldb, int trans_b);
long long tf32x3_workspace_bytes(int64_t m, int64_t n, int64_t k, const cosma_plan& p);
int launch_tc_tf32x3(const GemmArgs& g, const Sched& s, const cosma_plan& p, void* ws,
                     long long ws_bytes, int* status, long long wait_limit, cudaStream_t st);
int grouped_gemm(int count, const cosma_problem* problems, int dtype, const DeviceInfo& dev,
                 void* ws, long long ws_bytes, int* status, long long wait_limit, cudaStream_t st,
                 long long* needed, int requested_tile);
void grouped_release(int dev);
void host_release(int dev);
void complex_release(int dev);

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<cudaEvent_t> g_prof_ev;  // start, stop, start, stop, ...
static size_t g_prof_used = 0;

bool prof_enabled() {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  return g_prof_on;
}

void prof_mark(cudaStream_t st, bool begin) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (!g_prof_on) return;
  if (begin && (g_prof_used & 1)) return;   // unmatched begin: ignore
  if (!begin && !(g_prof_used & 1)) return;
  if (g_prof_used == g_prof_ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
    g_prof_ev.push_back(e);
  }
  cudaEventRecord(g_prof_ev[g_prof_used++], st);
}

namespace {

// One library-owned workspace per stream, so that calls on different streams
// never share scratch memory; beyond kArenas streams the least recently used
// arena is given to the new stream (cudaFree waits for the device first).
// A buffer that a stream capture recorded is never freed before
// cosma_finalize: the graph may be replayed after the arena has grown or
// changed hands, so such a buffer is retired instead.
constexpr int kArenas = 8;
struct Arena {
  cudaStream_t stream = nullptr;
  void* ptr = nullptr;
  size_t bytes = 0;
  unsigned long long last_use = 0;
  bool used = false;
  bool captured = false;       // ptr is recorded in a captured graph
};

struct DeviceState {
  bool ready = false;
  DeviceInfo info;
  int* d_status = nullptr;     // device status word (0 = ok)
  Arena arenas[kArenas];       // library-owned workspaces, one per stream
  unsigned long long uses = 0;
  void* borrowed = nullptr;    // caller-lent workspace (all streams)
  size_t borrowed_bytes = 0;
  std::vector<void*> retired;  // captured buffers an arena gave up; freed at finalize
};

constexpr int kMaxDevices = 16;
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
bool config_valid(const cosma_config& c) {
  if (!(c.delta >= 0.0 && c.delta < 1.0)) return false;
  if (c.selector < COSMA_SELECT_ANALYTIC || c.selector > COSMA_SELECT_LEARNED) return false;
  if (c.emu_slices < 0 || c.emu_slices > 12) return false;
  if (c.emu_slice_bits < 0 || c.emu_slice_bits > 8) return false;
  if (c.wait_limit < 0) return false;
  if (c.grouped_tile != 0 && c.grouped_tile != 64 && c.grouped_tile != 128 &&
      c.grouped_tile != 256 && c.grouped_tile != 512)
    return false;
  return true;
}

// Defaults, then COSMA_* environment variables (read once, when the library is
// loaded); a malformed or out-of-range value leaves its field at the default.
cosma_config env_config() {
  cosma_config c = {0.03, COSMA_SELECT_ANALYTIC, 0, 0, 0, 0};
  auto num = [](const char* name, double* out) {
    const char* v = getenv(name);
    if (!v || !*v) return false;
    char* end = nullptr;
    const double x = strtod(v, &end);
    if (!end || *end) return false;
    *out = x;
    return true;
  };
  auto apply = [&c](const cosma_config& trial) {
    if (config_valid(trial)) c = trial;
  };
  double x;
  cosma_config t;
  if (num("COSMA_DELTA", &x)) { t = c; t.delta = x; apply(t); }
  if (const char* v = getenv("COSMA_SELECTOR")) {
    t = c;
    if (!strcmp(v, "analytic") || !strcmp(v, "0")) t.selector = COSMA_SELECT_ANALYTIC;
    else if (!strcmp(v, "learned") || !strcmp(v, "1")) t.selector = COSMA_SELECT_LEARNED;
    else t.selector = -1;
    apply(t);
  }
  if (num("COSMA_EMU_SLICES", &x) && x == (int)x) { t = c; t.emu_slices = (int)x; apply(t); }
  if (num("COSMA_EMU_SLICE_BITS", &x) && x == (int)x) { t = c; t.emu_slice_bits = (int)x; apply(t); }
  if (num("COSMA_WAIT_LIMIT", &x) && x == (long long)x) { t = c; t.wait_limit = (long long)x; apply(t); }
  if (num("COSMA_GROUPED_TILE", &x) && x == (int)x) { t = c; t.grouped_tile = (int)x; apply(t); }
  return c;
}

cosma_config g_cfg = env_config();

const long long kDefaultWaitLimit = 1LL << 31;  // clock cycles (~1 s) before a device wait gives up

int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}

// Returns the state of the current device, initialising it once (outside any
// stream capture: it allocates the status word).
DeviceState* state(int* err) {
  const int d = current_device();
  if (d < 0) { *err = COSMA_ERR_CUDA; return nullptr; }
  DeviceState& s = g_dev[d];
  if (!s.ready) {
    DeviceInfo& in = s.info;
    in.device = d;
    if (cudaDeviceGetAttribute(&in.sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
      *err = COSMA_ERR_CUDA;
      return nullptr;
    }
    cudaDeviceGetAttribute(&in.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    cudaDeviceGetAttribute(&in.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
    cudaDeviceGetAttribute(&in.regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, d);
    cudaDeviceGetAttribute(&in.l2_bytes, cudaDevAttrL2CacheSize, d);
    cudaDeviceGetAttribute(&in.cc_major, cudaDevAttrComputeCapabilityMajor, d);
    cudaDeviceGetAttribute(&in.cc_minor, cudaDevAttrComputeCapabilityMinor, d);
    if (cudaMalloc(&s.d_status, 256) != cudaSuccess) { *err = COSMA_ERR_CUDA; return nullptr; }
    if (cudaMemset(s.d_status, 0, 256) != cudaSuccess) { *err = COSMA_ERR_CUDA; return nullptr; }
    s.ready = true;
  }
  *err = COSMA_OK;
  return &s;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

// Gives up an arena's buffer: freed (cudaFree waits for the device), or kept
// until cosma_finalize when a captured graph holds its address.
void drop_buffer(DeviceState* s, Arena* a) {
  if (a->ptr) {
    if (a->captured) s->retired.push_back(a->ptr);
    else cudaFree(a->ptr);
  }
  a->ptr = nullptr;
  a->bytes = 0;
  a->captured = false;
}

// Workspace of at least `bytes`: the caller's lent buffer, else the arena
// (grown outside capture only).
int workspace(DeviceState* s, long long bytes, cudaStream_t st, void** out, long long* have) {
  *out = nullptr;
  *have = 0;
  if (bytes <= 0) return COSMA_OK;
  if (s->borrowed) {
    if ((long long)s->borrowed_bytes < bytes) return COSMA_ERR_NO_WORKSPACE;
    *out = s->borrowed;
    *have = (long long)s->borrowed_bytes;
    return COSMA_OK;
  }
  // this stream's arena, else a free slot, else the least recently used one
  Arena* a = nullptr;
  for (Arena& x : s->arenas)
    if (x.used && x.stream == st) a = &x;
  const bool cap = capturing(st);
  if (cap && (!a || (long long)a->bytes < bytes)) {
    // Capture cannot allocate: the usual pattern sizes an arena with an eager
    // call on another stream just before, so a capture takes the most recently
    // used arena that is big enough -- the one that call used, whose pointer
    // also keys the grouped tables (the graph then shares it with that stream).
    Arena* big = nullptr;
    for (Arena& x : s->arenas)
      if (x.used && (long long)x.bytes >= bytes && (!big || x.last_use > big->last_use)) big = &x;
    if (!big) return COSMA_ERR_NO_WORKSPACE;
    big->last_use = ++s->uses;
    big->captured = true;
    *out = big->ptr;
    *have = (long long)big->bytes;
    return COSMA_OK;
  }
  if (!a) {
    for (Arena& x : s->arenas)
      if (!x.used) { a = &x; break; }
    if (!a) {
      a = &s->arenas[0];
      for (Arena& x : s->arenas)
        if (x.last_use < a->last_use) a = &x;
      drop_buffer(s, a);
      *a = Arena{};
    }
    a->used = true;
    a->stream = st;
  }
  a->last_use = ++s->uses;
  if ((long long)a->bytes < bytes) {  // not capturing here
    if (a->ptr) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return COSMA_ERR_CUDA;
      drop_buffer(s, a);
    }
    size_t want = (size_t)bytes;
    want = (want + (1u << 20) - 1) & ~((size_t)(1u << 20) - 1);
    if (cudaMalloc(&a->ptr, want) != cudaSuccess) {
      cudaGetLastError();
      return COSMA_ERR_NO_WORKSPACE;
    }
    a->bytes = want;
  }
  if (cap) a->captured = true;
  *out = a->ptr;
  *have = (long long)a->bytes;
  return COSMA_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int elem_bytes_in(int dtype) {
  switch (dtype) {
    case COSMA_F32:
    case COSMA_F32_EMU_TF32: return 4;
    case COSMA_BF16: return 2;
    default: return 8;
  }
}
int elem_bytes_out(int dtype) {
  return dtype == COSMA_F32 || dtype == COSMA_BF16 || dtype == COSMA_F32_EMU_TF32 ? 4 : 8;
}

}  // namespace

constexpr int64_t kTf32MaxK = 65535LL * 32;

// Three-TF32 parts are written by grids with one y row per 32-deep k block; the
// bf16 slices likewise, per 32 columns of k padded to 2048-deep panels.  Every
// entry point refuses a longer k before it sizes or allocates anything.
int k_supported(int dtype, int64_t k) {
  if (dtype == COSMA_F32_EMU_TF32 && k > kTf32MaxK) return COSMA_ERR_UNSUPPORTED;
  if (dtype == COSMA_F64_EMU_BF16 && (emu_padded_k(k) + 31) / 32 > 65535)
    return COSMA_ERR_UNSUPPORTED;
  return COSMA_OK;
}

namespace {

int check_args(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
               int64_t ldb, const void* C, int64_t ldc, int dtype, int ta = 0, int tb = 0) {
  if (dtype < COSMA_F64 || dtype > COSMA_F32_EMU_TF32) return COSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return COSMA_ERR_INVALID_ARG;
  if ((ta != 0 && ta != 1) || (tb != 0 && tb != 1)) return COSMA_ERR_INVALID_ARG;
  const int64_t a_cols = ta ? m : k, b_cols = tb ? k : n;
  if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) || ldc < (n > 1 ? n : 1))
    return COSMA_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return COSMA_OK;
  if (k_supported(dtype, k) != COSMA_OK) return COSMA_ERR_UNSUPPORTED;
  if (!C) return COSMA_ERR_INVALID_ARG;
  if (k > 0 && (!A || !B)) return COSMA_ERR_INVALID_ARG;
  if ((uintptr_t)C % elem_bytes_out(dtype)) return COSMA_ERR_INVALID_ARG;
  if (k > 0 && ((uintptr_t)A % elem_bytes_in(dtype) || (uintptr_t)B % elem_bytes_in(dtype)))
    return COSMA_ERR_INVALID_ARG;
  if (!is_device_ptr(C)) return COSMA_ERR_INVALID_ARG;
  if (k > 0 && (!is_device_ptr(A) || !is_device_ptr(B))) return COSMA_ERR_INVALID_ARG;
  if (dtype == COSMA_F64_EMU_INT8) return COSMA_ERR_UNSUPPORTED;
  return COSMA_OK;
}

// Workspace of a plan; without operand pointers, the most any operands need.
long long total_workspace(int64_t m, int64_t n, int64_t k, int dtype, const cosma_plan& p,
                          const void* A = nullptr, int64_t lda = 0, const void* B = nullptr,
                          int64_t ldb = 0, int ta = 0, int tb = 0) {
  if (dtype == COSMA_F64_EMU_BF16)
    return emu_workspace_bytes(m, n, k, g_cfg, p.sms, p.pk > 1 ? m * n : 0);
  if (dtype == COSMA_BF16) return tc_workspace_bytes(m, n, k, p, A, lda, ta, B, ldb, tb);
  if (dtype == COSMA_F32_EMU_TF32) return tf32x3_workspace_bytes(m, n, k, p);
  // FMA paths: split-k partials, then untransposed copies of transposed operands
  const int w = dtype == COSMA_F32 ? 4 : 8;
  long long b = workspace_bytes(m, n, k, dtype, p);
  if (ta) b += (m * k * w + 255) / 256 * 256;
  if (tb) b += (k * n * w + 255) / 256 * 256;
  return b;
}

// C = alpha op(A) op(B) + beta C (op: transposed storage when ta / tb is 1).
int run(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B, int64_t ldb,
        void* C, int64_t ldc, int dtype, const cosma_plan* given, void* stream,
        double alpha = 1.0, double beta = 0.0, int ta = 0, int tb = 0) {
  const bool no_ab = k == 0 || alpha == 0.0;  // A and B are not read
  int rc = check_args(m, n, no_ab ? 0 : k, no_ab ? nullptr : A, lda, no_ab ? nullptr : B, ldb, C,
                      ldc, dtype, ta, tb);
  if (rc == COSMA_OK && no_ab) {  // the leading dimensions still have to be valid
    const int64_t a_cols = ta ? m : k, b_cols = tb ? k : n;
    if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1))
      rc = COSMA_ERR_INVALID_ARG;
  }
  if (rc != COSMA_OK) return rc;
  if (m == 0 || n == 0) return COSMA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState* s = state(&rc);
  if (!s) return rc;
  if (no_ab) {  // C = beta C
    GemmArgs gs{m, n, k, A, lda, B, ldb, C, ldc};
    gs.beta = beta;
    if (beta == 0.0) {
      const size_t w = (size_t)elem_bytes_out(dtype);
      count_launch();
      return cudaMemset2DAsync(C, (size_t)ldc * w, 0, (size_t)n * w, (size_t)m, st) ==
                     cudaSuccess
                 ? COSMA_OK
                 : COSMA_ERR_CUDA;
    }
    if (beta == 1.0) return COSMA_OK;
    return launch_scale(dtype, gs, st) == 0 ? COSMA_OK : COSMA_ERR_CUDA;
  }
  cosma_plan p;
  if (given) {
    p = *given;
    rc = validate_plan(m, n, k, dtype, s->info, p);
    if (rc != COSMA_OK) return rc;
  } else {
    rc = plan_gemm(m, n, k, dtype, g_cfg.selector, s->info, g_cfg, &p, !capturing(st));
    if (rc != COSMA_OK) return rc;
  }
  const long long need = total_workspace(m, n, k, dtype, p, A, lda, B, ldb, ta, tb);
  void* ws = nullptr;
  long long have = 0;
  rc = workspace(s, need, st, &ws, &have);
  if (rc != COSMA_OK) return rc;
  GemmArgs g{m, n, k, A, lda, B, ldb, C, ldc};
  g.alpha = alpha;
  g.beta = beta;
  g.trans_a = ta;
  g.trans_b = tb;
  const Sched sc = sched_from_plan(m, n, k, p);
  const long long wl = g_cfg.wait_limit > 0 ? g_cfg.wait_limit : kDefaultWaitLimit;
  int err = 0;
  switch (p.kernel) {
    case COSMA_KERNEL_SIMT_F64:
    case COSMA_KERNEL_SIMT_F32: {
      // Transposed operands are first copied untransposed after the partials.
      const int w = dtype == COSMA_F32 ? 4 : 8;
      uint8_t* extra = static_cast<uint8_t*>(ws) + workspace_bytes(m, n, k, dtype, p);
      if (ta) {
        err = launch_transpose(w, A, k, m, lda, extra, k, st);
        g.A = extra;
        g.lda = k;
        g.trans_a = 0;
        extra += (m * k * w + 255) / 256 * 256;
      }
      if (!err && tb) {
        err = launch_transpose(w, B, n, k, ldb, extra, n, st);
        g.B = extra;
        g.ldb = n;
        g.trans_b = 0;
      }
      if (!err) err = launch_simt(dtype, g, sc, ws, s->d_status, st);
      if (!err && p.pk > 1) err = launch_reduce(dtype, g, p.pk, ws, st);
      break;
    }
    case COSMA_KERNEL_TC_BF16:
      err = launch_tc_bf16(g, sc, p, ws, have, s->d_status, wl, st);
      break;
    case COSMA_KERNEL_EMU_BF16:
      err = launch_emu_bf16(g, p, g_cfg, ws, have, s->d_status, wl, st);
      break;
    case COSMA_KERNEL_TF32X3:
      err = launch_tc_tf32x3(g, sc, p, ws, have, s->d_status, wl, st);
      break;
    default:
      return COSMA_ERR_INVALID_ARG;
  }
  if (err < 0) return err;  // a cosma_status from a launcher
  return err == 0 ? COSMA_OK : COSMA_ERR_CUDA;
}

}  // namespace

int lib_scratch(long long bytes, cudaStream_t st, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  long long have = 0;
  return workspace(s, bytes, st, out, &have);
}

int current_info(DeviceInfo* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  *out = s->info;
  return COSMA_OK;
}

int lib_context(LibContext* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  out->info = s->info;
  out->cfg = g_cfg;
  out->status = s->d_status;
  out->wait_limit = g_cfg.wait_limit > 0 ? g_cfg.wait_limit : kDefaultWaitLimit;
  return COSMA_OK;
}

int run_device(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
               int64_t ldb, void* C, int64_t ldc, int dtype, void* stream) {
  return run(m, n, k, A, lda, B, ldb, C, ldc, dtype, nullptr, stream);
}

int run_device_ex(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
                  int64_t ldb, void* C, int64_t ldc, int dtype, double alpha, double beta,
                  int trans_a, int trans_b, void* stream) {
  return run(m, n, k, A, lda, B, ldb, C, ldc, dtype, nullptr, stream, alpha, beta, trans_a,
             trans_b);
}

}  // namespace cosma

using namespace cosma;

extern "C" {

int cosma_init(const cosma_config* cfg) {
  if (cfg && !config_valid(*cfg)) return COSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cfg) g_cfg = *cfg;
  int rc;
  return state(&rc) ? COSMA_OK : rc;
}

int cosma_get_config(cosma_config* out) {
  if (!out) return COSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  *out = g_cfg;
  return COSMA_OK;
}

int cosma_set_workspace(void* dptr, size_t bytes) {
  if (bytes > 0 && (!dptr || (uintptr_t)dptr % 256)) return COSMA_ERR_INVALID_ARG;
  if (bytes > 0 && !is_device_ptr(dptr)) return COSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  s->borrowed = bytes > 0 ? dptr : nullptr;
  s->borrowed_bytes = bytes;
  return COSMA_OK;
}

void cosma_finalize(void) {
  const int d = current_device();
  if (d < 0) return;
  host_release(d);  // these take their own locks, never while holding g_mu
  complex_release(d);
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& s = g_dev[d];
  if (!s.ready) return;
  cudaDeviceSynchronize();
  grouped_release(d);
  for (Arena& x : s.arenas)
    if (x.ptr) cudaFree(x.ptr);
  for (void* p : s.retired) cudaFree(p);
  if (s.d_status) cudaFree(s.d_status);
  s = DeviceState{};
}

int cosma_gemm(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
               int64_t ldb, void* C, int64_t ldc, int dtype, void* stream) {
  return run(m, n, k, A, lda, B, ldb, C, ldc, dtype, nullptr, stream);
}

int cosma_gemm_ex(int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                  const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                  int64_t ldc, int dtype, void* stream) {
  return run(m, n, k, A, lda, B, ldb, C, ldc, dtype, nullptr, stream, alpha, beta, trans_a,
             trans_b);
}

int cosma_gemm_planned(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                       const void* B, int64_t ldb, void* C, int64_t ldc, int dtype,
                       const cosma_plan* plan, void* stream) {
  if (!plan) return COSMA_ERR_INVALID_ARG;
  return run(m, n, k, A, lda, B, ldb, C, ldc, dtype, plan, stream);
}

int cosma_gemm_grouped(int count, const cosma_problem* problems, int dtype, void* stream) {
  if (count < 0 || (count > 0 && !problems)) return COSMA_ERR_INVALID_ARG;
  if (dtype != COSMA_F32 && dtype != COSMA_BF16) return COSMA_ERR_UNSUPPORTED;
  if (count == 0) return COSMA_OK;
  for (int i = 0; i < count; ++i) {
    const cosma_problem& q = problems[i];
    const int rc = check_args(q.m, q.n, q.k, q.A, q.lda, q.B, q.ldb, q.C, q.ldc, dtype);
    if (rc != COSMA_OK) return rc;
    // a work-unit record keeps the k-block count in 30 bits and tile indices in int
    if (q.k >= (1LL << 35) || q.m >= (1LL << 38) || q.n >= (1LL << 38))
      return COSMA_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  long long need = 0;
  rc = grouped_gemm(count, problems, dtype, s->info, nullptr, 0, s->d_status, 0, st, &need,
                    g_cfg.grouped_tile);
  if (rc != COSMA_OK) return rc;
  void* ws = nullptr;
  long long have = 0;
  rc = workspace(s, need, st, &ws, &have);
  if (rc != COSMA_OK) return rc;
  // Problems with k == 0 get C = 0; empty ones need nothing.
  const size_t w = (size_t)elem_bytes_out(dtype);
  for (int i = 0; i < count; ++i) {
    const cosma_problem& q = problems[i];
    if (q.m > 0 && q.n > 0 && q.k == 0) {
      if (cudaMemset2DAsync(q.C, (size_t)q.ldc * w, 0, (size_t)q.n * w, (size_t)q.m, st) !=
          cudaSuccess)
        return COSMA_ERR_CUDA;
    }
  }
  const long long wl = g_cfg.wait_limit > 0 ? g_cfg.wait_limit : kDefaultWaitLimit;
  rc = grouped_gemm(count, problems, dtype, s->info, ws, have, s->d_status, wl, st, nullptr,
                    g_cfg.grouped_tile);
  if (rc < 0) return rc;
  return rc == 0 ? COSMA_OK : COSMA_ERR_CUDA;
}

int cosma_plan_query(int64_t m, int64_t n, int64_t k, int dtype, int selector, cosma_plan* out) {
  if (!out) return COSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return COSMA_ERR_INVALID_ARG;
  if (selector < COSMA_SELECT_ANALYTIC || selector > COSMA_SELECT_LEARNED) return COSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceInfo info;
  int rc;
  DeviceState* s = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) s = state(&rc);
  else cudaGetLastError();
  if (s) info = s->info;
  else info.sms = 148;  // planning without a device (host-only tests)
  rc = plan_gemm(m, n, k, dtype, selector, info, g_cfg, out);
  if (rc == COSMA_OK) out->workspace_bytes = total_workspace(m, n, k, dtype, *out);
  return rc;
}

long long cosma_plan_units(int64_t m, int64_t n, int64_t k, const cosma_plan* plan,
                           int64_t* units, long long max_units) {
  if (!plan || m < 1 || n < 1 || k < 1 || max_units < 0 || (max_units > 0 && !units))
    return COSMA_ERR_INVALID_ARG;
  if (plan->tile_m < 1 || plan->tile_n < 1 || plan->k_block < 1 || plan->pk < 1 ||
      plan->ctas < 1 || plan->order < 0 || plan->order > 1)
    return COSMA_ERR_INVALID_ARG;
  if (plan->order == 0 && (long long)plan->pm * plan->pn * plan->pk != plan->ctas)
    return COSMA_ERR_INVALID_ARG;
  const Sched s = sched_from_plan(m, n, k, *plan);
  long long total = 0;
  for (int c = 0; c < s.ctas; ++c) {
    const int64_t nu = units_of_cta(s, c);
    for (int64_t i = 0; i < nu; ++i, ++total) {
      if (total >= max_units) continue;
      const Unit u = plan->kernel == COSMA_KERNEL_EMU_BF16 ? emu_unit_of_cta(s, c, i)
                                                          : unit_of_cta(s, c, i);
      int64_t* o = units + 6 * total;
      o[0] = u.tile_row * s.tile_m;
      o[1] = (u.tile_row + 1) * s.tile_m < m ? (u.tile_row + 1) * s.tile_m : m;
      o[2] = u.tile_col * s.tile_n;
      o[3] = (u.tile_col + 1) * s.tile_n < n ? (u.tile_col + 1) * s.tile_n : n;
      o[4] = u.kb0 * s.k_block;
      o[5] = u.kb1 * s.k_block < k ? u.kb1 * s.k_block : k;
    }
  }
  return total;
}

int cosma_stream_status(void* stream) {
  std::lock_guard<std::mutex> lock(g_mu);
  int rc;
  DeviceState* s = state(&rc);
  if (!s) return rc;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return COSMA_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, s->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return COSMA_ERR_CUDA;
  if (h != 0 && cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) return COSMA_ERR_CUDA;
  return h;
}

const char* cosma_status_string(int status) {
  switch (status) {
    case COSMA_OK: return "ok";
    case COSMA_ERR_INVALID_ARG: return "invalid argument";
    case COSMA_ERR_UNSUPPORTED: return "unsupported";
    case COSMA_ERR_CUDA: return "CUDA error";
    case COSMA_ERR_TIMEOUT: return "device wait timed out";
    case COSMA_ERR_NONFINITE: return "non-finite input to the emulated path";
    case COSMA_ERR_NO_WORKSPACE: return "no workspace";
  }
  return "unknown status";
}

long long cosma_launch_count(void) { return g_launches.load(); }

int cosma_profile_enable(int on) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_prof_on = on != 0;
  return COSMA_OK;
}

int cosma_profile_read(double* main_kernel_ms, long long* launches) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  double total = 0.0;
  long long n = 0;
  int rc = COSMA_OK;
  for (size_t i = 0; i + 1 < g_prof_used; i += 2) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_prof_ev[i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, g_prof_ev[i], g_prof_ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      rc = COSMA_ERR_CUDA;
      continue;
    }
    total += ms;
    ++n;
  }
  g_prof_used = 0;
  if (main_kernel_ms) *main_kernel_ms = total;
  if (launches) *launches = n;
  return rc;
}

int cosma_device_sms(void) {
  int d = -1, sms = 0;
  if (cudaGetDevice(&d) != cudaSuccess) { cudaGetLastError(); return 0; }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

}  // extern "C"
