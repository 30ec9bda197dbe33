/*
 * cosma.h -- C ABI of a single-GPU, I/O-aware matrix-multiplication library
 * for NVIDIA GB300 (sm_103a), after Kwasniewski et al., "Red-Blue Pebbling
 * Revisited: Near Optimal Parallel Matrix-Matrix Multiplication" (SC'19,
 * arXiv 1908.09606).
 *
 * The operation is classical C = A B (no Strassen), A m x k, B k x n, C m x n
 * (Sec. 2.4), computed under the paper's schedule (Alg. 1) mapped onto one GPU:
 * the SMs are the processors, one SM's shared memory + tensor memory (or
 * register file) is the fast memory S, and L2/HBM traffic is the I/O.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major; lda, ldb, ldc are leading dimensions in elements
 *     (lda >= k, ldb >= n, ldc >= n).  C is overwritten (no alpha/beta).
 *   - A, B, C are DEVICE pointers owned by the caller.  The library never
 *     frees or retains them beyond the call's kernels.
 *   - m, n, k >= 0.  m == 0 or n == 0: no-op.  k == 0: C is set to zero.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on it.  Argument errors are returned before any
 *     launch; launch failures return COSMA_ERR_CUDA; device-side conditions
 *     (a bounded wait that gave up, non-finite input to the emulated path) are
 *     recorded in a per-device status word read by cosma_stream_status().
 *   - There is no CPU fallback: without a usable GPU every compute entry point
 *     returns COSMA_ERR_CUDA.
 *   - Calls on one stream are ordered.  Calls on different streams may run
 *     concurrently: the library keeps one workspace per stream (up to 8 per
 *     device; a ninth stream takes the least recently used one, after the
 *     device has finished with it).  A workspace lent with cosma_set_workspace
 *     serves every stream, so calls using it must not overlap; inside a stream
 *     capture a stream without a large enough workspace of its own records the
 *     most recently used one that is large enough (size it with an eager call
 *     just before capturing).  cosma_gemm_host, cosma_zgemm / cosma_cgemm and
 *     cosma_gemm_grouped also keep per-device staging or tables: their calls
 *     must not overlap across streams.  A workspace, staging buffer or grouped
 *     table that a capture recorded is never freed or overwritten before
 *     cosma_finalize (a later call that needs more takes a new buffer), so a
 *     graph stays valid until then; replays share those buffers with the
 *     calls that use them and must not overlap with them.
 */
#ifndef COSMA_GB300_H
#define COSMA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COSMA_ABI_VERSION 1

/* Element types of a call.  BF16: A and B are bf16, C is fp32.
 * F64_EMU_BF16: A, B, C are fp64; the product is formed from bf16 slices on
 * the tensor cores (Ozaki-style splitting) and recombined in high precision;
 * k <= 2^21 - 2048 (1023 slice panels of 2048; else COSMA_ERR_UNSUPPORTED
 * before any launch or allocation).
 * F64_EMU_INT8 returns COSMA_ERR_UNSUPPORTED: the INT8-slice variant of the
 * emulation has no fast path on this GPU (sm_103a) -- the tensor-core MMA has
 * no integer kind there (ptxas rejects tcgen05.mma .kind::i8 for sm_103a), and
 * the legacy mma.sync s8 path measured 151 TOPS on one GB300 against 2300
 * TFLOP/s of 256-wide bf16 tcgen05 MMAs (6.6 %), far below the bf16 slices.
 * F32_EMU_TF32: A, B, C are fp32; each operand is split into TF32 hi and lo
 * parts and C = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in fp32 on the
 * tensor cores, 64-deep k segments summed in fp32 round to nearest (elementwise
 * error within (1.002 gamma_3k(2^-23) + 3.01 2^-22) |A||B|); k <= 2^21 - 32
 * (65535 k blocks of 32; else COSMA_ERR_UNSUPPORTED before any launch or
 * allocation); Inf / NaN inputs give non-finite entries where an
 * IEEE product does, possibly NaN for Inf. */
typedef enum {
  COSMA_F64 = 0,
  COSMA_F32 = 1,
  COSMA_BF16 = 2,
  COSMA_F64_EMU_BF16 = 3,
  COSMA_F64_EMU_INT8 = 4,
  COSMA_F32_EMU_TF32 = 5
} cosma_dtype;

typedef enum {
  COSMA_OK = 0,
  COSMA_ERR_INVALID_ARG = -1,
  COSMA_ERR_UNSUPPORTED = -2,
  COSMA_ERR_CUDA = -3,
  COSMA_ERR_TIMEOUT = -4,
  COSMA_ERR_NONFINITE = -5,
  COSMA_ERR_NO_WORKSPACE = -6
} cosma_status;

/* How a plan is chosen.  ANALYTIC: the paper's FindSeqSchedule + FitRanks
 * (Alg. 1) with the library's cost model.  LEARNED: the MLP cost model, with
 * ANALYTIC as the fallback outside its training range. */
typedef enum {
  COSMA_SELECT_ANALYTIC = 0,
  COSMA_SELECT_LEARNED = 1
} cosma_selector;

/* Kernel families a plan can name. */
typedef enum {
  COSMA_KERNEL_SIMT_F64 = 0,  /* FP64 FMA, C tile in registers          */
  COSMA_KERNEL_SIMT_F32 = 1,  /* FP32 FMA, C tile in registers          */
  COSMA_KERNEL_TC_BF16 = 2,   /* tcgen05 kind::f16, C tile in TMEM       */
  COSMA_KERNEL_EMU_BF16 = 3,  /* tcgen05 bf16 slices, FP64 recombination */
  COSMA_KERNEL_TF32X3 = 4     /* tcgen05 kind::tf32, three part products   */
} cosma_kernel;

/* Library configuration (all fields have defaults; see cosma_init).  The
 * defaults can be changed by environment variables read once when the library
 * is loaded -- COSMA_DELTA, COSMA_SELECTOR (analytic | learned), COSMA_EMU_SLICES,
 * COSMA_EMU_SLICE_BITS, COSMA_WAIT_LIMIT, COSMA_GROUPED_TILE -- a malformed or
 * out-of-range value leaving its field at the built-in default; cosma_init
 * replaces the whole configuration. */
typedef struct cosma_config {
  double delta;        /* FitRanks: max fraction of SMs left idle (Sec. 7.1); default 0.03 */
  int selector;        /* default cosma_selector for cosma_gemm; default ANALYTIC */
  int emu_slices;      /* slices per operand for F64_EMU_BF16; 0 = default (6) */
  int emu_slice_bits;  /* digit width beta in bits, 2..8; 0 = default (8) */
  long long wait_limit;/* clock cycles before a device wait gives up; 0 = default (2^31, ~1 s) */
  int grouped_tile;    /* C tile width of cosma_gemm_grouped: 0 = chosen by the library;
                          bf16: 128 or 256 (tile 128 x N), or 512 (256 x 256 tiles on
                          CTA pairs); f32: 64 or 128 (square tile) */
} cosma_config;

/* A schedule for one product: the outcome of Alg. 1's FindSeqSchedule
 * (tile_m x tile_n C tile and k_block x stages input ring that fit in S),
 * ParallelizeSched/FitRanks (processor grid pm x pn x pk over the SMs; pk > 1
 * is a split of k followed by the Reduce step), and the assignment order.
 * COSMA_KERNEL_EMU_BF16 plans use order 1 and cut k at multiples of 4096 (the
 * kernels' super-chunk), so 1 <= pk <= ceil(k / 4096); their k slices sum the
 * same exact integers as an unsplit product, and C is bit-for-bit the same. */
typedef struct cosma_plan {
  int kernel;          /* cosma_kernel */
  int tile_m, tile_n;  /* C tile held in fast memory (the paper's a x b)  */
  int k_block;         /* k extent of one staged A/B panel pair           */
  int stages;          /* panel pairs in flight (Alg. 1 step size s = k_block*stages) */
  int pm, pn, pk;      /* processor grid over tiles/k (Sec. 6.1)          */
  int order;           /* 0: rectangular local domains, 1: balanced stripes of tiles */
  int ctas;            /* CTAs launched                                   */
  int sms;             /* SMs on the device                               */
  long long workspace_bytes;  /* device workspace the call needs          */
  double fast_words;   /* S: fast-memory words per SM for this kernel     */
  double io_words;     /* L2->SM words the schedule moves (loads + stores) */
  double bound_words;  /* Theorem 1 at S: 2mnk/sqrt(S) + mn               */
  double est_seconds;  /* cost-model estimate                             */
} cosma_plan;

/* One problem of a grouped call (all DEVICE pointers, same conventions as
 * cosma_gemm). */
typedef struct cosma_problem {
  int64_t m, n, k;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
} cosma_problem;

/* ---- lifecycle -------------------------------------------------------- */

/* Optional.  Applies cfg (NULL = defaults) and queries the current device.
 * Returns COSMA_ERR_INVALID_ARG for out-of-range fields. */
int cosma_init(const cosma_config* cfg);

/* Copies the active configuration to *out. */
int cosma_get_config(cosma_config* out);

/* Lends the library a caller-owned device buffer as workspace (split-k
 * partials, emulation slices, grouped tables).  The caller keeps ownership and
 * must keep it alive while calls that use it are in flight.  There is no
 * stream argument: one lent buffer serves calls on every stream, so calls that
 * use it must be ordered (one stream, or events between streams).  bytes == 0
 * returns to the library-owned arena, which grows with cudaMalloc outside
 * stream capture; inside capture a call that needs more than is available
 * returns COSMA_ERR_NO_WORKSPACE.  dptr must be 256-byte aligned. */
int cosma_set_workspace(void* dptr, size_t bytes);

/* Releases the library arena and cached state for the current device. */
void cosma_finalize(void);

/* ---- the product ------------------------------------------------------ */

/* C = A B for one problem (Alg. 1 end to end: plan, staged main loop, Reduce).
 * dtype is a cosma_dtype.  Returns cosma_status. */
int cosma_gemm(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
               int64_t ldb, void* C, int64_t ldc, int dtype, void* stream);

/* C = alpha op(A) op(B) + beta C: the BLAS / ScaLAPACK GEMM surface over the same
 * schedule (the paper's integration target; op only changes how a panel is read,
 * alpha and beta only the epilogue and the Reduce).
 *   trans_a = 0: A is m x k row-major (lda >= k); 1: A holds op(A)^T, k x m
 *   row-major (lda >= m).  trans_b = 0: B is k x n (ldb >= n); 1: B holds
 *   op(B)^T, n x k (ldb >= k).  C is m x n row-major (ldc >= n).
 *   beta == 0: C is not read (NaN or Inf there do not propagate).  k == 0 or
 *   alpha == 0: C = beta C and A, B are not read.  alpha and beta are applied
 *   in the output precision (f32 for COSMA_F32 / COSMA_BF16).
 *   COSMA_BF16 reads transposed operands in place (MN-major A, K-major B);
 *   COSMA_F64_EMU_BF16 splits them directly; COSMA_F64 / COSMA_F32 first copy a
 *   transposed operand untransposed into the workspace (one extra pass over it).
 * Other arguments, ownership and errors as cosma_gemm. */
int cosma_gemm_ex(int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                  const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                  int64_t ldc, int dtype, void* stream);

/* Complex double: C = alpha op(A) op(B) + beta C over interleaved (re, im) pairs
 * (C99 double complex / std::complex<double> layout, 16-byte aligned), run as
 * four real products on `engine` (COSMA_F64 or COSMA_F64_EMU_BF16; else
 * COSMA_ERR_UNSUPPORTED): Tr = Ar Br - Ai Bi, Ti = Ar Bi + Ai Br.
 *   op_a / op_b: 0 none, 1 transpose, 2 conjugate transpose; a transposed operand
 *   is stored transposed (A as k x m with lda >= m, B as n x k with ldb >= k).
 *   alpha, beta: HOST arrays {re, im}.  Leading dimensions count complex
 *   elements.  beta == 0 does not read C; alpha == 0 or k == 0 does not read A, B.
 * The planar parts and Tr, Ti (2 (mk + kn + mn) doubles) live in a library-owned
 * buffer grown with cudaMalloc outside capture (COSMA_ERR_NO_WORKSPACE inside
 * capture when too small); calls overlapping on the GPU must be serialised.  The
 * paper has no counterpart beyond the ScaLAPACK interface it targets. */
int cosma_zgemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, const double* alpha,
                const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta,
                void* C, int64_t ldc, int engine, void* stream);

/* Complex single: as cosma_zgemm over interleaved float (re, im) pairs (C99 float
 * complex layout, 8-byte aligned), the four real products on `engine` COSMA_F32
 * (FMA) or COSMA_F32_EMU_TF32 (three TF32 products each); else
 * COSMA_ERR_UNSUPPORTED.  alpha, beta: HOST float arrays {re, im}, applied in
 * single precision.  Staging (2 (mk + kn + mn) floats) shares cosma_zgemm's
 * library-owned buffer, with the same capture and serialisation rules. */
int cosma_cgemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, const float* alpha,
                const void* A, int64_t lda, const void* B, int64_t ldb, const float* beta,
                void* C, int64_t ldc, int engine, void* stream);

/* Same as cosma_gemm but runs the given plan (e.g. from cosma_plan_query or an
 * autotuner).  The plan is validated against the kernel's limits first. */
int cosma_gemm_planned(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                       const void* B, int64_t ldb, void* C, int64_t ldc, int dtype,
                       const cosma_plan* plan, void* stream);

/* `count` independent products in one persistent launch.  problems is a HOST
 * array; it may be reused once the call returns.  dtype: COSMA_F32 or
 * COSMA_BF16 (bf16 requires each A 16-byte aligned with lda a multiple of 8).
 * The first call with a given set of problems builds a device table of the
 * group (tensor maps, sizes, a cost-balanced assignment of tiles to CTAs) and
 * caches it (8 groups per device, until cosma_finalize).  A repeated call
 * with the same problems, pointers and workspace only launches kernels, so it
 * may be captured in a CUDA graph; during capture a group that is not cached
 * yet returns COSMA_ERR_NO_WORKSPACE.  A problem with k >= 2^35 or m or n >=
 * 2^38 returns COSMA_ERR_UNSUPPORTED. */
int cosma_gemm_grouped(int count, const cosma_problem* problems, int dtype, void* stream);

/* C = A B with A, B and C in HOST memory: the call copies the operands in and
 * the product out itself.  Arguments and dtypes as cosma_gemm, except that A,
 * B and C must be host pointers (device pointers: COSMA_ERR_INVALID_ARG).
 * Page-locked memory (cudaHostAlloc / cudaHostRegister) lets the copies
 * overlap the kernels; pageable memory works outside stream capture but
 * serialises them.  The call is asynchronous on `stream`: C holds the product
 * once the stream has reached the call (e.g. cudaStreamSynchronize), and A, B,
 * C must stay alive (A and B unchanged) until then.
 * The product is cut into at most 2 x 2 blocks (rows of A x columns of B, each
 * cut only when it is at least 8192 long); the host-to-device copies of the
 * next blocks, the kernels of the current block and the device-to-host copy of
 * the finished C block run concurrently, on two library-owned copy streams
 * that fork from and join back to `stream` through events (capturable).
 * Device staging -- the m x k and k x n inputs and the m x n result, rows
 * padded to a multiple of 8 elements -- is a library-owned buffer grown with
 * cudaMalloc outside capture; inside capture a call that needs more returns
 * COSMA_ERR_NO_WORKSPACE.  Calls whose work overlaps on the GPU (other streams
 * or threads) share that buffer and must be serialised.  The paper has no
 * counterpart: its operands start in the processors' memories. */
int cosma_gemm_host(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* B,
                    int64_t ldb, void* C, int64_t ldc, int dtype, void* stream);

/* ---- allocation-free variant ------------------------------------------ */

/* Size of the device array cosma_gemm_splitk_static uses for its partial sums
 * (32 MiB, reserved on every GPU that loads the library until process exit). */
#define COSMA_STATIC_SCRATCH_BYTES (32u << 20)

/* C = A B (dtype COSMA_F64 or COSMA_F32) with k split into pk slices whose
 * partial products go to a fixed, statically allocated device array, then a
 * fixed-order Reduce; the call never allocates device memory (no cudaMalloc,
 * no library arena).  The paper has no counterpart: it exists for callers
 * that cannot allocate once running -- graph capture in the global mode,
 * programs that own all device memory through their own pool, loops that
 * cannot take cudaMalloc's implicit synchronisation.
 *   pk >= 1 and at most ceil(k / k_block) of the planned tile
 *   (else COSMA_ERR_INVALID_ARG); pk * m * n * sizeof(element) must not exceed
 *   COSMA_STATIC_SCRATCH_BYTES (else COSMA_ERR_NO_WORKSPACE, nothing launched).
 *   Other arguments and errors as cosma_gemm.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress)
 * with that device current; make it before any stream capture.  All calls share
 * the array and it keeps the last call's contents: calls whose kernels overlap
 * on the GPU (other streams or threads) race on it and must be serialised. */
int cosma_gemm_splitk_static(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                             const void* B, int64_t ldb, void* C, int64_t ldc, int dtype,
                             int pk, void* stream);

/* ---- planning --------------------------------------------------------- */

/* Plan for an m x n x k product of the given dtype with the given selector
 * (cosma_selector).  ANALYTIC is host only; LEARNED runs the selector's
 * forward kernel once per new shape (synchronously) and caches the choice.
 * Returns cosma_status. */
int cosma_plan_query(int64_t m, int64_t n, int64_t k, int dtype, int selector,
                     cosma_plan* out);

/* Work units of a plan in execution order, as int64 sextuples
 * (row0, row1, col0, col1, k0, k1) per CTA, CTAs one after another (for an
 * emulated FP64 plan, as its kernels number them: k slice first).  Writes
 * at most max_units units to `units` (HOST, 6*max_units int64) and returns the
 * total number of units (so a first call with max_units = 0 sizes the buffer),
 * or a negative cosma_status. */
long long cosma_plan_units(int64_t m, int64_t n, int64_t k, const cosma_plan* plan,
                           int64_t* units, long long max_units);

/* FindSeqSchedule of Alg. 1 / Sec. 5.2: the integer (a, b) maximising
 * ab/(a + b) subject to ab + a + 1 <= S (ties: smaller ab, then smaller a).
 * S in words, S >= 3. */
int cosma_find_seq_schedule(long long S, int* a, int* b);

/* FitRanks of Alg. 1 / Sec. 7.1: the processor grid [pm, pn, pk] with
 * pm*pn*pk in [p - floor(delta p), p] that minimises the words of one local
 * domain ceil(m/pm)ceil(k/pk) + ceil(k/pk)ceil(n/pn) + ceil(m/pm)ceil(n/pn)
 * (ties: more processors used, then the lexicographically smaller grid). */
int cosma_fit_ranks(int64_t m, int64_t n, int64_t k, int p, double delta, int grid[3]);

/* ---- learned selector (MLP cost model) -------------------------------- */

/* The selector is a 3-layer FP32 network IN -> 64 -> 64 -> OUT with ReLU that
 * maps a product's features to the predicted log2-time of each of the OUT plan
 * candidates.  Parameter vector layout: W1 (64 x IN, row-major), b1 (64),
 * W2 (64 x 64), b2 (64), W3 (OUT x 64), b3 (OUT).  Not in the paper. */
#define COSMA_MLP_IN 7
#define COSMA_MLP_HIDDEN 64
#define COSMA_MLP_OUT 16
#define COSMA_MLP_PARAMS (COSMA_MLP_HIDDEN * COSMA_MLP_IN + COSMA_MLP_HIDDEN + \
                          COSMA_MLP_HIDDEN * COSMA_MLP_HIDDEN + COSMA_MLP_HIDDEN + \
                          COSMA_MLP_OUT * COSMA_MLP_HIDDEN + COSMA_MLP_OUT)

/* Plan candidate c (0 <= c < COSMA_MLP_OUT) for an m x n x k product: tile
 * class c / 8 (0: the kernel's largest C tile, 1: its smaller one), k split
 * pk = {1, 2, 4, 8}[(c / 2) % 4] and assignment order c % 2 (0: the FitRanks
 * grid of rectangular local domains, 1: balanced stripes).  Host only.
 * Returns COSMA_ERR_UNSUPPORTED when the candidate does not apply (k too
 * short for the split, a kernel without that tile or split). */
int cosma_plan_candidate(int64_t m, int64_t n, int64_t k, int dtype, int c, cosma_plan* out);

/* Selector input row x[COSMA_MLP_IN] (HOST) of a product: log2(m)/16,
 * log2(n)/16, log2(k)/16 and a one-hot of the dtype (F64, F32, BF16,
 * F64_EMU_BF16).  m, n, k >= 1. */
int cosma_selector_features(int64_t m, int64_t n, int64_t k, int dtype, float* x);

/* K-MLP-FWD: Y[b] = MLP(X[b]) for b < batch.  X (batch x IN), params, Y
 * (batch x OUT) are DEVICE pointers; asynchronous on `stream`. */
int cosma_mlp_forward(int batch, const float* X, const float* params, float* Y, void* stream);

/* K-MLP-BWD: loss L = (1/batch) sum_b (Y[b][cand[b]] - target[b])^2 and its
 * gradient with respect to params, summed over the batch in a fixed order
 * (deterministic).  All pointers DEVICE (loss: one float, may be NULL; grad:
 * COSMA_MLP_PARAMS floats).  Uses library workspace (grown outside capture). */
int cosma_mlp_loss_grad(int batch, const float* X, const int* cand, const float* target,
                        const float* params, float* grad, float* loss, void* stream);

/* K-MLP-ADAM: one Adam step (Kingma and Ba) on n parameters, step counting
 * from 1; m, v are the moment buffers.  DEVICE pointers. */
int cosma_mlp_adam(int n, float* params, const float* grad, float* m, float* v, int step,
                   float lr, float beta1, float beta2, float eps, void* stream);

/* Installs a trained network (HOST parameter vector) for COSMA_SELECT_LEARNED
 * on the current device, valid for sizes with log2 in [log2_lo, log2_hi];
 * outside that range (or with no network) plans fall back to the analytic
 * selector.  The network's outputs are read as log2 seconds per candidate.
 * params == NULL removes the network. */
int cosma_selector_set(const float* params, double log2_lo, double log2_hi);

/* Sets, for one dtype on the current device, how much faster (log2 seconds,
 * >= 0; INFINITY: never) the network must predict a candidate than the analytic
 * plan before COSMA_SELECT_LEARNED takes it; the default is 0.05 (about 3.5 %).
 * Kept across cosma_selector_set.  COSMA_ERR_INVALID_ARG for a bad dtype or a
 * negative / NaN margin; COSMA_ERR_CUDA without a device. */
int cosma_selector_margin(int dtype, float log2_margin);

/* Restricts the installed network to the dtypes whose bit (1 << dtype) is set in
 * dtype_mask -- the ones it was trained on; plans of other dtypes use the
 * analytic selector.  cosma_selector_set resets the mask to every dtype.
 * COSMA_ERR_UNSUPPORTED when no network is installed on the current device. */
int cosma_selector_restrict(unsigned dtype_mask);

/* Runs K-MLP-FWD on `count` shapes (HOST array mnk of 3*count int64) and
 * writes, per shape, the learned selector's choice (best, HOST, count ints)
 * and optionally all predictions (pred, HOST, count x OUT floats, may be
 * NULL).  The choice is the analytic plan -- written as its candidate index
 * when it is one of the candidates, else as -1 -- unless the network predicts
 * another applicable candidate faster by at least the dtype's margin
 * (cosma_selector_margin), whose index is then written.  Synchronous. */
int cosma_selector_predict(int count, const int64_t* mnk, int dtype, int* best, float* pred);

/* ---- measurement ------------------------------------------------------ */

/* on != 0 enables timing of each call's dominant kernel (the main loop:
 * K-F64, K-F32, K-BF16, K-EMU or the grouped kernel -- not the transposes,
 * slice extraction or the Reduce).  While enabled the library records a CUDA
 * event pair around that kernel on the call's stream.  Do not enable it while
 * a stream is being captured into a graph. */
int cosma_profile_enable(int on);

/* Waits for the recorded event pairs, writes their summed elapsed time in
 * milliseconds and their number, and clears them.  Either pointer may be NULL. */
int cosma_profile_read(double* main_kernel_ms, long long* launches);

/* Phases of the last cosma_gemm_host call on the current device made while
 * profiling was enabled (and not under stream capture), in milliseconds of
 * device time: phases[0] the whole call, [1] the head (until the first block
 * product starts: the first blocks' host->device copies and preparation), [2]
 * the block products together, [3] the tail (after the last block product: the
 * last C block's device->host copy), [4] the host->device copies (call start to
 * the last copy landed), [5] the number of block products.  phases is a HOST
 * array of `count` doubles; at most 6 are written.  Waits for that call's end.
 * Returns the number written, or COSMA_ERR_INVALID_ARG if no such call was
 * recorded (or bad arguments), COSMA_ERR_CUDA without a device. */
int cosma_profile_host(double* phases, int count);

/* ---- status ----------------------------------------------------------- */

/* Synchronises `stream`, then reads and clears the device status word of the
 * current device.  Returns COSMA_OK, COSMA_ERR_TIMEOUT, COSMA_ERR_NONFINITE or
 * COSMA_ERR_CUDA. */
int cosma_stream_status(void* stream);

/* Static human-readable text for a cosma_status value. */
const char* cosma_status_string(int status);

/* Number of SMs of the current device (0 without a device). */
int cosma_device_sms(void);

/* Running count of kernels this library has launched in this process (all
 * devices, all streams), for accounting in benchmarks. */
long long cosma_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* COSMA_GB300_H */
