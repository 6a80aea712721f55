/*
 * tucker.h -- C ABI of a GB300 (sm_103a) library for the fixed-rank Tucker
 * approximation with adaptive shifts: shifted randomized T-HOSVD
 * (Algorithm 2) and shifted randomized ST-HOSVD (Algorithm 3) of
 * Che, Wei, Wu, Yan (arXiv 2506.04840).
 *
 * Problem (Problem 2.1, Section 2.2): given a tensor A of size
 * n_1 x ... x n_d and a Tucker rank (r_1..r_d) with r_k < n_k, find
 * orthonormal U_k (n_k x r_k) such that A ~ A x_1 U_1U_1^T ... x_d U_dU_d^T;
 * the core is G = A x_1 U_1^T ... x_d U_d^T.
 *
 * Conventions shared by every entry point
 *  - Tensors are dense and column-major: entry (i_1..i_d), 0-based, sits at
 *    i_1 + n_1*(i_2 + n_2*(i_3 + ...)).  The mode-k unfolding A_(k)
 *    (n_k x prod_{m!=k} n_m, Section 2) orders its columns lowest remaining
 *    mode fastest; it is never materialised.
 *  - Matrices (Y, Q, U_k) are column-major with leading dimension = rows.
 *  - Every data pointer is a DEVICE pointer owned by the caller unless a
 *    comment says "host".  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it unless they return host data
 *    (tk_stats, tucker_server_poll), which synchronise the stream.
 *  - Errors are returned as tk_status; nothing crosses the ABI as an
 *    exception and no kernel traps.  Argument errors are detected before any
 *    launch (TK_EINVAL).  Problems found on the device (non-finite values,
 *    a bounded wait that ran out) are recorded in a device status word and
 *    reported by the next call that synchronises.
 *  - Omega_k (Algorithms 2/3, "draw a standard Gaussian matrix") is never
 *    stored: entry (j, c) is regenerated from Philox4x32-10 with key =
 *    (seed mod 2^32, seed >> 32) and counter (j mod 2^32, j >> 32, c >> 2,
 *    (k & 0xff) | (tag << 8)), then Box-Muller with the library's own FP32
 *    log/sin/cos (tucker_debug_omega returns the exact values).
 *  - svd results are sorted by descending singular value and each column's
 *    sign is fixed so that its entry of largest magnitude is positive.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TK_MAX_D 8     /* largest supported tensor order d */
#define TK_MAX_Q 32    /* largest power-iteration count q */
#define TK_MAX_L 128   /* largest sketch width l_k = r_k + s_k */
#define TK_ORDER_DESCENDING (-2)   /* tk_opts.order[0]: modes by non-increasing n_k */

typedef enum {
  TK_OK = 0,
  TK_EINVAL = 1,       /* invalid argument (checked before any launch) */
  TK_ENOMEM = 2,       /* device allocation failed */
  TK_ECUDA = 3,        /* a CUDA runtime call failed */
  TK_EBREAKDOWN = 4,   /* non-finite value met on the device */
  TK_ETIMEOUT = 5,     /* a bounded device wait ran out */
  TK_ENOTIMPL = 6,     /* valid request outside the built kernels' limits */
  TK_EWORKSPACE = 7    /* caller workspace smaller than tucker_workspace_size */
} tk_status;

typedef enum { TK_F64 = 0, TK_F32 = 1, TK_BF16 = 2 } tk_dtype;

/* Shift rule of the power loop.
 * TK_SHIFT_PAPER: alpha_0 = 0; after step t, if Sigma(l,l) > alpha_{t-1} then
 *   alpha_t = (Sigma(l,l) + alpha_{t-1})/2 else alpha_t = alpha_{t-1}
 *   (Algorithm 2, Algorithm 3).
 * TK_SHIFT_NONE: alpha = 0 throughout (Algorithm A.1, the unshifted model). */
typedef enum { TK_SHIFT_PAPER = 0, TK_SHIFT_NONE = 1 } tk_shift;

/* Precision form.  TK_PREC_PLAIN: every pass reads the tensor in its own
 * dtype.  TK_PREC_BF16_POWER (FP32 tensors only): power steps 1..q-1 read a
 * bfloat16 copy of the current tensor (FP32 accumulation on tensor cores);
 * the sketch, power step q, the TTM shrink and the core read FP32. */
typedef enum { TK_PREC_PLAIN = 0, TK_PREC_BF16_POWER = 1 } tk_precision;

/* Test matrix Omega_k of the sketch (Section 5.5 compares these four; the
 * remark after Algorithm 3 motivates the structured ones).
 * TK_OMEGA_GAUSS: i.i.d. N(0,1), generated inside the sketch pass, never
 *   stored (the draw defined above).
 * TK_OMEGA_UNIFORM: i.i.d. uniform on [-1, 1]; entry (j, c) maps word
 *   c mod 4 of the Gaussian entry's Philox counter to
 *   u = (2*(w >> 8) + 1 - 2^24) * 2^-24 (exact in FP32).
 * TK_OMEGA_KR_GAUSS, TK_OMEGA_KR_UNIFORM: the Khatri-Rao product of one
 *   factor F_m (n_m x l, n_m the current size of mode m) per mode m != k,
 *   Omega_k(j, c) = prod_{m != k} F_m(i_m(j), c) with (i_m) the unfolding's
 *   column j (lowest mode fastest), multiplied in FP64 in ascending m and
 *   rounded once to the sketch's accumulation type (FP32 or FP64).
 *   F_m(i, c) comes from the counter (i, 2^31 | m, c >> 2,
 *   (k & 0xff) | (tag << 8)), then Box-Muller (pairs of words, as above) or
 *   the uniform map.
 * The three structured kinds are written into the W buffer of the power
 * steps (prod_{m != k} n_m x l_k in the accumulation type) and the sketch
 * reads them there. */
typedef enum {
  TK_OMEGA_GAUSS = 0,
  TK_OMEGA_UNIFORM = 1,
  TK_OMEGA_KR_GAUSS = 2,
  TK_OMEGA_KR_UNIFORM = 3
} tk_omega;

/* A dense tensor.  data: device pointer, column-major, dtype F64 or F32
 * (BF16 only where stated). */
typedef struct {
  int d;                   /* order, 1 <= d <= TK_MAX_D */
  int64_t n[TK_MAX_D];     /* sizes n_1..n_d, each >= 1 */
  tk_dtype dtype;
  const void* data;
} tk_tensor;

/* Options of Algorithms 2/3 (inputs of the boxes: s, q; plus the draw). */
typedef struct {
  int q;                   /* power parameter q, 0 <= q <= TK_MAX_Q
                              (q = 0: sketch only) */
  int s[TK_MAX_D];         /* oversampling s_k; l_k = min(r_k+s_k, n_k, cols) */
  uint64_t seed;           /* Omega key */
  uint32_t tag;            /* Omega stream tag, < 2^24 */
  tk_shift shift;
  tk_precision prec;
  int order[TK_MAX_D];     /* ST-HOSVD processing order (0-based modes, a
                              permutation); order[0] = TK_ORDER_DESCENDING:
                              non-increasing n_k (Section 3.2, ties in
                              ascending mode index); other order[0] < 0:
                              0..d-1 */
  void* workspace;         /* device workspace or NULL (then the call
                              allocates and frees it on `stream`) */
  size_t workspace_bytes;
  tk_omega omega;          /* test matrix kind (0 = Gaussian) */
} tk_opts;

/* Per-call statistics (HOST memory; filling it synchronises the stream). */
typedef struct {
  int d;
  int q;
  int l[TK_MAX_D];                      /* clamped sketch widths */
  int order[TK_MAX_D];                  /* processing order used */
  double alpha[TK_MAX_D][TK_MAX_Q];     /* alpha_t^(k), t = 1..q */
  double sigma_l[TK_MAX_D][TK_MAX_Q];   /* Sigma_k(l,l) after step t */
  double sigma[TK_MAX_D][TK_MAX_L];     /* final Sigma_k (first l entries) */
} tk_stats;

/* Human-readable name of a status code (static string). */
const char* tucker_status_string(tk_status s);

/* Bytes of device workspace tucker_rthosvd (st = 0) or tucker_rsthosvd
 * (st = 1) needs for these arguments; 0 if the arguments are invalid. */
size_t tucker_workspace_size(const tk_tensor* A, const int* r, const tk_opts* o, int st);

/* Rows [row0, row0+rows) of Omega_k for a sketch of width l (Algorithm 2/3,
 * "draw a standard Gaussian matrix"), written as a rows x l column-major
 * FP32 matrix `out` (device).  k: 0-based mode; tag < 2^24. */
tk_status tucker_debug_omega(int k, int64_t row0, int64_t rows, int l, uint64_t seed,
                             uint32_t tag, float* out, void* stream);

/* Test entry point: one product D = A B on the tcgen05 tensor cores in
 * kind::tf32 (four K = 8 instructions accumulating in tensor memory), used to
 * fix how the instruction rounds FP32 operands to TF32 and how its FP32
 * accumulator rounds between instructions (the paper has no counterpart;
 * the FP32 tensor-core contractions depend on both).
 * A: 128 x 32, B: 32 x 64, D: 128 x 64, all row-major FP32, device.
 * mode 0: A read from shared memory (K-major, 128-byte swizzle); 1: A from
 * tensor memory.  Synchronises the stream; TK_ETIMEOUT if the tensor cores
 * did not finish within 2 s; TK_EINVAL for another mode. */
tk_status tucker_debug_tf32_mma(const float* A, const float* B, float* D, int mode,
                                void* stream);

/* Holistic variants (Algorithm B.1 for ST-HOSVD with TK_SHIFT_PAPER;
 * Algorithm A.2, ST or T-HOSVD case, with TK_SHIFT_NONE; the T-HOSVD case
 * with the shift is the variant the remark after Algorithm B.1 names).
 * Per mode k = 1..d: the sketch and q power steps of Algorithms 2/3 with all
 * l_k = min(r_k + s_k, n_k, columns) columns kept as Q_k, on the shrinking
 * tensor B (st = 1) or on A (st = 0); B <- B x_k Q_k^T.  Then the
 * deterministic ST-HOSVD of the l_1 x ... x l_d tensor B (held in FP64;
 * V_k = the leading r_k eigenvectors of B_(k) B_(k)^T, summed in FP64 and
 * solved by the svd in the input's precision, sorted and sign-fixed like
 * the svd results) gives the core, and U_k = Q_k V_k.  Modes in natural order
 * (o->order ignored); plain precision only (TK_EINVAL otherwise); any
 * tk_omega kind.  Outputs, workspace (tucker_holistic_workspace_size bytes,
 * or allocated on `stream` when o->workspace is NULL) and errors as
 * tucker_rsthosvd: TK_EINVAL for r_k >= n_k or s_k < 0, TK_ENOTIMPL when an
 * l_k exceeds TK_MAX_L.  stats describe the range finder (l_k, its shifts
 * and Sigma).  Appendices A and B of the paper. */
tk_status tucker_holistic(const tk_tensor* A, const int* r, const tk_opts* o, int st, void* core,
                          void* const* U, tk_stats* stats, void* stream);
/* Bytes of device workspace tucker_holistic needs; 0 for invalid arguments. */
size_t tucker_holistic_workspace_size(const tk_tensor* A, const int* r, const tk_opts* o,
                                      int st);

/* Omega_k of any kind (tk_omega) for a tensor of order d and sizes n, in the
 * unfolding's own row order, written as a (prod_{m != k} n_m) x l
 * column-major FP32 matrix `out` (device).  Returns TK_EINVAL for a bad
 * kind, k, l (1..TK_MAX_L), sizes or tag; the Khatri-Rao kinds allocate
 * their factor scratch on `stream`. */
tk_status tucker_debug_omega_matrix(tk_omega kind, int d, const int64_t* n, int k, int l,
                                    uint64_t seed, uint32_t tag, float* out, void* stream);

/* Sketch Y = A_(k) Omega_k (Algorithm 2: svd argument before the power
 * loop; Algorithm 3 with the current tensor G).  A: F64, F32 or BF16.
 * Y: n_k x l FP64 (device), the exact sum of per-block FP32 (F32/BF16) or
 * FP64 partial products reduced in FP64.  Omega_k is generated in
 * registers, never stored. */
tk_status tucker_sketch(const tk_tensor* A, int k, int l, uint64_t seed, uint32_t tag,
                        double* Y, void* stream);

/* The sketch of tucker_sketch, computed without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory on their behalf (servers that
 * reserve all device memory up front, plugins whose host application owns
 * the allocator, loops that must not risk an allocation failing or stalling
 * mid-request).  It calls no cudaMalloc, cudaFree or allocating routine.
 * Its partial products live in one static device array of
 * TK_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit.  Arguments, layout and result are those of tucker_sketch.
 * Limits: n_k * (l rounded up to 16, 32, 64 or 128) * 4 bytes (8 for F64
 * tensors) must not exceed TK_NOALLOC_SCRATCH_BYTES, else TK_EWORKSPACE is
 * returned and nothing runs.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  The address is
 * kept for the life of the process and belongs to the device's primary
 * context: after cudaDeviceReset, or with another driver context current,
 * it is no longer valid, so use the primary context only.  All calls share
 * the array: calls that overlap on the GPU (different streams, concurrent
 * threads) race on it and must be serialised by the caller. */
#define TK_NOALLOC_SCRATCH_BYTES (8u << 20)
tk_status tucker_sketch_noalloc(const tk_tensor* A, int k, int l, uint64_t seed, uint32_t tag,
                                double* Y, void* stream);

/* q steps of the shifted power loop on A_(k) (Algorithm 2 inner loop):
 *   [Q, Sigma] = svd(A_(k)(A_(k)^T Q) - alpha_{t-1} Q, 'econ'), shift update.
 * Q:     in: n_k x l orthonormal (FP64, device); out: left singular vectors.
 * sigma: out: the l singular values of the last step (FP64, device).
 * alpha: in: alpha_{t0}; out: alpha after q steps (one FP64, device).
 * A: F64, F32 or BF16 (BF16: the reduced-precision pass, one fused read of
 * A per step on tensor cores).  l <= TK_MAX_L. */
tk_status tucker_shifted_power(const tk_tensor* A, int k, int l, int q, tk_shift rule,
                               double* Q, double* sigma, double* alpha, void* stream);

/* Shifted randomized T-HOSVD, Algorithm 2.  r: host array of d ranks,
 * 1 <= r_k < n_k (Problem 2.1).  core: r_1 x ... x r_d in A's dtype
 * (device).  U: host array of d device pointers, U[k] n_k x r_k in A's
 * dtype.  st: optional host stats (NULL = none).  A: F64 or F32. */
tk_status tucker_rthosvd(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                         void* const* U, tk_stats* st, void* stream);

/* Shifted randomized ST-HOSVD, Algorithm 3 (arguments as tucker_rthosvd;
 * o->order gives the processing order, Section 2.2). */
tk_status tucker_rsthosvd(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                          void* const* U, tk_stats* st, void* stream);

/* Algorithm 4: Algorithm 3 with the power count q_k of each mode chosen by
 * the PVE accuracy test (Section 3.3).  After the sketch, steps
 * t = 1..q_max (q_max = o->q, 1 <= q_max <= TK_MAX_Q) run until
 *   max_{i <= r_k} |sigma_t(i) - sigma_{t-1}(i)| <= tol * sigma_t(r_k + 1),
 * where sigma_t = diag(Sigma) + alpha_{t-1} after step t's svd, sigma_0 = 0,
 * and sigma_t(r_k + 1) is the l_k-th entry when l_k = r_k; q_k = that t
 * (q_max when the test never holds).  The shift update of Algorithm 3
 * follows a step that does not stop.  tol >= 0 (host).  The test is taken
 * on the host after each step, so the call synchronises `stream` once per
 * power step.  q_out: host array of d ints, the chosen q_k (NULL = not
 * returned).  o->prec must be TK_PREC_PLAIN.  Other arguments as
 * tucker_rsthosvd; in st, q is q_max and the per-step entries past q_k are 0. */
tk_status tucker_rsthosvd_pve(const tk_tensor* A, const int* r, const tk_opts* o, double tol,
                              void* core, void* const* U, int* q_out, tk_stats* st,
                              void* stream);
/* Algorithm 2 (T-HOSVD) with the same PVE-controlled counts: every mode's
 * sketch and power steps read A; arguments, errors and q_out as
 * tucker_rsthosvd_pve.  The modes run one after the other (the host reads
 * each step's Sigma back). */
tk_status tucker_rthosvd_pve(const tk_tensor* A, const int* r, const tk_opts* o, double tol,
                             void* core, void* const* U, int* q_out, tk_stats* st,
                             void* stream);

/* Relative error RE = ||A - G x_1 U_1 ... x_d U_d|| / ||A|| (Section 5,
 * definition of RE).  core, U as returned by tucker_r(s)thosvd (A's dtype);
 * r: host ranks.  rel_err: one FP64 (device).  The reconstruction is never
 * stored: the last mode product is fused with the squared-difference sum. */
tk_status tucker_error(const tk_tensor* A, const void* core, const int* r, const void* const* U,
                       double* rel_err, void* stream);

/* ---- many independent problems: batched launches and a serving loop ------
 * The paper treats one tensor at a time; these entry points run Algorithm 3
 * (shifted randomized ST-HOSVD, modes in natural or descending order, plain
 * precision) on many tensors at once.  Each step kind runs as ONE launch over a work list
 * holding every problem's blocks of that step (a persistent grid strides over
 * them), so uneven shapes share the GPU.  A problem's blocks do exactly the
 * work the single-problem call does, in the same order: its results are
 * bitwise those of tucker_rsthosvd (+ tucker_error) on the same arguments,
 * whatever else shares the launches. */
typedef struct {
  tk_tensor A;             /* F64 or F32, device, caller-owned */
  int r[TK_MAX_D];         /* Tucker rank, 1 <= r_k < n_k */
  int s[TK_MAX_D];         /* oversampling s_k */
  int q;                   /* power steps, 0 <= q <= TK_MAX_Q */
  uint64_t seed;           /* Omega key */
  uint32_t tag;            /* Omega stream tag, < 2^24 (e.g. the item index) */
  void* core;              /* out: r_1 x ... x r_d, A's dtype (device) */
  void* U[TK_MAX_D];       /* out: U[k] n_k x r_k, A's dtype (device) */
  double* rel_err;         /* out: RE of (core, U) as tucker_error computes
                              it (one FP64, device), or NULL = not computed */
  int order;               /* processing order: 0 = natural (modes 1..d),
                              TK_ORDER_DESCENDING = non-increasing n_k
                              (Section 3.2); other values: TK_EINVAL */
} tk_item;

typedef struct tk_batch_s* tk_batch;

/* Plans a batch: validates every item (TK_EINVAL names nothing; check each
 * item with tucker_rsthosvd's rules), allocates the device workspace and job
 * tables (owned by the batch) and, if use_graph != 0, captures the launches
 * into a CUDA graph.  All items share one dtype.  Items must stay valid
 * (tensors readable, outputs writable) for every run. */
tk_status tucker_batch_create(const tk_item* items, int count, tk_shift rule, int use_graph,
                              tk_batch* out);
/* Runs the batch on `stream` (asynchronous).  Runs of one batch must not
 * overlap: they share its workspace. */
tk_status tucker_batch_run(tk_batch b, void* stream);
/* Waits for the last run and copies each item's device status into
 * status[count] (host; NULL = skip).  Returns the first non-OK status. */
tk_status tucker_batch_wait(tk_batch b, int* status);
/* Launches per run and device bytes the batch holds (host outputs, NULL = skip). */
tk_status tucker_batch_info(tk_batch b, int64_t* launches, size_t* device_bytes);
tk_status tucker_batch_destroy(tk_batch b);
/* One-shot: create (no graph), run on `stream`, wait, destroy. */
tk_status tucker_batch_rsthosvd(const tk_item* items, int count, tk_shift rule, void* stream);

/* Autotuner of the split-K counts (the batching pattern's "tile shapes and
 * split-K chosen by an autotuner"; the paper has no counterpart).  The FP32
 * CUDA-core products split their contraction over CTAs: Y = X_(k) W over the
 * unfolding's columns, the TTM over the rows when it has few column tiles.
 * With tuning enabled, every call and batch takes these split counts from a
 * process-wide table keyed by shape class (product kind, n_k, output width,
 * column count rounded up to a power of two); classes missing from the table
 * keep the fixed heuristic.  Single calls and batches read the same table,
 * so a batch item's results stay bitwise equal to its single call.  Change
 * the table or the switch only between calls (plans made under one setting
 * size their partial buffers for it). */
tk_status tucker_tune_enable(int on);          /* default: off */
tk_status tucker_tune_clear(void);
tk_status tucker_tune_entries(int* count);
/* Text file: a header line, then one line per class.  Load merges into the
 * table; TK_EINVAL on a missing or malformed file (table unchanged). */
tk_status tucker_tune_save(const char* path);
tk_status tucker_tune_load(const char* path);
/* Plans and times the batch of `items` (CUDA graph, 2 warm-up + 3 timed
 * runs on `stream`) once per candidate: the heuristic split counts scaled
 * by 2, 1, 1/2, 1/4, 1/8 and 1/16.  Stores the fastest candidate's count for
 * every shape class the batch uses.  Blocks until done.  Outputs (host,
 * NULL = skip): the fastest run's ms, the heuristic's ms, the fastest
 * scale as a shift (-1 = x2, 0 = x1, k = x2^-k).  The items' outputs are
 * written by the timing runs. */
tk_status tucker_tune_batch(const tk_item* items, int count, tk_shift rule, void* stream,
                            double* best_ms, double* base_ms, int* best_shift);

/* Serving loop.  A worker thread admits submitted requests in arrival order
 * while their workspace fits in a reserved device pool and fewer than
 * max_active are in flight, then advances every admitted request by one
 * phase (sketch, one power step, finish of a mode, error) per tick, each tick
 * being one batched launch per step kind over all admitted requests; ticks
 * are pipelined on the server's stream.  A request's result does not depend
 * on what it shares ticks with (see above). */
typedef struct {
  size_t pool_bytes;       /* device pool for request workspaces (0: half of
                              the free memory at creation) */
  int max_active;          /* most requests in flight (0: 256) */
  tk_shift rule;
} tk_server_opts;

typedef struct {
  uint64_t id;             /* as returned by tucker_server_submit */
  int status;              /* tk_status of the request */
  double submit_s;         /* host clock (seconds since the server started) */
  double admit_s;
  double done_s;           /* when the worker saw the request's last tick end */
} tk_completion;

typedef struct tk_server_s* tk_server;

/* Creates the server on the current device; reserves the pool. */
tk_status tucker_server_create(const tk_server_opts* o, tk_server* out);
/* Queues a request (validated here: TK_EINVAL; TK_ENOMEM if its workspace
 * can never fit the pool).  The item's buffers stay caller-owned and must
 * stay valid until its completion has been returned by tucker_server_poll. */
tk_status tucker_server_submit(tk_server s, const tk_item* item, uint64_t* id);
/* Returns up to `max` completions (host array), oldest first; never blocks. */
int tucker_server_poll(tk_server s, tk_completion* out, int max);
/* Blocks until every submitted request has completed or timeout_s passed
 * (TK_ETIMEOUT). */
tk_status tucker_server_drain(tk_server s, double timeout_s);
/* Server clock (seconds since creation), for arrival bookkeeping. */
double tucker_server_clock(tk_server s);
/* Finishes the requests in flight, stops the worker, frees the pool. */
tk_status tucker_server_destroy(tk_server s);

/* ---- instrumentation (no counterpart in the paper; used by the benchmark)
 * When enabled, every launch of the kernel classes below is bracketed by
 * CUDA events recorded on the launch stream, together with the algorithmic
 * bytes and flops of that launch (the data the method must move / the
 * arithmetic it must do, not the kernel's actual traffic). */
typedef enum {
  TK_K_SKETCH = 0,      /* Y = X_(k) Omega_k */
  TK_K_POWER_W = 1,     /* W = X_(k)^T Q (CUDA-core power step, first half) */
  TK_K_POWER_Y = 2,     /* Y = X_(k) W (CUDA-core power step, second half) */
  TK_K_POWER_FUSED = 3, /* Y = X_(k)(X_(k)^T Q) - alpha Q, one fused pass */
  TK_K_SMALL_SVD = 4,   /* svd of the n_k x l iterate + shift update */
  TK_K_TTM = 5,         /* G <- G x_k U_k^T */
  TK_K_ERROR = 6,       /* reconstruction-error passes */
  TK_K_CONVERT = 7,     /* bf16 shadow, copies, reductions, polish */
  TK_K_RITZ = 8,        /* Rayleigh-Ritz rotation of W before the precision
                           form's FP32 step (Gram, l x l eigenvectors, W Z) */
  TK_K_KINDS = 9
} tk_kernel_kind;

typedef struct {
  int64_t launches[TK_K_KINDS];   /* launches recorded */
  double ms[TK_K_KINDS];          /* summed event-timed duration */
  double bytes[TK_K_KINDS];       /* summed algorithmic bytes */
  double flops[TK_K_KINDS];       /* summed algorithmic flops */
  int64_t kernels;                /* all kernels launched since the last reset */
} tk_profile;

/* on != 0 starts recording (and clears what was recorded); 0 stops. */
tk_status tucker_profile_enable(int on);
/* Waits for the recorded events, fills *out (host) and clears the record. */
tk_status tucker_profile_read(tk_profile* out);

/* Round count FP32 values to bfloat16 (round to nearest, ties to even);
 * out holds count uint16 bit patterns (device).  The precision form's
 * shadow copy. */
tk_status tucker_to_bf16(const float* x, int64_t count, uint16_t* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_H */
