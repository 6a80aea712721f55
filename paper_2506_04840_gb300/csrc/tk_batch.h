// Work-list ("batched") launches: one launch runs the same step kind for many
// independent problems.  Each job is one problem's launch of that step (its
// grid given by `blocks`); a launch's blocks are the concatenation of its
// jobs' blocks, and a persistent grid strides over them.  A job computes
// exactly what the single-problem launch of that step computes, with the same
// block decomposition, so its result does not depend on what else shares the
// launch.
#pragma once

#include <cuda.h>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "tk_internal.h"

namespace tk {

// Y_part = X_(k) B (B = Omega_k when W == NULL), grid gx x splits.
struct XbJob {
  const void* X;
  int64_t P, n, S;
  const void* W;
  int64_t cps;          // columns per split (multiple of the column chunk)
  void* part;
  uint64_t seed;
  uint32_t tag;
  int l, mode, gx;
};

// Y = sum of partials - alpha Q, grid ceil(n l / 256).
struct ReduceJob {
  const void* part;
  int64_t n;
  const double* Q;
  const double* alpha;
  double* Y;
  int splits, l, lc;
  const void* part_lo;  // compensated partials: the lo plane (or NULL)
};

// svd of an n x l iterate in one CTA (+ shift update), grid 1.
struct SvdJob {
  const double* Y;
  double* Q;
  double* sigma;
  double* alpha;
  double* ahist;
  double* shist;
  int* status;
  int n, l, shift_rule, update_shift, basis_only;
};

// svd of an n x l iterate too long for one CTA: the two-level TSQR chain of
// the single call (leaf QR, root QR + svd + shift update, leaf Q, sign), one
// job per problem in each of four launches, on the single call's scratch
// carve.  Blocks: leaf QR Pb; root 1; leaf Q Pb (register-resident: Pb x
// ceil(l / 16)); sign l.
struct TsqrJob {
  const double* Y;
  double* Q;
  double* sigma;
  double* alpha;
  double* ahist;
  double* shist;
  int* status;
  void* V;              // leaf reflectors (solver type: FP32 or FP64)
  void* tau;
  void* Rst;            // stacked leaf R's
  void* Mout;           // root result
  double* colmax;       // per leaf and column: largest |entry| and its row
  int* colidx;
  int64_t n;
  int l, MB, Pb, shift_rule, update_shift, basis_only;
};

// out = X x_k B^T (EPI 0) or the fused error expansion (EPI 1), grid gx x gy.
struct XtbJob {
  const void* X;
  int64_t P, n, S;
  const double* B;
  int64_t b_ri, b_cm;
  void* out;
  const void* A;
  double* err;
  int m, gx;
};

// CholeskyQR polish of an n x r factor: Gram partials, then the update.
struct GramJob {
  const double* U;
  double* part;
  int64_t n;
  int r;
};
struct PolishJob {
  double* U;
  const double* part;
  int* status;
  int64_t n;
  int r, nblk;
};

// dst (rows x cols) = src converted to the destination type.
struct CopyJob {
  const double* src;
  void* dst;
  int64_t lds, ldd, rows, cols;
};

// rel = sqrt(sum e^2 / sum a^2) over `blocks` partial pairs, grid 1.
struct ErrFinalJob {
  const double* part;
  double* rel;
  int blocks;
};

// FP32 mode-major (P == 1) register-tiled contractions (k_contract32.cu).
struct Xtb32Job {
  const void* X;
  int64_t n, cols;
  const float* B;       // B rounded to FP32 (as the single-problem path rounds it)
  int64_t b_ri, b_cm;
  void* out;
  void* part;           // non-null: row splits write partials here (ks > 1)
  int64_t kps;          // rows per split
  int m, gx, gy, tout;
};
// Last-mode expansion fused with the squared-difference sums (S == 1).
struct Err32Job {
  const void* T;
  int64_t P;
  const float* B;       // the returned FP32 factor
  int64_t b_ri, b_cm;
  const void* A;
  double* err;
  int K, m, gx;
};
struct Xtb32RedJob {
  const void* part;
  void* out;
  int64_t cols;
  int m, ks, tout;
};
struct Xb32Job {
  const void* X;
  int64_t n, cols;
  const void* W;
  int64_t cps, ka, kb;
  void* part;
  void* part_lo;        // compensated sums of Y = X W: the lo plane (flag bit 4)
  uint64_t seed;
  uint32_t tag;
  int l, lc, mode, gx, gy;
};

// W = X^T B on the tensor cores (k_tc32.cu): one problem's tensor maps and
// sizes; a single call passes it as a kernel parameter, batches and the
// server keep it in their job tables (64-byte aligned).
struct alignas(64) Tc32XtbJob {
  CUtensorMap mx;     // X_(k): inner n (rows), outer cols, box 32 x 128
  CUtensorMap mb;     // the B planes: inner n_pad, outer 128, box 32 x 64
  float* out;
  int* err;           // the problem's status word (TK_ETIMEOUT if a wait ran out)
  long long cols;     // columns of X_(k)
  long long units;    // ceil(cols / 256)
  long long ld;       // out_mode 2: row stride of the planes
  int n;              // rows of X_(k) (the contraction)
  int nk;             // stages per unit: ceil(n / 32)
  int m;              // outputs written (<= 64)
  int out_mode;       // 0: out[c + m j]; 1: out[j + cols c]; 2: planes (hi, lo)
};

// The sketch Y_part = X_(k) Omega_k on the tensor cores (k_tc32.cu) for one
// problem: units of 256 rows x one column group, partials part[g][n][64].
struct alignas(64) Tc32SketchJob {
  CUtensorMap mx;     // X_(k): inner n (rows), outer cols, box 32 x 32
  float* part;        // [groups][n][64] FP32 partials
  int* err;
  __nv_bfloat16* shadow;  // or NULL: also write the bfloat16 copy of X (RNE)
  long long cols;
  long long cpg;      // columns per group (multiple of 32)
  long long units;    // nrb * groups
  long long ka, kb;   // Omega row map of the layout (jk = j / ka + kb (j % ka))
  uint64_t seed;
  uint32_t tag;
  int n, nrb, groups, l, mode;
};

// B (n x m, FP64) -> its hi/lo TF32 planes for one problem.
struct Tc32SplitJob {
  const double* B;
  int64_t b_ri, b_cm;
  float* B2;
  int n, m, n_pad;
};

enum BatchKind {
  BK_XB = 0, BK_REDUCE, BK_SVD, BK_XTB, BK_GRAM, BK_POLISH, BK_COPY, BK_ERRFIN, BK_XTB32,
  BK_XB32, BK_XTB32RED, BK_ERR32, BK_TC32SPLIT, BK_TC32XTB, BK_TC32SKETCH,
  BK_TSQR_LEAF, BK_TSQR_ROOT, BK_TSQR_LEAFQ, BK_TSQR_SIGN
};

constexpr size_t kJobBytes = 384;   // every job struct fits (two tensor maps + sizes)

struct BatchLaunch {
  int kind;           // BatchKind
  int xt;             // XType of the data (copy: of the destination)
  int tile;           // xb / xtb: column tile LC; svd: threads per CTA
  int flag;           // xb: 1 = Omega; xtb: EPI; copy: 1 = round through FP32;
                      // xb32 / xtb32: (Omega) | (warps along rows) << 1;
                      // tsqr: 2 or 4 = register-resident kernels with that
                      // many columns per warp, 0 = shared-memory kernels
  const void* jobs;   // device array of njobs job structs
  const uint32_t* start;   // device: first block of each job
  int njobs;
  uint32_t total;     // blocks over all jobs
  size_t smem;        // dynamic shared memory per CTA
};

cudaError_t launch_batch(const BatchLaunch& b, cudaStream_t st);
void batch_kernels_init();
void c32_batch_init();   // part of batch_kernels_init (k_contract32.cu)
// per-file dispatchers
cudaError_t launch_batch_contract(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_small(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_misc(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_c32(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_tc32(const BatchLaunch& b, cudaStream_t st);

// The tensor-core W = X^T B of one problem as job structs (false when the
// view is not eligible, tc32_ok); blocks of its split job.
bool tc32_xtb_jobs(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm, int m,
                   float* out, int out_mode, int64_t ld, void* scratch, int* err,
                   Tc32SplitJob* sj, Tc32XtbJob* xj);
uint32_t tc32_split_blocks(const Tc32SplitJob& j);
size_t tc32_xtb_smem();
// The tensor-core sketch of one problem (false when not eligible); its
// partial count (column groups) and bytes.
bool tc32_sketch_job(const void* X, View v, int l, uint64_t seed, uint32_t tag, int mode,
                     int64_t ka, int64_t kb, float* part, int* err, void* shadow,
                     Tc32SketchJob* j);
int tc32_sketch_groups(View v);
size_t tc32_sketch_part_bytes(View v);
size_t tc32_sketch_smem();
cudaError_t launch_tc32_sketch(const Tc32SketchJob& j, cudaStream_t st);
// Launch shapes of the FP32 mode-major kernels.
struct Xtb32Shape {
  int wj, wc, gx, gy, threads, ks;
  int64_t kps;
};
struct Xb32Shape {
  int wi, wc, lc, gx, gy, splits, threads;
  int64_t cps;
};
// allow_split: rows may be split (needs xtb32_scratch bytes of scratch).
Xtb32Shape xtb32_shape(View v, int m, bool allow_split);
// splits = 0: the default split count; else that many column splits.
Xb32Shape xb32_shape(View v, int l, int splits = 0);

// Per-job launch shapes, as the single-problem launchers choose them.
int xb_grid_x(View v, int l);
int64_t xb_cols_per_split(XType xt, View v, int splits);
int xtb_tile(int m);
int svd_threads(int64_t n, int l, bool fp64);
// 0: shared-memory svd; 2 or 4: register-resident svd with that many columns per warp
int svd_variant(int64_t n, int l, bool fp64);
size_t svd_smem(int64_t n, int l, bool fp64);
// The TSQR chain of one svd (plan with Pb > 1) as a job and its four stages
// (kind, blocks, dynamic shared memory), in launch order; returns the flag
// of its launches.
struct TsqrStage {
  int kind;
  uint32_t blocks;
  size_t smem;
};
int tsqr_job(const SmallPlan& pl, bool fp64, const double* Y, int64_t n, double* Q,
             double* sigma, void* scratch, int shift_rule, bool update_shift, bool basis_only,
             double* alpha, double* ahist, double* shist, int* status, TsqrJob* job,
             TsqrStage stages[4]);
int polish_blocks(int64_t n);
size_t gram_smem(int r);
size_t polish_smem(int r);

#ifdef __CUDACC__
// Launch a work-list kernel on a persistent grid: as many CTAs as fit on the
// GPU at once, but no more than there are blocks of work.
template <typename Job>
cudaError_t run_batch(void (*kern)(const Job*, const uint32_t*, int, uint32_t),
                      const BatchLaunch& b, int threads, cudaStream_t st) {
  if (b.total == 0 || b.njobs == 0) return cudaSuccess;
  int per = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, b.smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const uint64_t cap = (uint64_t)per * (uint64_t)num_sms();
  const unsigned grid = (unsigned)(b.total < cap ? b.total : cap);
  count_kernels(1);
  kern<<<grid, threads, b.smem, st>>>((const Job*)b.jobs, b.start, b.njobs, b.total);
  return cudaGetLastError();
}
#endif

}  // namespace tk
