// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "tucker.h"

namespace tk {

// Mode-k view of a column-major tensor: X(p, i, s) at p + P*(i + n*s), with
// P = n_1..n_{k-1}, n = n_k, S = n_{k+1}..n_d.  Column j of the unfolding
// X_(k) is j = p + P*s (Kolda order).
struct View {
  int64_t P, n, S;
  int64_t cols() const { return P * S; }
};

enum XType { X_F64 = 0, X_F32 = 1, X_BF16 = 2 };

inline size_t xsize(XType t) { return t == X_F64 ? 8 : (t == X_F32 ? 4 : 2); }
inline size_t asize(XType t) { return t == X_F64 ? 8 : 4; }  // accumulation type

int num_sms();
// Split-K count of an FP32 CUDA-core product of shape class (kind, n,
// width, columns): the tuned value when tuning is on and the class is in the
// table (or a tuning run's candidate), else `heuristic`; clamped to
// [1, maxs].  kind: TUNE_XB32 (Y = X W splits columns), TUNE_XTB32 (the TTM
// splits rows).
enum { TUNE_XB32 = 0, TUNE_XTB32 = 1 };
int tune_splits(int kind, int64_t n, int width, int64_t cols, int heuristic, int maxs);

// ---- instrumentation (tucker_api.cu) --------------------------------------
// Counts kernel launches always; when profiling is on, brackets the scope
// with CUDA events on `st` and records the algorithmic bytes and flops.
void count_kernels(int n);
struct ProfScope {
  ProfScope(int kind, double bytes, double flops, cudaStream_t st);
  ~ProfScope();
  int idx;
  cudaStream_t st;
};

// ---- contraction kernels (k_contract.cu) ---------------------------------
// Partial products Y_part[split][i][c] of Y = X_(k) B with B = Omega_k
// (generated) or B = W stored in the (P, l, S) layout.  Returns the number
// of splits used; part must hold splits*n*lc accumulation-type values.
int xb_splits(XType xt, View v, int l);
int xb_lc(int l);
// FP32 mode-major (P == 1) register-tiled versions (k_contract32.cu), used
// by launch_xb / launch_xtb when they apply.
bool xtb32_ok(XType xt, View v, const void* X);
// tout: write out[j + cols*c] (the contracted mode moves last) instead of
// out[c + m*j].  ka, kb: Omega's row for layout column j is j/ka + kb*(j%ka)
// (ka = 0: the natural layout, row j).
// scratch (may be NULL): xtb32_scratch bytes; lets few-column products split
// their rows over more CTAs and holds B rounded to FP32 once.
// B32 (may be NULL): B already in FP32 with the same strides (then B is
// not read).
// comp: slab-compensated sums over the rows (the TTM: its output is the next
// mode's tensor and the core).
cudaError_t launch_xtb32(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                         int m, void* out, cudaStream_t st, int tout = 0,
                         void* scratch = nullptr, const float* B32 = nullptr,
                         bool comp = false);
size_t xtb32_scratch(View v, int m);
// W = X_(k)^T B in 3xTF32 on tcgen05 tensor cores (k_tc32.cu), for an FP32
// mode-major view with n_k % 4 == 0 and m <= 64.  out_mode 0: out[c + m j];
// 1: out[j + cols c]; 2: the planes out[c][j] = hi(w), out[64 + c][j] = lo(w)
// with row stride ld (the B operand of the tensor-core Y = X W).  scratch:
// tc32_xtb_scratch(v) bytes (B split into hi/lo planes).  err: device status
// word (TK_ETIMEOUT if a wait ran out).
bool tc32_ok(View v, int m, const void* X);
size_t tc32_xtb_scratch(View v);
cudaError_t launch_tc32_xtb(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                            int m, float* out, int out_mode, int64_t ld, void* scratch, int* err,
                            cudaStream_t st);

// offset of the FP32 copy of B inside that scratch
size_t xtb32_b32_offset(View v, int m);
// FP32 last-mode expansion fused with the error sums (S == 1): err_part gets
// err32_blocks(v, m) (e^2, a^2) pairs.
bool err32_ok(XType xt, View v);
int err32_blocks(View v, int m);
// the row-tile error pass applies (K = v.n small enough) and its dynamic
// shared memory
bool err32c_ok(View v);
size_t err32c_smem(int K);
cudaError_t launch_err32(const void* T, View v, const double* B, int64_t b_ri, int64_t b_cm,
                         int m, const void* A, double* err_part, cudaStream_t st,
                         const float* B32 = nullptr);
// shadow (sketch only, may be NULL): also write the bfloat16 copy of X
// (round to nearest even) in the same pass.
cudaError_t launch_xb32(const void* X, View v, const void* W, int l, uint64_t seed, uint32_t tag,
                        int mode, void* part, int splits, cudaStream_t st, int64_t ka = 0,
                        int64_t kb = 1, void* part_lo = nullptr, void* shadow = nullptr);
// ka, kb: Omega row map of a rotated layout (see launch_xb32; FP32
// mode-major views only; ka = 0 is the natural layout).
// part_lo (FP32 mode-major Y = X W only): compensated accumulation, the
// partials as (hi in part, lo in part_lo) pairs.
cudaError_t launch_xb(XType xt, const void* X, View v, const void* W, int l, uint64_t seed,
                      uint32_t tag, int mode, void* part, int splits, cudaStream_t st,
                      int64_t ka = 0, int64_t kb = 1, void* part_lo = nullptr);
// Y = sum_split part - alpha*Q (Q, alpha may be NULL): n x l FP64.
// part_lo: optional second plane of partials added to the first.
cudaError_t launch_reduce(XType xt, const void* part, int splits, int64_t n, int l, int lc,
                          const double* Q, const double* alpha, double* Y, cudaStream_t st,
                          const void* part_lo = nullptr);
// out(P, m, S) = X x_k B^T with B(i, c) at B[i*b_ri + c*b_cm] (FP64):
// out[j, c] = sum_i X(p, i, s) B(i, c).  Output in the accumulation type of
// X (or `out_bf16` when non-null: BF16 output is not supported here).
// tout = 1 (FP32 mode-major views only): out[j + cols*c] instead of the
// (P, m, S) layout.
// B32 (may be NULL): B in FP32 with the same strides, used by the FP32
// mode-major kernels.
cudaError_t launch_xtb(XType xt, const void* X, View v, const double* B, int64_t b_ri,
                       int64_t b_cm, int m, void* out, cudaStream_t st, int tout = 0,
                       void* scratch = nullptr, const float* B32 = nullptr,
                       bool comp = false);
// Fused last-mode expansion and error sums: for S == 1, a_hat(p, c) =
// sum_i T(p, i) B(i, c); accumulates (A - a_hat)^2 and A^2 per block into
// err_part[2*block].  Returns the number of blocks via *blocks.
cudaError_t launch_xtb_error(XType xt, const void* T, View v, const double* B, int64_t b_ri,
                             int64_t b_cm, int m, const void* A, double* err_part, int* blocks,
                             cudaStream_t st, const float* B32 = nullptr);
int xtb_error_blocks(XType xt, View v, int m);
cudaError_t launch_error_final(const double* err_part, int blocks, double* rel_err,
                               cudaStream_t st);

// ---- fused bfloat16 power step on tcgen05 (k_power_tc.cu) ------------------
// Y_part = X_(k)(X_(k)^T Q) for a mode-major (P == 1) bfloat16 view.  The
// partials are [groups][n][l_pad] FP32 (l_pad = l rounded up to 32); sum them
// with launch_reduce(X_BF16, part, groups, n, l, l_pad, ...).  scratch holds
// the bfloat16 Q^T operand (power_tc_scratch bytes).
bool power_tc_supported(View v, int l, const void* X);
int power_tc_groups(View v, int l);
size_t power_tc_scratch(View v, int l);
int power_tc_lpad(View v, int l);   // row stride of the partials
cudaError_t launch_power_tc(const void* X, View v, const double* Q, int l, void* scratch,
                            float* part, int groups, int* err, cudaStream_t st);

// ---- small dense solver (k_small.cu) -------------------------------------
// [Q, Sigma] = svd(Y, 'econ') of an n x l FP64 matrix by a two-level
// Householder TSQR, one-sided Jacobi on the l x l triangle, and the sign
// convention; optional shift update.  `T` selects the working precision.
// basis_only: Q = any orthonormal basis of span(Y) (Householder Q), no Sigma
// (used where only the span matters: the sketch before a power step).
struct SmallPlan {
  int l, MB, Pb;
  size_t scratch_bytes;
  int reg;   // register-resident FP32 kernels
};
SmallPlan small_plan(int64_t n, int l, bool fp64);
cudaError_t launch_small_svd(bool fp64, const SmallPlan& pl, const double* Y, int64_t n,
                             double* Q, double* sigma, void* scratch, int shift_rule,
                             bool update_shift, double* alpha, double* alpha_hist,
                             double* sigl_hist, int* status, cudaStream_t st,
                             bool basis_only = false);

// One CholeskyQR step (U <- U R^{-1}, R^T R = U^T U) to first order on an
// n x r FP64 factor computed in FP32 arithmetic; scratch: polish_scratch(n, r)
// bytes.
size_t polish_scratch(int64_t n, int r);
cudaError_t launch_polish(double* U, int64_t n, int r, void* scratch, int* status,
                          cudaStream_t st);

// Rayleigh-Ritz rotation of W = X^T Q in place (precision form, before its
// FP32 step Y = X W): G = W^T W, Z = eigenvectors of G by descending
// eigenvalue, W <- W Z.  W holds cols x l FP32 entries in the (P, l, S)
// layout the products use (entry (j, c) at j % P + P (c + l (j / P))).
// scratch: ritz_scratch(l) bytes.
size_t ritz_scratch(int l);
cudaError_t launch_ritz_rotate(float* W, int64_t cols, int64_t P, int l, void* scratch,
                               int* status, cudaStream_t st);

// ---- misc (k_misc.cu) -----------------------------------------------------
cudaError_t launch_omega(int k, int64_t row0, int64_t rows, int l, uint64_t seed, uint32_t tag,
                         float* out, cudaStream_t st);
cudaError_t launch_to_bf16(const float* x, int64_t count, uint16_t* out, cudaStream_t st);
// Structured test matrices (tk_omega): the modes m != k of a tensor with
// sizes dims, in ascending order, with their sizes and the offsets (floats)
// of their Khatri-Rao factors in the scratch (rows padded to l rounded up
// to 4).
struct OmegaGeom {
  int nf;
  int mode[TK_MAX_D];
  int64_t size[TK_MAX_D];
  int64_t off[TK_MAX_D + 1];
};
OmegaGeom omega_geom(const int64_t* dims, int d, int k, int l);
// Scratch bytes launch_omega_fill needs for kind (0 for the dense kinds).
size_t omega_scratch(int kind, const int64_t* dims, int d, int k, int l);
// Writes Omega_k of the given kind for the unfolding's columns in the
// layout's order (jk = j / ka + kb (j % ka); ka <= 0: the natural order):
// P >= 1 the (P, l, S) W layout of the products, P = 0 column-major; FP64
// (f64) or FP32 values.  kr: omega_scratch bytes (Khatri-Rao kinds).
cudaError_t launch_omega_fill(int kind, const int64_t* dims, int d, int k, int l, uint64_t seed,
                              uint32_t tag, int64_t ka, int64_t kb, float* kr, void* out,
                              bool f64, int64_t P, cudaStream_t st);
// dst (rows x cols, ld_dst) = src (FP64, ld_src) converted to dtype.
cudaError_t launch_copy_matrix(const double* src, int64_t ld_src, void* dst, int64_t ld_dst,
                               int64_t rows, int64_t cols, XType dt, cudaStream_t st);
cudaError_t launch_copy_tensor(const void* src, void* dst, int64_t count, XType dt,
                               cudaStream_t st);
cudaError_t launch_to_f64_from_f32(const float* x, int64_t count, double* y, cudaStream_t st);
// Holistic variants: M (n x n) = B_(k) B_(k)^T of an FP64 tensor's strided
// view; U (n x r, dt) = Q (n x l) V (l x r), FP64 sums.
cudaError_t launch_gram_unfold(const double* B, View v, double* M, cudaStream_t st);
cudaError_t launch_qv(const double* Q, int64_t n, int l, const double* V, int r, void* U,
                      XType dt, cudaStream_t st);
cudaError_t launch_check_finite(const double* x, int64_t count, int* status, cudaStream_t st);

}  // namespace tk
