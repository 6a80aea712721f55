// C ABI and host orchestration of Algorithms 2 (shifted randomized
// T-HOSVD) and 3 (shifted randomized ST-HOSVD).  Control stays on the host
// only for launches: the shift alpha, Q, Sigma and Y live on the device and
// no device-to-host copy happens inside the mode loop.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <mutex>
#include <deque>
#include <vector>

#include "tk_common.cuh"
#include "tk_internal.h"
#include "tk_batch.h"
#include "tk_plan.h"

namespace tk {

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached = n > 0 ? n : 1;
  }
  return cached;
}

// ---------------------------------------------------------------------------
// Instrumentation: launch counter and optional per-scope CUDA-event timing.
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  int kind;
  double bytes, flops;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<int64_t> g_kernels{0};

cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void count_kernels(int n) { g_kernels.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(int kind, double bytes, double flops, cudaStream_t s) : idx(-1), st(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  ProfRec r{kind, bytes, flops, pool_event(), pool_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  idx = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (idx < (int)g_recs.size()) cudaEventRecord(g_recs[idx].b, st);
}

// ---------------------------------------------------------------------------
// Plan of one tucker_rthosvd / tucker_rsthosvd call.
// ---------------------------------------------------------------------------
tk_status make_plan(const tk_tensor* A, const int* r, const tk_opts* o, bool st,
                    HosvdPlan& p, bool full_ok) {
  if (!valid_tensor(A, false) || !r || !o) return TK_EINVAL;
  p.d = A->d;
  p.st = st;
  p.xt = xtype(A->dtype);
  p.n.assign(A->n, A->n + A->d);
  p.r.assign(r, r + A->d);
  p.s.assign(o->s, o->s + A->d);
  p.q = o->q;
  p.rule = o->shift;
  p.bf16 = o->prec == TK_PREC_BF16_POWER;
  if (o->q < 0 || o->q > TK_MAX_Q) return TK_EINVAL;
  if (o->tag >= (1u << 24)) return TK_EINVAL;
  if (o->shift != TK_SHIFT_PAPER && o->shift != TK_SHIFT_NONE) return TK_EINVAL;
  if (o->prec != TK_PREC_PLAIN && o->prec != TK_PREC_BF16_POWER) return TK_EINVAL;
  if (p.bf16 && A->dtype != TK_F32) return TK_EINVAL;
  if (o->omega < TK_OMEGA_GAUSS || o->omega > TK_OMEGA_KR_UNIFORM) return TK_EINVAL;
  p.omega = o->omega;
  for (int k = 0; k < p.d; ++k) {
    if (p.r[k] < 1 || p.r[k] > p.n[k]) return TK_EINVAL;
    if (p.r[k] == p.n[k] && !full_ok) return TK_EINVAL;      // Problem 2.1: r_k < n_k
    if (p.s[k] < 0) return TK_EINVAL;
  }
  if (o->order[0] == TK_ORDER_DESCENDING) {
    // the processing order of Section 3.2: n_{p_1} >= n_{p_2} >= ... >= n_{p_d}
    // (ties in ascending mode index)
    p.order.resize(p.d);
    for (int k = 0; k < p.d; ++k) p.order[k] = k;
    std::stable_sort(p.order.begin(), p.order.end(),
                     [&](int a, int b) { return p.n[a] > p.n[b]; });
    if (!st)
      for (int k = 0; k < p.d; ++k) p.order[k] = k;   // T-HOSVD: order is immaterial
  } else if (o->order[0] < 0) {
    p.order.resize(p.d);
    for (int k = 0; k < p.d; ++k) p.order[k] = k;
  } else {
    p.order.assign(o->order, o->order + p.d);
    std::vector<int> seen(p.d, 0);
    for (int k = 0; k < p.d; ++k) {
      if (p.order[k] < 0 || p.order[k] >= p.d || seen[p.order[k]]) return TK_EINVAL;
      seen[p.order[k]] = 1;
    }
    if (!st)
      for (int k = 0; k < p.d; ++k) p.order[k] = k;   // T-HOSVD: order is immaterial
  }
  bool natural = true;
  for (int k = 0; k < p.d; ++k) natural = natural && p.order[k] == k;
  p.rot = st && natural && p.xt == X_F32;
  const size_t es = xsize(p.xt), ta = asize(p.xt);
  p.l.assign(p.d, 0);
  p.sp.assign(p.d, SmallPlan{});
  p.dims_at.assign(p.d, {});
  std::vector<int64_t> cur = p.n;
  for (int step = 0; step < p.d; ++step) {
    const int k = p.order[step];
    p.dims_at[k] = cur;
    int64_t ka, kb;
    const View v = step_view(p, cur, k, &ka, &kb);
    const int64_t cols = v.cols();
    const int64_t lk = std::min<int64_t>({(int64_t)p.r[k] + p.s[k], v.n, cols});
    if (lk < p.r[k]) return TK_EINVAL;        // U_k = Q(:, 1:r_k) needs l_k >= r_k
    if (lk > TK_MAX_L) return TK_ENOTIMPL;
    p.l[k] = (int)lk;
    p.sp[k] = small_plan(v.n, (int)lk, p.xt == X_F64);
    if (p.sp[k].Pb <= 0) return TK_ENOTIMPL;
    p.small = std::max(p.small, p.sp[k].scratch_bytes);
    // the tensor-core W = X^T Q splits Q into that scratch; the tensor-core
    // sketch writes its column-group partials into the partial buffer
    if (p.xt == X_F32 && v.P == 1 && (v.n % 4) == 0 && lk <= 64) {
      if (p.q > 0) p.small = std::max(p.small, tc32_xtb_scratch(v));
      p.part = std::max(p.part, tc32_sketch_part_bytes(v));
    }
    if (p.xt != X_F64) p.small = std::max(p.small, polish_scratch(v.n, p.r[k]));
    const int lc = xb_lc((int)lk);
    const int splits = xb_splits(p.xt, v, (int)lk);
    // the power steps' Y = X W on FP32 mode-major views keep (hi, lo) partial pairs
    const bool comp_y = p.q >= 1 && xtb32_ok(p.xt, v, (const void*)1);
    p.part = std::max(p.part, (size_t)splits * v.n * lc * ta * (comp_y ? 2 : 1));
    if (p.bf16 && p.q >= 2) p.part = std::max(p.part, ritz_scratch((int)lk));
    if (xtb32_ok(p.xt, v, (const void*)1)) {   // row-split scratch of W = X^T Q and the TTM
      p.part = std::max(p.part, xtb32_scratch(v, (int)lk));
      p.part = std::max(p.part, xtb32_scratch(v, p.r[k]));
    }
    // W holds the power steps' X^T Q, and Omega_k when it is not generated
    // inside the sketch pass
    if (p.q > 0 || p.omega != TK_OMEGA_GAUSS) p.wbuf = std::max(p.wbuf, (size_t)cols * lk * ta);
    p.kr = std::max(p.kr, omega_scratch(p.omega, cur.data(), p.d, k, (int)lk));
    p.ymat = std::max(p.ymat, (size_t)v.n * lk * sizeof(double));
    if (p.bf16 && p.q >= 2) {
      p.shadow = std::max(p.shadow, (size_t)prod(cur) * 2);
      if (v.P == 1) {   // the fused tensor-core pass may run on this mode
        p.part = std::max(p.part, (size_t)power_tc_groups(v, (int)lk) * v.n *
                                      power_tc_lpad(v, (int)lk) * sizeof(float));
        p.small = std::max(p.small, power_tc_scratch(v, (int)lk));
      }
    }
    if (st) {
      cur[k] = p.r[k];
      if (step < p.d - 1) p.gbuf = std::max(p.gbuf, (size_t)prod(cur) * es);
    }
  }
  if (!st) {
    std::vector<int64_t> c2 = p.n;
    for (int k = 0; k < p.d - 1; ++k) {
      c2[k] = p.r[k];
      p.gbuf = std::max(p.gbuf, (size_t)prod(c2) * es);
    }
    for (int k = 0; k < p.d; ++k) p.qd += al((size_t)p.n[k] * p.r[k] * sizeof(double));
  }
  return TK_OK;
}

// T-HOSVD factors its modes concurrently (one stream each), so every mode
// gets its own W, partials, Y, Q, small-solver scratch and shift; ST-HOSVD
// (sequential by definition) lays out one set.  ws (when given) receives
// workspace_copies(p) entries.
int workspace_copies(const HosvdPlan& p) { return p.st ? 1 : p.d; }

size_t carve(const HosvdPlan& p, unsigned char* base, HosvdWs* ws) {
  Arena a;
  a.base = base;
  HosvdWs w{};
  w.g[0] = a.take(p.gbuf);
  w.g[1] = a.take(p.gbuf);
  w.shadow = a.take(p.shadow);
  w.qd = (double*)a.take(p.qd);
  w.ahist = (double*)a.take(sizeof(double) * TK_MAX_D * TK_MAX_Q);
  w.shist = (double*)a.take(sizeof(double) * TK_MAX_D * TK_MAX_Q);
  w.sig = (double*)a.take(sizeof(double) * TK_MAX_D * TK_MAX_L);
  w.status = (int*)a.take(sizeof(int));
  const int copies = workspace_copies(p);
  for (int c = 0; c < copies; ++c) {
    HosvdWs m = w;
    m.w = a.take(p.wbuf);
    m.part = a.take(p.part);
    m.Y = (double*)a.take(p.ymat);
    m.Q = (double*)a.take(p.ymat);
    m.small = a.take(p.small);
    m.alpha = (double*)a.take(sizeof(double));
    m.kr = (float*)a.take(p.kr);
    if (ws) ws[c] = m;
  }
  return al(a.off) + 256;
}

// Sketch, q shifted power steps and the final svd for mode k of X
// (Algorithm 2/3 steps for one k).  Leaves Q (n x l) and Sigma in ws.
// shadow_ready: the bfloat16 copy of X is already in w.shadow (T-HOSVD
// converts A once for all modes).
// PVE control (Algorithm 4): stop the power steps when the estimates settle.
struct PveCtl {
  double tol = -1.0;   // < 0: run all p.q steps (Algorithms 2, 3)
  int q_used = 0;      // out: steps run
};

static tk_status factor_mode(const HosvdPlan& p, int k, const void* X, XType xt, View v,
                             int64_t ka, int64_t kb, uint64_t seed, uint32_t tag,
                             const HosvdWs& w, cudaStream_t st, bool shadow_ready = false,
                             PveCtl* pve = nullptr) {
  const int l = p.l[k];
  const int lc = xb_lc(l);
  const int splits = xb_splits(xt, v, l);
  const bool fp64 = xt == X_F64;
  double* sig = w.sig + (size_t)k * TK_MAX_L;
  const double N = (double)v.P * (double)v.n * (double)v.S;
  const double nl = (double)v.n * l;
  const double red_bytes = (double)splits * v.n * lc * asize(xt) + nl * 8.0;
  const double svd_flops = 4.0 * nl * l + 2.0 * (double)l * l * l;
  const bool dense_gauss = p.omega == TK_OMEGA_GAUSS;
  const double om_bytes = dense_gauss ? 0.0 : (double)v.cols() * l * asize(xt);
  if (!dense_gauss) {
    // the structured test matrices (Section 5.5) are written out into W
    ProfScope ps(TK_K_SKETCH, om_bytes, 0.0, st);
    TK_TRY(launch_omega_fill(p.omega, p.dims_at[k].data(), p.d, k, l, seed, tag, ka, kb, w.kr,
                             w.w, fp64, v.P, st));
  }
  // precision form on an FP32 mode-major view: the sketch pass writes the
  // bfloat16 copy of X as it reads X (no separate conversion pass)
  const bool fuse_shadow = p.bf16 && p.q >= 2 && !shadow_ready && dense_gauss &&
                           xtb32_ok(xt, v, X);
  // FP32 mode-major views with Gaussian Omega: the sketch on the tensor cores
  Tc32SketchJob skj;
  const bool tc_sketch = xt == X_F32 && dense_gauss &&
                         tc32_sketch_job(X, v, l, seed, tag, k, ka, kb, (float*)w.part, w.status,
                                         fuse_shadow ? w.shadow : nullptr, &skj);
  {
    ProfScope ps(TK_K_SKETCH, N * xsize(xt) + om_bytes + (fuse_shadow ? N * 2.0 : 0.0),
                 2.0 * N * l, st);
    if (tc_sketch)
      TK_TRY(launch_tc32_sketch(skj, st));
    else if (fuse_shadow)
      TK_TRY(launch_xb32(X, v, nullptr, l, seed, tag, k, w.part, splits, st, ka, kb, nullptr,
                         w.shadow));
    else
      TK_TRY(launch_xb(xt, X, v, dense_gauss ? nullptr : w.w, l, seed, tag, k, w.part, splits,
                       st, ka, kb));
  }
  {
    const int sp = tc_sketch ? skj.groups : splits;
    const int slc = tc_sketch ? 64 : lc;
    ProfScope ps(TK_K_CONVERT, (double)sp * v.n * slc * asize(xt) + nl * 8.0, (double)sp * nl,
                 st);
    TK_TRY(launch_reduce(xt, w.part, sp, v.n, l, slc, nullptr, nullptr, w.Y, st));
  }
  TK_TRY(cudaMemsetAsync(w.alpha, 0, sizeof(double), st));
  {
    ProfScope ps(TK_K_SMALL_SVD, 2.0 * nl * 8.0, svd_flops, st);
    // before an FP32 (or FP64) power step only span(Y) matters (alpha_0 = 0
    // needs no Sigma), so the sketch's svd reduces to an orthonormal basis.
    // Before a bfloat16 power step the singular-vector basis is kept: its
    // columns are graded by sigma, so rounding Q and W to bfloat16 perturbs
    // each direction relative to its own size (an arbitrary basis of the span
    // spreads the large directions' rounding into the small ones: measured at
    // 1000^3, RE 1.0198e-6 against 1.0163e-6).
    const bool basis_only = p.q >= 1 && !(p.bf16 && p.q >= 2);
    TK_TRY(launch_small_svd(fp64, p.sp[k], w.Y, v.n, w.Q, sig, w.small, (int)p.rule, false,
                            w.alpha, nullptr, nullptr, w.status, st, basis_only));
  }
  if (p.bf16 && p.q >= 2 && !shadow_ready && !fuse_shadow) {
    ProfScope ps(TK_K_CONVERT, N * 6.0, 0.0, st);
    TK_TRY(launch_to_bf16((const float*)X, v.P * v.n * v.S, (uint16_t*)w.shadow, st));
  }
  std::vector<double> sig_hat(pve ? l : 0, 0.0), sig_h(pve ? l : 0);
  double alpha_prev = 0.0;
  if (pve) pve->q_used = p.q;
  for (int t = 1; t <= p.q; ++t) {
    const bool low = p.bf16 && t < p.q;
    // precision form: the FP32 step after the bfloat16 ones
    const bool last32 = p.bf16 && p.q >= 2 && t == p.q;
    const void* Xp = low ? w.shadow : X;
    const XType xp = low ? X_BF16 : xt;
    // precision form: the shift sequence restarts when the step switches
    // from the bfloat16 copy to the FP32 tensor (the bfloat16 Sigma(l,l)
    // sits on the copy's rounding floor, far above sigma_l(X X^T)/2)
    if (last32) TK_TRY(cudaMemsetAsync(w.alpha, 0, sizeof(double), st));
    if (low && power_tc_supported(v, l, Xp)) {
      // one fused tensor-core pass over the bfloat16 copy
      const int groups = power_tc_groups(v, l);
      const int lp = power_tc_lpad(v, l);
      {
        ProfScope ps(TK_K_POWER_FUSED, N * 2.0, 4.0 * N * l, st);
        TK_TRY(launch_power_tc(Xp, v, w.Q, l, w.small, (float*)w.part, groups, w.status, st));
      }
      {
        ProfScope ps(TK_K_CONVERT, (double)groups * v.n * lp * 4.0 + nl * 8.0,
                     (double)groups * nl, st);
        TK_TRY(launch_reduce(X_BF16, w.part, groups, v.n, l, lp, w.Q, w.alpha, w.Y, st));
      }
    } else {
      {
        ProfScope ps(TK_K_POWER_W, N * xsize(xp), 2.0 * N * l, st);
        if (xp == X_F32 && tc32_ok(v, l, Xp)) {
          // W = X^T Q in 3xTF32 on the tensor cores (Q split into the small
          // solver's scratch, which the svd only needs after this step)
          TK_TRY(launch_tc32_xtb(Xp, v, w.Q, 1, v.n, l, (float*)w.w, 0, 0, w.small, w.status,
                                 st));
        } else {
          TK_TRY(launch_xtb(xp, Xp, v, w.Q, 1, v.n, l, w.w, st, 0, w.part));
        }
      }
      // The precision form's FP32 step has to resolve the weak directions
      // the bfloat16 steps left inexact, to the FP32 path's accuracy:
      //  * Q's weak columns carry components along the leading directions at
      //    the copy's rounding level; in Y = X W these dominate the weak
      //    columns and FP32 rounding of them buries the weak directions, so W
      //    is first rotated to the Ritz vectors (Y Z = X (W Z) spans the same
      //    subspace, alpha = 0 at this step);
      //  * the sums of Y = X W over the unfolding's columns are compensated
      //    (slab sums folded into (hi, lo) pairs).
      if (last32) {
        const double cw = (double)v.cols() * l;
        ProfScope ps(TK_K_RITZ, 3.0 * cw * 4.0, 4.0 * cw * l, st);
        TK_TRY(launch_ritz_rotate((float*)w.w, v.cols(), v.P, l, w.part, w.status, st));
      }
      // Y = X W on FP32 mode-major views: compensated sums (slab sums folded
      // into (hi, lo) pairs), so the weak directions of the iterate are not
      // lost under the rounding of sums over the unfolding's ~N/n columns
      void* plo = nullptr;
      if (xtb32_ok(xp, v, Xp))
        plo = (unsigned char*)w.part + (size_t)splits * v.n * lc * asize(xp);
      {
        ProfScope ps(TK_K_POWER_Y, N * xsize(xp), 2.0 * N * l, st);
        TK_TRY(launch_xb(xp, Xp, v, w.w, l, seed, tag, k, w.part, splits, st, 0, 1, plo));
      }
      {
        ProfScope ps(TK_K_CONVERT, red_bytes, (double)splits * nl, st);
        TK_TRY(launch_reduce(xp, w.part, splits, v.n, l, lc, w.Q, w.alpha, w.Y, st, plo));
      }
    }
    {
      ProfScope ps(TK_K_SMALL_SVD, 2.0 * nl * 8.0, svd_flops, st);
      TK_TRY(launch_small_svd(fp64, p.sp[k], w.Y, v.n, w.Q, sig, w.small, (int)p.rule, true,
                              w.alpha, w.ahist + (size_t)k * TK_MAX_Q + (t - 1),
                              w.shist + (size_t)k * TK_MAX_Q + (t - 1), w.status, st));
    }
    if (pve) {
      // Algorithm 4's test on sigma_t = diag(Sigma) + alpha_{t-1}; the svd
      // has already applied the shift update, which only matters if the
      // loop goes on
      double alpha_new = 0.0;
      TK_TRY(cudaMemcpyAsync(sig_h.data(), sig, (size_t)l * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(&alpha_new, w.alpha, sizeof(double), cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaStreamSynchronize(st));
      const int r = p.r[k];
      double dmax = 0.0;
      for (int i = 0; i < l; ++i) sig_h[i] += alpha_prev;
      for (int i = 0; i < r; ++i) dmax = std::max(dmax, std::fabs(sig_h[i] - sig_hat[i]));
      const double thr = pve->tol * sig_h[std::min(r, l - 1)];
      if (dmax <= thr) {
        pve->q_used = t;
        break;
      }
      alpha_prev = alpha_new;
      sig_hat = sig_h;
    }
  }
  return TK_OK;
}

// TTM shrink G <- G x_k U_k^T with U_k = Q(:, 1:r_k) (Algorithm 2/3, last
// step of each k), instrumented.
// U32: the same factor in FP32 (the returned U_k of an FP32 tensor), or NULL.
static cudaError_t ttm(XType xt, const void* X, View v, const double* U, int r, void* out,
                       cudaStream_t st, int tout = 0, void* scratch = nullptr,
                       const void* U32 = nullptr) {
  const double N = (double)v.P * (double)v.n * (double)v.S;
  ProfScope ps(TK_K_TTM, (N + N / v.n * r) * xsize(xt), 2.0 * N * r, st);
  return launch_xtb(xt, X, v, U, 1, v.n, r, out, st, tout, scratch,
                    xt == X_F32 ? (const float*)U32 : nullptr, /*comp=*/true);
}

static cudaError_t polish(double* Q, int64_t n, int r, void* scratch, int* status,
                          cudaStream_t st) {
  ProfScope ps(TK_K_CONVERT, 2.0 * n * r * 8.0, 2.0 * n * r * r, st);
  return launch_polish(Q, n, r, scratch, status, st);
}

// Per-host-thread, per-device side streams and fork/join events for the
// concurrent T-HOSVD modes (created on first use, kept for the process).
struct SideStreams {
  int dev = -1;
  cudaStream_t s[TK_MAX_D] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[TK_MAX_D] = {};
};

static SideStreams& side_streams(int d) {
  thread_local std::deque<SideStreams> pool;   // stable addresses
  int dev = 0;
  cudaGetDevice(&dev);
  for (auto& e : pool)
    if (e.dev == dev) return e;
  pool.emplace_back();
  SideStreams& e = pool.back();
  e.dev = dev;
  cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming);
  for (int k = 1; k < TK_MAX_D; ++k) {
    cudaStreamCreateWithFlags(&e.s[k], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&e.join[k], cudaEventDisableTiming);
  }
  (void)d;
  return e;
}

static tk_status run_hosvd(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                           void* const* U, tk_stats* stats, cudaStream_t st, bool sequential,
                           double pve_tol = -1.0, int* q_out = nullptr) {
  HosvdPlan p;
  tk_status s = make_plan(A, r, o, sequential, p);
  if (s != TK_OK) return s;
  if (!core || !U) return TK_EINVAL;
  for (int k = 0; k < p.d; ++k)
    if (!U[k]) return TK_EINVAL;
  const size_t need = carve(p, nullptr, nullptr);
  unsigned char* base = (unsigned char*)o->workspace;
  bool owned = false;
  if (base == nullptr) {
    TK_TRY(cudaMallocAsync((void**)&base, need, st));
    owned = true;
  } else if (o->workspace_bytes < need) {
    return TK_EWORKSPACE;
  }
  HosvdWs wm[TK_MAX_D];
  carve(p, (unsigned char*)(((uintptr_t)base + 255) & ~(uintptr_t)255), wm);
  const HosvdWs& w = wm[0];
  tk_status rs = TK_OK;
  auto run = [&]() -> tk_status {
    TK_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    TK_TRY(cudaMemsetAsync(w.ahist, 0, sizeof(double) * TK_MAX_D * TK_MAX_Q, st));
    TK_TRY(cudaMemsetAsync(w.shist, 0, sizeof(double) * TK_MAX_D * TK_MAX_Q, st));
    TK_TRY(cudaMemsetAsync(w.sig, 0, sizeof(double) * TK_MAX_D * TK_MAX_L, st));
    const size_t es = xsize(p.xt);
    if (p.st) {
      const void* X = A->data;
      std::vector<int64_t> cur = p.n;
      int pp = 0;
      for (int step = 0; step < p.d; ++step) {
        const int k = p.order[step];
        int64_t ka, kb;
        const View v = step_view(p, cur, k, &ka, &kb);
        PveCtl pve;
        pve.tol = pve_tol;
        tk_status e = factor_mode(p, k, X, p.xt, v, ka, kb, o->seed, o->tag, w, st, false,
                                  pve_tol >= 0.0 ? &pve : nullptr);
        if (e != TK_OK) return e;
        if (q_out) q_out[k] = pve_tol >= 0.0 ? pve.q_used : p.q;
        if (p.xt != X_F64) TK_TRY(polish(w.Q, v.n, p.r[k], w.small, w.status, st));
        TK_TRY(launch_copy_matrix(w.Q, v.n, U[k], v.n, v.n, p.r[k], p.xt, st));
        void* out = (step == p.d - 1) ? core : w.g[pp];
        TK_TRY(ttm(p.xt, X, v, w.Q, p.r[k], out, st, p.rot ? 1 : 0, w.part, U[k]));
        X = out;
        pp ^= 1;
        cur[k] = p.r[k];
      }
    } else {
      // Algorithm 2's modes are independent: each factors on its own stream
      // (forked from and joined back to the call's stream by events)
      size_t off = 0;
      std::vector<double*> qd(p.d);
      if (p.bf16 && p.q >= 2) {
        const double N = (double)prod(p.n);
        ProfScope ps(TK_K_CONVERT, N * 6.0, 0.0, st);
        TK_TRY(launch_to_bf16((const float*)A->data, prod(p.n), (uint16_t*)w.shadow, st));
      }
      SideStreams& ss = side_streams(p.d);
      TK_TRY(cudaEventRecord(ss.fork, st));
      tk_status first = TK_OK;
      for (int k = 0; k < p.d; ++k) {
        qd[k] = (double*)((unsigned char*)w.qd + off);
        off += al((size_t)p.n[k] * p.r[k] * sizeof(double));
        const View v = view_of(p.n, k);
        const HosvdWs& wk = wm[k];
        cudaStream_t sk = k == 0 ? st : ss.s[k];
        if (k > 0) TK_TRY(cudaStreamWaitEvent(sk, ss.fork, 0));
        // with the PVE test the host reads each step back, so the modes
        // then run one after the other
        PveCtl pve;
        pve.tol = pve_tol;
        tk_status e = factor_mode(p, k, A->data, p.xt, v, 0, 1, o->seed, o->tag, wk, sk, true,
                                  pve_tol >= 0.0 ? &pve : nullptr);
        if (q_out) q_out[k] = pve_tol >= 0.0 ? pve.q_used : p.q;
        if (e == TK_OK && p.xt != X_F64) e = from_cuda(polish(wk.Q, v.n, p.r[k], wk.small, wk.status, sk));
        if (e == TK_OK) e = from_cuda(launch_copy_matrix(wk.Q, v.n, qd[k], v.n, v.n, p.r[k], X_F64, sk));
        if (e == TK_OK) e = from_cuda(launch_copy_matrix(wk.Q, v.n, U[k], v.n, v.n, p.r[k], p.xt, sk));
        if (k > 0) {
          // join even after an error, so no side-stream work outlives the call
          cudaError_t j = cudaEventRecord(ss.join[k], sk);
          if (j == cudaSuccess) j = cudaStreamWaitEvent(st, ss.join[k], 0);
          if (e == TK_OK && j != cudaSuccess) e = from_cuda(j);
        }
        if (first == TK_OK) first = e;
        if (e != TK_OK) break;
      }
      if (first != TK_OK) return first;
      // core G = A x_1 U_1^T ... x_d U_d^T (Algorithm 2, last step of each k)
      const void* X = A->data;
      std::vector<int64_t> cur = p.n;
      for (int k = 0; k < p.d; ++k) {
        const View v = view_of(cur, k);
        void* out = (k == p.d - 1) ? core : w.g[k & 1];
        TK_TRY(ttm(p.xt, X, v, qd[k], p.r[k], out, st, 0, nullptr, U[k]));
        X = out;
        cur[k] = p.r[k];
      }
    }
    (void)es;
    if (stats) {
      std::vector<double> ah(TK_MAX_D * TK_MAX_Q), sh(TK_MAX_D * TK_MAX_Q), sg(TK_MAX_D * TK_MAX_L);
      int status = 0;
      TK_TRY(cudaMemcpyAsync(ah.data(), w.ahist, ah.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(sh.data(), w.shist, sh.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(sg.data(), w.sig, sg.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaStreamSynchronize(st));
      std::memset(stats, 0, sizeof(*stats));
      stats->d = p.d;
      stats->q = p.q;
      for (int k = 0; k < p.d; ++k) {
        stats->l[k] = p.l[k];
        stats->order[k] = p.order[k];
        for (int t = 0; t < TK_MAX_Q; ++t) {
          stats->alpha[k][t] = ah[k * TK_MAX_Q + t];
          stats->sigma_l[k][t] = sh[k * TK_MAX_Q + t];
        }
        for (int i = 0; i < TK_MAX_L; ++i) stats->sigma[k][i] = sg[k * TK_MAX_L + i];
      }
      if (status != 0) return (tk_status)status;
    }
    return TK_OK;
  };
  rs = run();
  if (owned) {
    cudaError_t e = cudaFreeAsync(base, st);
    if (rs == TK_OK && e != cudaSuccess) rs = from_cuda(e);
  }
  return rs;
}

// ---------------------------------------------------------------------------
// Holistic variants (Algorithms A.2 and B.1).
// ---------------------------------------------------------------------------
struct HolisticPlan {
  HosvdPlan p;                  // the range finder: ranks r' = l, s' = 0
  std::vector<int> r;           // the requested ranks
  std::vector<SmallPlan> sm;    // svd of each l_k x l_k Gram matrix (FP64)
  size_t qk = 0, bx = 0, b64 = 0, v = 0, small = 0, sig = 0;
};

static tk_status holistic_plan(const tk_tensor* A, const int* r, const tk_opts* o, bool st,
                               HolisticPlan& h) {
  if (!valid_tensor(A, false) || !r || !o) return TK_EINVAL;
  if (o->prec != TK_PREC_PLAIN) return TK_EINVAL;
  const int d = A->d;
  std::vector<int64_t> cur(A->n, A->n + d);
  int rl[TK_MAX_D];
  for (int k = 0; k < d; ++k) {
    if (r[k] < 1 || r[k] >= A->n[k] || o->s[k] < 0) return TK_EINVAL;
    int64_t cols = 1;
    for (int m = 0; m < d; ++m)
      if (m != k) cols *= st ? cur[m] : A->n[m];
    const int64_t lk = std::min<int64_t>({(int64_t)r[k] + o->s[k], A->n[k], cols});
    if (lk < r[k]) return TK_EINVAL;
    if (lk > TK_MAX_L) return TK_ENOTIMPL;
    rl[k] = (int)lk;
    if (st) cur[k] = lk;
  }
  tk_opts o2 = *o;
  for (int k = 0; k < TK_MAX_D; ++k) o2.s[k] = 0;
  o2.order[0] = -1;
  tk_status s = make_plan(A, rl, &o2, st, h.p, true);
  if (s != TK_OK) return s;
  h.r.assign(r, r + d);
  const size_t es = xsize(h.p.xt);
  size_t lprod = 1;
  h.sm.assign(d, SmallPlan{});
  for (int k = 0; k < d; ++k) {
    h.qk += al((size_t)A->n[k] * rl[k] * sizeof(double));
    h.v += al((size_t)rl[k] * r[k] * sizeof(double));
    lprod *= (size_t)rl[k];
    // the eigenvectors need the accuracy of B's own arithmetic: the FP32
    // register svd (then polished) for FP32 tensors, FP64 for FP64
    h.sm[k] = small_plan(rl[k], rl[k], h.p.xt == X_F64);
    if (h.sm[k].Pb <= 0) return TK_ENOTIMPL;
    h.small = std::max(h.small, h.sm[k].scratch_bytes);
    if (h.p.xt != X_F64) h.small = std::max(h.small, polish_scratch(rl[k], r[k]));
  }
  h.bx = lprod * es;
  h.b64 = lprod * sizeof(double);
  h.sig = TK_MAX_L * sizeof(double);
  return TK_OK;
}

static size_t holistic_bytes(const HolisticPlan& h) {
  return carve(h.p, nullptr, nullptr) + 256 + al(h.qk) + al(h.bx) + 2 * al(h.b64) + al(h.v) +
         al(h.small) + al(h.sig) + 1024;
}

static tk_status run_holistic(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                              void* const* U, tk_stats* stats, cudaStream_t st, bool sequential) {
  HolisticPlan h;
  tk_status s = holistic_plan(A, r, o, sequential, h);
  if (s != TK_OK) return s;
  const HosvdPlan& p = h.p;
  if (!core || !U) return TK_EINVAL;
  for (int k = 0; k < p.d; ++k)
    if (!U[k]) return TK_EINVAL;
  const size_t need = holistic_bytes(h);
  unsigned char* base = (unsigned char*)o->workspace;
  bool owned = false;
  if (base == nullptr) {
    TK_TRY(cudaMallocAsync((void**)&base, need, st));
    owned = true;
  } else if (o->workspace_bytes < need) {
    return TK_EWORKSPACE;
  }
  unsigned char* b0 = (unsigned char*)(((uintptr_t)base + 255) & ~(uintptr_t)255);
  HosvdWs wm[TK_MAX_D];
  const size_t main = carve(p, b0, wm);
  Arena a;
  a.base = b0 + al(main);
  unsigned char* qk0 = (unsigned char*)a.take(h.qk);
  void* bx = a.take(h.bx);
  double* b64[2] = {(double*)a.take(h.b64), (double*)a.take(h.b64)};
  unsigned char* v0 = (unsigned char*)a.take(h.v);
  void* small = a.take(h.small);
  double* sig = (double*)a.take(h.sig);
  const HosvdWs& w = wm[0];
  std::vector<double*> qk(p.d), vk(p.d);
  {
    size_t oq = 0, ov = 0;
    for (int k = 0; k < p.d; ++k) {
      qk[k] = (double*)(qk0 + oq);
      vk[k] = (double*)(v0 + ov);
      oq += al((size_t)p.n[k] * p.l[k] * sizeof(double));
      ov += al((size_t)p.l[k] * h.r[k] * sizeof(double));
    }
  }
  auto run = [&]() -> tk_status {
    TK_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    TK_TRY(cudaMemsetAsync(w.ahist, 0, sizeof(double) * TK_MAX_D * TK_MAX_Q, st));
    TK_TRY(cudaMemsetAsync(w.shist, 0, sizeof(double) * TK_MAX_D * TK_MAX_Q, st));
    TK_TRY(cudaMemsetAsync(w.sig, 0, sizeof(double) * TK_MAX_D * TK_MAX_L, st));
    // range finder: Q_k with l_k columns; B <- B x_k Q_k^T (ST case: on the
    // shrinking tensor; T-HOSVD case: every Q_k from A, then the chain)
    const void* X = A->data;
    std::vector<int64_t> cur = p.n;
    int pp = 0;
    for (int k = 0; k < p.d; ++k) {
      const int lk = p.l[k];
      int64_t ka = 0, kb = 1;
      const View v = p.st ? step_view(p, cur, k, &ka, &kb) : view_of(p.n, k);
      const tk_status e = factor_mode(p, k, p.st ? X : A->data, p.xt, v, ka, kb, o->seed,
                                      o->tag, w, st);
      if (e != TK_OK) return e;
      if (p.xt != X_F64) TK_TRY(polish(w.Q, v.n, lk, w.small, w.status, st));
      TK_TRY(launch_copy_matrix(w.Q, v.n, qk[k], v.n, v.n, lk, X_F64, st));
      if (p.st) {
        void* out = (k == p.d - 1) ? bx : w.g[pp];
        TK_TRY(ttm(p.xt, X, v, qk[k], lk, out, st, p.rot ? 1 : 0, w.part));
        X = out;
        pp ^= 1;
        cur[k] = lk;
      }
    }
    if (!p.st) {
      for (int k = 0; k < p.d; ++k) {
        const View v = view_of(cur, k);
        void* out = (k == p.d - 1) ? bx : w.g[k & 1];
        TK_TRY(ttm(p.xt, X, v, qk[k], p.l[k], out, st, 0, w.part));
        X = out;
        cur[k] = p.l[k];
      }
    }
    // deterministic ST-HOSVD (Algorithm 1) of B, held in FP64: V_k = leading
    // eigenvectors of B_(k) B_(k)^T (FP64 sums), B <- B x_k V_k^T; then
    // U_k = Q_k V_k
    const int64_t cnt = prod(cur);
    if (p.xt == X_F64)
      TK_TRY(cudaMemcpyAsync(b64[0], bx, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                             st));
    else
      TK_TRY(launch_to_f64_from_f32((const float*)bx, cnt, b64[0], st));
    int cb = 0;
    for (int k = 0; k < p.d; ++k) {
      const int lk = p.l[k];
      const View v = view_of(cur, k);
      {
        ProfScope ps(TK_K_SMALL_SVD, (double)v.P * v.n * v.S * 8.0,
                     2.0 * v.P * v.n * v.S * v.n, st);
        TK_TRY(launch_gram_unfold(b64[cb], v, w.Y, st));
        TK_TRY(launch_small_svd(p.xt == X_F64, h.sm[k], w.Y, lk, w.Q, sig, small,
                                (int)TK_SHIFT_NONE, false, w.alpha, nullptr, nullptr, w.status,
                                st));
      }
      if (p.xt != X_F64) TK_TRY(polish(w.Q, lk, h.r[k], small, w.status, st));
      TK_TRY(launch_copy_matrix(w.Q, lk, vk[k], lk, lk, h.r[k], X_F64, st));
      TK_TRY(ttm(X_F64, b64[cb], v, vk[k], h.r[k], b64[cb ^ 1], st));
      cb ^= 1;
      cur[k] = h.r[k];
    }
    TK_TRY(launch_copy_matrix(b64[cb], prod(cur), core, prod(cur), prod(cur), 1, p.xt, st));
    for (int k = 0; k < p.d; ++k)
      TK_TRY(launch_qv(qk[k], p.n[k], p.l[k], vk[k], h.r[k], U[k], p.xt, st));
    if (stats) {
      std::vector<double> ah(TK_MAX_D * TK_MAX_Q), sh(TK_MAX_D * TK_MAX_Q), sg(TK_MAX_D * TK_MAX_L);
      int status = 0;
      TK_TRY(cudaMemcpyAsync(ah.data(), w.ahist, ah.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(sh.data(), w.shist, sh.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(sg.data(), w.sig, sg.size() * 8, cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
      TK_TRY(cudaStreamSynchronize(st));
      std::memset(stats, 0, sizeof(*stats));
      stats->d = p.d;
      stats->q = p.q;
      for (int k = 0; k < p.d; ++k) {
        stats->l[k] = p.l[k];
        stats->order[k] = k;
        for (int t = 0; t < TK_MAX_Q; ++t) {
          stats->alpha[k][t] = ah[k * TK_MAX_Q + t];
          stats->sigma_l[k][t] = sh[k * TK_MAX_Q + t];
        }
        for (int i = 0; i < TK_MAX_L; ++i) stats->sigma[k][i] = sg[k * TK_MAX_L + i];
      }
      if (status != 0) return (tk_status)status;
    }
    return TK_OK;
  };
  tk_status rs = run();
  if (owned) {
    cudaError_t e = cudaFreeAsync(base, st);
    if (rs == TK_OK && e != cudaSuccess) rs = from_cuda(e);
  }
  return rs;
}

}  // namespace tk

using namespace tk;

extern "C" {

size_t tucker_holistic_workspace_size(const tk_tensor* A, const int* r, const tk_opts* o,
                                      int st) {
  HolisticPlan h;
  if (holistic_plan(A, r, o, st != 0, h) != TK_OK) return 0;
  return holistic_bytes(h);
}

tk_status tucker_holistic(const tk_tensor* A, const int* r, const tk_opts* o, int st, void* core,
                          void* const* U, tk_stats* stats, void* stream) {
  return run_holistic(A, r, o, core, U, stats, (cudaStream_t)stream, st != 0);
}

const char* tucker_status_string(tk_status s) {
  switch (s) {
    case TK_OK: return "TK_OK";
    case TK_EINVAL: return "TK_EINVAL: invalid argument";
    case TK_ENOMEM: return "TK_ENOMEM: device allocation failed";
    case TK_ECUDA: return "TK_ECUDA: CUDA runtime error";
    case TK_EBREAKDOWN: return "TK_EBREAKDOWN: non-finite value on the device";
    case TK_ETIMEOUT: return "TK_ETIMEOUT: bounded device wait ran out";
    case TK_ENOTIMPL: return "TK_ENOTIMPL: outside the built kernels' limits";
    case TK_EWORKSPACE: return "TK_EWORKSPACE: workspace too small";
  }
  return "unknown tk_status";
}

size_t tucker_workspace_size(const tk_tensor* A, const int* r, const tk_opts* o, int st) {
  HosvdPlan p;
  if (make_plan(A, r, o, st != 0, p) != TK_OK) return 0;
  return carve(p, nullptr, nullptr);
}

tk_status tucker_debug_omega(int k, int64_t row0, int64_t rows, int l, uint64_t seed,
                             uint32_t tag, float* out, void* stream) {
  if (k < 0 || k > 255 || row0 < 0 || rows < 0 || l < 0 || tag >= (1u << 24)) return TK_EINVAL;
  if (rows > 0 && l > 0 && out == nullptr) return TK_EINVAL;
  TK_TRY(launch_omega(k, row0, rows, l, seed, tag, out, (cudaStream_t)stream));
  return TK_OK;
}

tk_status tucker_debug_omega_matrix(tk_omega kind, int d, const int64_t* n, int k, int l,
                                    uint64_t seed, uint32_t tag, float* out, void* stream) {
  if (kind < TK_OMEGA_GAUSS || kind > TK_OMEGA_KR_UNIFORM || d < 1 || d > TK_MAX_D || !n ||
      k < 0 || k >= d || l < 1 || l > TK_MAX_L || tag >= (1u << 24) || !out)
    return TK_EINVAL;
  for (int m = 0; m < d; ++m)
    if (n[m] < 1) return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t kb = omega_scratch(kind, n, d, k, l);
  float* kr = nullptr;
  if (kb) TK_TRY(cudaMallocAsync((void**)&kr, kb, st));
  cudaError_t e = launch_omega_fill(kind, n, d, k, l, seed, tag, 0, 1, kr, out, false, 0, st);
  cudaError_t e2 = kr ? cudaFreeAsync(kr, st) : cudaSuccess;
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(e2);
}

tk_status tucker_sketch(const tk_tensor* A, int k, int l, uint64_t seed, uint32_t tag, double* Y,
                        void* stream) {
  if (!valid_tensor(A, true) || k < 0 || k >= A->d || l < 1 || l > TK_MAX_L || !Y ||
      tag >= (1u << 24))
    return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> dims(A->n, A->n + A->d);
  const View v = view_of(dims, k);
  const XType xt = xtype(A->dtype);
  const int splits = xb_splits(xt, v, l);
  const int lc = xb_lc(l);
  void* part = nullptr;
  TK_TRY(cudaMallocAsync(&part, (size_t)splits * v.n * lc * asize(xt), st));
  cudaError_t e = launch_xb(xt, A->data, v, nullptr, l, seed, tag, k, part, splits, st);
  if (e == cudaSuccess) e = launch_reduce(xt, part, splits, v.n, l, lc, nullptr, nullptr, Y, st);
  cudaError_t e2 = cudaFreeAsync(part, st);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(e2);
}

tk_status tucker_shifted_power(const tk_tensor* A, int k, int l, int q, tk_shift rule,
                               double* Q, double* sigma, double* alpha, void* stream) {
  if (!valid_tensor(A, true) || k < 0 || k >= A->d || l < 1 || l > TK_MAX_L || q < 0 ||
      q > TK_MAX_Q || !Q || !sigma || !alpha)
    return TK_EINVAL;
  if (rule != TK_SHIFT_PAPER && rule != TK_SHIFT_NONE) return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> dims(A->n, A->n + A->d);
  const View v = view_of(dims, k);
  if (l > v.n || l > v.cols()) return TK_EINVAL;
  const XType xt = xtype(A->dtype);
  const bool fp64 = xt == X_F64;
  const SmallPlan sp = small_plan(v.n, l, fp64);
  if (sp.Pb <= 0) return TK_ENOTIMPL;
  const int splits = xb_splits(xt, v, l);
  const int lc = xb_lc(l);
  // bfloat16 mode-major tensors take the fused tensor-core pass
  const bool tc = xt == X_BF16 && power_tc_supported(v, l, A->data);
  const int groups = tc ? power_tc_groups(v, l) : 0;
  const int lp = power_tc_lpad(v, l);
  Arena b;
  const size_t o_w = b.offset(tc ? 0 : (size_t)v.cols() * l * asize(xt));
  const bool comp_y = !tc && xtb32_ok(xt, v, A->data);
  const size_t o_part = b.offset(tc ? (size_t)groups * v.n * lp * sizeof(float)
                                    : (size_t)splits * v.n * lc * asize(xt) * (comp_y ? 2 : 1));
  const size_t o_y = b.offset((size_t)v.n * l * sizeof(double));
  // FP32 mode-major views take W = X^T Q on the tensor cores (Q split into B2)
  const bool tcw = !tc && xt == X_F32 && tc32_ok(v, l, A->data);
  const size_t o_sm = b.offset(std::max({sp.scratch_bytes, tc ? power_tc_scratch(v, l) : 0,
                                         tcw ? tc32_xtb_scratch(v) : 0}));
  const size_t o_st = b.offset(sizeof(int));
  unsigned char* base = nullptr;
  TK_TRY(cudaMallocAsync((void**)&base, b.off + 256, st));
  void* wv = base + o_w;
  void* part = base + o_part;
  void* Y = base + o_y;
  void* sm = base + o_sm;
  int* stt = (int*)(base + o_st);
  const double N = (double)v.P * (double)v.n * (double)v.S;
  auto body = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(stt, 0, sizeof(int), st);
    for (int t = 1; t <= q && e == cudaSuccess; ++t) {
      if (tc) {
        {
          ProfScope ps(TK_K_POWER_FUSED, N * 2.0, 4.0 * N * l, st);
          e = launch_power_tc(A->data, v, Q, l, sm, (float*)part, groups, stt, st);
        }
        if (e == cudaSuccess)
          e = launch_reduce(X_BF16, part, groups, v.n, l, lp, Q, alpha, (double*)Y, st);
      } else {
        {
          ProfScope ps(TK_K_POWER_W, N * xsize(xt), 2.0 * N * l, st);
          e = tcw ? launch_tc32_xtb(A->data, v, Q, 1, v.n, l, (float*)wv, 0, 0, sm, stt, st)
                  : launch_xtb(xt, A->data, v, Q, 1, v.n, l, wv, st);
        }
        void* plo = comp_y ? (unsigned char*)part + (size_t)splits * v.n * lc * asize(xt)
                           : nullptr;
        if (e == cudaSuccess) {
          ProfScope ps(TK_K_POWER_Y, N * xsize(xt), 2.0 * N * l, st);
          e = launch_xb(xt, A->data, v, wv, l, 0, 0, k, part, splits, st, 0, 1, plo);
        }
        if (e == cudaSuccess)
          e = launch_reduce(xt, part, splits, v.n, l, lc, Q, alpha, (double*)Y, st, plo);
      }
      if (e == cudaSuccess)
        e = launch_small_svd(fp64, sp, (const double*)Y, v.n, Q, sigma, sm, (int)rule, true,
                             alpha, nullptr, nullptr, stt, st);
    }
    return e;
  };
  cudaError_t e = body();
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, stt, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(base, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  if (e2 != cudaSuccess) return from_cuda(e2);
  return (tk_status)status;
}

tk_status tucker_rthosvd(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                         void* const* U, tk_stats* st, void* stream) {
  return run_hosvd(A, r, o, core, U, st, (cudaStream_t)stream, false);
}

tk_status tucker_rsthosvd(const tk_tensor* A, const int* r, const tk_opts* o, void* core,
                          void* const* U, tk_stats* st, void* stream) {
  return run_hosvd(A, r, o, core, U, st, (cudaStream_t)stream, true);
}

tk_status tucker_rsthosvd_pve(const tk_tensor* A, const int* r, const tk_opts* o, double tol,
                              void* core, void* const* U, int* q_out, tk_stats* st,
                              void* stream) {
  if (!o || !(tol >= 0.0) || o->q < 1 || o->prec != TK_PREC_PLAIN) return TK_EINVAL;
  return run_hosvd(A, r, o, core, U, st, (cudaStream_t)stream, true, tol, q_out);
}

tk_status tucker_rthosvd_pve(const tk_tensor* A, const int* r, const tk_opts* o, double tol,
                             void* core, void* const* U, int* q_out, tk_stats* st,
                             void* stream) {
  if (!o || !(tol >= 0.0) || o->q < 1 || o->prec != TK_PREC_PLAIN) return TK_EINVAL;
  return run_hosvd(A, r, o, core, U, st, (cudaStream_t)stream, false, tol, q_out);
}

tk_status tucker_error(const tk_tensor* A, const void* core, const int* r, const void* const* U,
                       double* rel_err, void* stream) {
  if (!valid_tensor(A, false) || !core || !r || !U || !rel_err) return TK_EINVAL;
  const int d = A->d;
  for (int k = 0; k < d; ++k)
    if (r[k] < 1 || r[k] > A->n[k] || !U[k]) return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const XType xt = xtype(A->dtype);
  const size_t es = xsize(xt);
  // expansion chain sizes: after step k the dims are (n_1..n_k, r_{k+1}..r_d)
  std::vector<int64_t> cur(r, r + d);
  size_t tbuf = 0;
  for (int k = 0; k < d - 1; ++k) {
    cur[k] = A->n[k];
    tbuf = std::max(tbuf, (size_t)prod(cur) * es);
  }
  std::vector<int64_t> last(r, r + d);
  for (int k = 0; k < d - 1; ++k) last[k] = A->n[k];
  const View vl = view_of(last, d - 1);
  const int blocks = xtb_error_blocks(xt, vl, (int)A->n[d - 1]);
  Arena a;
  const size_t t0 = a.offset(tbuf);
  const size_t t1 = a.offset(tbuf);
  std::vector<size_t> uoff(d);
  for (int k = 0; k < d; ++k) uoff[k] = a.offset((size_t)A->n[k] * r[k] * sizeof(double));
  const size_t ep = a.offset((size_t)blocks * 2 * sizeof(double));
  unsigned char* base = nullptr;
  TK_TRY(cudaMallocAsync((void**)&base, a.off + 256, st));
  auto body = [&]() -> cudaError_t {
    std::vector<double*> Ud(d);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < d && e == cudaSuccess; ++k) {
      Ud[k] = (double*)(base + uoff[k]);
      if (xt == X_F64)
        e = cudaMemcpyAsync(Ud[k], U[k], (size_t)A->n[k] * r[k] * 8, cudaMemcpyDeviceToDevice, st);
      else
        e = launch_to_f64_from_f32((const float*)U[k], (int64_t)A->n[k] * r[k], Ud[k], st);
    }
    const void* X = core;
    std::vector<int64_t> dims(r, r + d);
    void* tb[2] = {base + t0, base + t1};
    for (int k = 0; k < d - 1 && e == cudaSuccess; ++k) {
      const View v = view_of(dims, k);
      // B(i = core index, c = output index) = U_k(c, i)
      const double cin = (double)v.P * v.n * v.S;
      ProfScope ps(TK_K_ERROR, (cin + cin / v.n * A->n[k]) * es, 2.0 * cin / v.n * A->n[k] * v.n,
                   st);
      e = launch_xtb(xt, X, v, Ud[k], A->n[k], 1, (int)A->n[k], tb[k & 1], st, 0, nullptr,
                     xt == X_F32 ? (const float*)U[k] : nullptr, /*comp=*/true);
      X = tb[k & 1];
      dims[k] = A->n[k];
    }
    int nb = 0;
    const double Nf = (double)vl.P * (double)A->n[d - 1];
    ProfScope ps(TK_K_ERROR, Nf * es + (double)vl.P * vl.n * es, 2.0 * Nf * vl.n, st);
    if (e == cudaSuccess)
      e = launch_xtb_error(xt, X, vl, Ud[d - 1], A->n[d - 1], 1, (int)A->n[d - 1], A->data,
                           (double*)(base + ep), &nb, st,
                           xt == X_F32 ? (const float*)U[d - 1] : nullptr);
    if (e == cudaSuccess) e = launch_error_final((double*)(base + ep), nb, rel_err, st);
    return e;
  };
  cudaError_t e = body();
  cudaError_t e2 = cudaFreeAsync(base, st);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(e2);
}

tk_status tucker_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_recs) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_recs.clear();
  g_prof_on = on != 0;
  g_kernels.store(0);
  return TK_OK;
}

tk_status tucker_profile_read(tk_profile* out) {
  if (!out) return TK_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::memset(out, 0, sizeof(*out));
  tk_status st = TK_OK;
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      st = TK_ECUDA;
    if (r.kind >= 0 && r.kind < TK_K_KINDS) {
      out->launches[r.kind] += 1;
      out->ms[r.kind] += ms;
      out->bytes[r.kind] += r.bytes;
      out->flops[r.kind] += r.flops;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_recs.clear();
  out->kernels = g_kernels.exchange(0);
  return st;
}

tk_status tucker_to_bf16(const float* x, int64_t count, uint16_t* out, void* stream) {
  if (count < 0 || (count > 0 && (!x || !out))) return TK_EINVAL;
  TK_TRY(launch_to_bf16(x, count, out, (cudaStream_t)stream));
  return TK_OK;
}

}  // extern "C"
