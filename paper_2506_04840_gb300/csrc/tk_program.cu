// Compiles one problem of Algorithm 3 into phases of work-list jobs and
// merges any problems' phases into batched launches (tk_program.h).
#include <algorithm>
#include <cstring>

#include "tk_program.h"

namespace tk {

namespace {

template <typename J>
Op make_op(int pos, int prof, int kind, XType xt, int tile, int flag, size_t smem,
           uint32_t blocks, double bytes, double flops, const J& job) {
  static_assert(sizeof(J) <= kJobBytes, "job struct too large");
  Op o;
  std::memset(&o, 0, sizeof(o));
  o.pos = pos;
  o.prof = prof;
  o.key.kind = kind;
  o.key.xt = (int)xt;
  o.key.tile = tile;
  o.key.flag = flag;
  o.key.smem = smem;
  o.blocks = blocks;
  o.bytes = bytes;
  o.flops = flops;
  std::memcpy(o.job, &job, sizeof(J));
  return o;
}

size_t job_size(int kind) {
  switch (kind) {
    case BK_XB: return sizeof(XbJob);
    case BK_REDUCE: return sizeof(ReduceJob);
    case BK_SVD: return sizeof(SvdJob);
    case BK_XTB: return sizeof(XtbJob);
    case BK_GRAM: return sizeof(GramJob);
    case BK_POLISH: return sizeof(PolishJob);
    case BK_COPY: return sizeof(CopyJob);
    case BK_XTB32: return sizeof(Xtb32Job);
    case BK_XTB32RED: return sizeof(Xtb32RedJob);
    case BK_ERR32: return sizeof(Err32Job);
    case BK_XB32: return sizeof(Xb32Job);
    case BK_TC32SPLIT: return sizeof(Tc32SplitJob);
    case BK_TC32XTB: return sizeof(Tc32XtbJob);
    case BK_TC32SKETCH: return sizeof(Tc32SketchJob);
    case BK_TSQR_LEAF:
    case BK_TSQR_ROOT:
    case BK_TSQR_LEAFQ:
    case BK_TSQR_SIGN: return sizeof(TsqrJob);
    default: return sizeof(ErrFinalJob);
  }
}

uint32_t cdiv(int64_t a, int64_t b) { return (uint32_t)((a + b - 1) / b); }

// out = X x_k B^T (EPI 0) as the single-problem launch_xtb runs it (with the
// same scratch): the FP32 mode-major kernel where it applies (+ the sum of its
// row splits at position pos + 1), else the generic one.
// The FP32 kernel reads B in FP32: B32 (same strides) when given, else B is
// first rounded into the scratch (at position pos - 1; scratch required).
void xtb_ops(Phase& ph, int pos, int prof, XType xt, const void* X, View v, const double* B,
             int64_t b_ri, int64_t b_cm, int m, void* out, double bytes, double flops,
             int tout = 0, void* scratch = nullptr, const float* B32 = nullptr,
             bool comp = false) {
  if (xtb32_ok(xt, v, X)) {
    const Xtb32Shape sh = xtb32_shape(v, m, scratch != nullptr);
    void* part = sh.ks > 1 ? scratch : nullptr;
    if (B32 == nullptr) {
      // B is a column-major n x m FP64 factor here (b_ri = 1, b_cm = n)
      float* b32 = (float*)((unsigned char*)scratch + xtb32_b32_offset(v, m));
      CopyJob cj{B, b32, b_cm, v.n, v.n, m};
      ph.push_back(make_op(pos - 1, TK_K_CONVERT, BK_COPY, X_F32, 0, 0, 0, cdiv(v.n * m, 256),
                           (double)v.n * m * 12.0, 0.0, cj));
      B32 = b32;
      b_ri = 1;
      b_cm = v.n;
    }
    Xtb32Job j{X, v.n, v.cols(), B32, b_ri, b_cm, out, part, sh.kps, m, sh.gx, sh.gy, tout};
    ph.push_back(make_op(pos, prof, BK_XTB32, xt, sh.wc, (sh.wj << 1) | (comp ? 1 : 0), 0,
                         (uint32_t)sh.gx * sh.gy * sh.ks, bytes, flops, j));
    if (part) {
      Xtb32RedJob rj{part, out, v.cols(), m, sh.ks, tout};
      ph.push_back(make_op(pos + 1, prof, BK_XTB32RED, xt, 0, 0, 0, cdiv(v.cols() * m, 256),
                           0.0, 0.0, rj));
    }
    return;
  }
  const int mt = xtb_tile(m);
  const int gx = (int)cdiv(v.cols(), 128);
  XtbJob j{X, v.P, v.n, v.S, B, b_ri, b_cm, out, nullptr, nullptr, m, gx};
  ph.push_back(make_op(pos, prof, BK_XTB, xt, mt, 0, 0, (uint32_t)gx * cdiv(m, mt), bytes, flops,
                       j));
}

// partials of Y = X_(k) B (B = W, or Omega_k when W == NULL) as launch_xb runs them.
Op xb_op(int pos, int prof, XType xt, const void* X, View v, const void* W, int l,
         uint64_t seed, uint32_t tag, int mode, void* part, int splits, double bytes,
         double flops, int64_t ka = 0, int64_t kb = 1, void* part_lo = nullptr) {
  if (xtb32_ok(xt, v, X)) {
    const Xb32Shape sh = xb32_shape(v, l, splits);
    if (ka <= 0) {
      ka = v.cols();
      kb = 1;
    }
    void* plo = W != nullptr ? part_lo : nullptr;
    Xb32Job j{X, v.n, v.cols(), W, sh.cps, ka, kb, part, plo, seed, tag, l, sh.lc, mode,
              sh.gx, sh.gy};
    return make_op(pos, prof, BK_XB32, xt, sh.wc,
                   (W == nullptr ? 1 : 0) | (sh.wi << 1) | (plo != nullptr ? 16 : 0), 0,
                   (uint32_t)sh.gx * sh.gy * sh.splits, bytes, flops, j);
  }
  const int lc = xb_lc(l);
  const int gx = xb_grid_x(v, l);
  const int64_t cps = xb_cols_per_split(xt, v, splits);
  XbJob j{X, v.P, v.n, v.S, W, cps, part, seed, tag, l, mode, gx};
  return make_op(pos, prof, BK_XB, xt, lc, W == nullptr ? 1 : 0, 0, (uint32_t)gx * splits, bytes,
                 flops, j);
}

// [Q, Sigma] = svd(Y) (+ shift update) as launch_small_svd runs it, at
// positions pos.. of the phase: one CTA (one op), or the TSQR chain (four ops
// at pos .. pos + 3 on the svd scratch).
void svd_ops(Phase& ph, int pos, const SmallPlan& pl, XType xt, const double* Y, int64_t n,
             double* Q, double* sigma, void* scratch, int rule, bool update_shift,
             bool basis_only, double* alpha, double* ahist, double* shist, int* status) {
  const bool fp64 = xt == X_F64;
  const int l = pl.l;
  const double nl = (double)n * l;
  const double flops = 4.0 * nl * l + 2.0 * (double)l * l * l;
  if (pl.Pb == 1) {
    SvdJob sv{Y, Q, sigma, alpha, ahist, shist, status, (int)n, l, rule,
              update_shift ? 1 : 0, basis_only ? 1 : 0};
    ph.push_back(make_op(pos, TK_K_SMALL_SVD, BK_SVD, xt, svd_threads(n, l, fp64),
                         svd_variant(n, l, fp64), svd_smem(n, l, fp64), 1, 2.0 * nl * 8.0,
                         flops, sv));
    return;
  }
  TsqrJob tj;
  TsqrStage stg[4];
  const int flag = tsqr_job(pl, fp64, Y, n, Q, sigma, scratch, rule, update_shift, basis_only,
                            alpha, ahist, shist, status, &tj, stg);
  for (int i = 0; i < 4; ++i)
    ph.push_back(make_op(pos + i, TK_K_SMALL_SVD, stg[i].kind, xt, 0, flag, stg[i].smem,
                         stg[i].blocks, i == 0 ? 2.0 * nl * 8.0 : 0.0, i == 0 ? flops : 0.0,
                         tj));
}

// Extra per-problem buffers beyond the single-call workspace.
struct Extras {
  size_t state, qd[TK_MAX_D], tb[2], ep;
  int eblocks;
};

size_t layout(const tk_item& it, const HosvdPlan& p, Extras* ex) {
  Arena a;
  const size_t hos = carve(p, nullptr, nullptr);
  a.offset(hos);
  ex->state = a.offset(sizeof(ItemState));
  ex->eblocks = 0;
  ex->tb[0] = ex->tb[1] = ex->ep = 0;
  for (int k = 0; k < TK_MAX_D; ++k) ex->qd[k] = 0;
  if (it.rel_err) {
    const int d = p.d;
    const size_t es = xsize(p.xt);
    for (int k = 0; k < d; ++k) ex->qd[k] = a.offset((size_t)p.n[k] * p.r[k] * sizeof(double));
    std::vector<int64_t> cur(p.r.begin(), p.r.end());
    size_t tbuf = 0;
    for (int k = 0; k < d - 1; ++k) {
      cur[k] = p.n[k];
      tbuf = std::max(tbuf, (size_t)prod(cur) * es);
    }
    ex->tb[0] = a.offset(tbuf);
    ex->tb[1] = a.offset(tbuf);
    std::vector<int64_t> last(p.r.begin(), p.r.end());
    for (int k = 0; k < d - 1; ++k) last[k] = p.n[k];
    ex->eblocks = xtb_error_blocks(p.xt, view_of(last, d - 1), (int)p.n[d - 1]);
    ex->ep = a.offset((size_t)ex->eblocks * 2 * sizeof(double));
  }
  return al(a.off);
}

}  // namespace

tk_status problem_plan(const tk_item& it, tk_shift rule, Problem* pr) {
  if (it.A.dtype != TK_F32 && it.A.dtype != TK_F64) return TK_EINVAL;
  if (!it.core) return TK_EINVAL;
  for (int k = 0; k < it.A.d && k < TK_MAX_D; ++k)
    if (!it.U[k]) return TK_EINVAL;
  tk_opts o;
  std::memset(&o, 0, sizeof(o));
  o.q = it.q;
  for (int k = 0; k < TK_MAX_D; ++k) o.s[k] = it.s[k];
  o.seed = it.seed;
  o.tag = it.tag;
  o.shift = rule;
  o.prec = TK_PREC_PLAIN;
  if (it.order != 0 && it.order != TK_ORDER_DESCENDING) return TK_EINVAL;
  o.order[0] = it.order == TK_ORDER_DESCENDING ? TK_ORDER_DESCENDING : -1;
  tk_status s = make_plan(&it.A, it.r, &o, true, pr->p);
  if (s != TK_OK) return s;
  Extras ex;
  pr->ws_bytes = layout(it, pr->p, &ex);
  return TK_OK;
}

tk_status problem_build(const tk_item& it, unsigned char* base, Problem* pr) {
  const HosvdPlan& p = pr->p;
  Extras ex;
  layout(it, p, &ex);
  carve(p, base, &pr->w);
  HosvdWs& w = pr->w;
  ItemState* stt = (ItemState*)(base + ex.state);
  pr->state = stt;
  w.status = &stt->status;
  const XType xt = p.xt;
  const bool fp64 = xt == X_F64;
  const size_t es = xsize(xt);
  const int d = p.d;
  double* qd[TK_MAX_D] = {nullptr};
  if (it.rel_err)
    for (int k = 0; k < d; ++k) qd[k] = (double*)(base + ex.qd[k]);
  std::vector<Phase>& prog = pr->prog;
  prog.clear();
  pr->slot.clear();
  const int per_step = TK_MAX_Q + 2;

  const void* X = it.A.data;
  std::vector<int64_t> cur = p.n;
  int pp = 0;
  for (int step = 0; step < d; ++step) {
    const int k = p.order[step];
    int64_t ka, kb;
    const View v = step_view(p, cur, k, &ka, &kb);
    const int l = p.l[k];
    const int lc = xb_lc(l);
    const int splits = xb_splits(xt, v, l);
    const double N = (double)v.P * (double)v.n * (double)v.S;
    const double nl = (double)v.n * l;
    const double red_bytes = (double)splits * v.n * lc * asize(xt) + nl * 8.0;
    const XType acc = fp64 ? X_F64 : X_F32;
    double* sig = stt->sig + (size_t)k * TK_MAX_L;
    double* alpha = stt->alpha + k;

    // ---- sketch phase
    {
      Phase ph;
      Tc32SketchJob skj;
      int sp = splits, slc = lc;
      if (xt == X_F32 && tc32_sketch_job(X, v, l, it.seed, it.tag, k, ka, kb, (float*)w.part,
                                         w.status, nullptr, &skj)) {
        // the sketch on the tensor cores, as the single call runs it
        ph.push_back(make_op(0, TK_K_SKETCH, BK_TC32SKETCH, xt, 0, 0, tc32_sketch_smem(),
                             (uint32_t)skj.units, N * es, 2.0 * N * l, skj));
        sp = skj.groups;
        slc = 64;
      } else {
        ph.push_back(xb_op(0, TK_K_SKETCH, xt, X, v, nullptr, l, it.seed, it.tag, k, w.part,
                           splits, N * es, 2.0 * N * l, ka, kb));
      }
      ReduceJob rd{w.part, v.n, nullptr, nullptr, w.Y, sp, l, slc, nullptr};
      ph.push_back(make_op(1, TK_K_CONVERT, BK_REDUCE, acc, 0, 0, 0, cdiv(v.n * l, 32),
                           red_bytes, (double)splits * nl, rd));
      svd_ops(ph, 2, p.sp[k], acc, w.Y, v.n, w.Q, sig, w.small, (int)p.rule, false, p.q >= 1,
              alpha, nullptr, nullptr, w.status);
      prog.push_back(ph);
      pr->slot.push_back(step * per_step);
    }
    // ---- power phases
    for (int t = 1; t <= p.q; ++t) {
      Phase ph;
      Tc32SplitJob sj;
      Tc32XtbJob xj;
      if (xt == X_F32 &&
          tc32_xtb_jobs(X, v, w.Q, 1, v.n, l, (float*)w.w, 0, 0, w.small, w.status, &sj, &xj)) {
        // W = X^T Q in 3xTF32 on the tensor cores, as the single call runs it
        ph.push_back(make_op(0, TK_K_CONVERT, BK_TC32SPLIT, xt, 0, 0, 0, tc32_split_blocks(sj),
                             (double)v.n * l * 16.0, 0.0, sj));
        ph.push_back(make_op(1, TK_K_POWER_W, BK_TC32XTB, xt, 0, 0, tc32_xtb_smem(),
                             (uint32_t)xj.units, N * es, 2.0 * N * l, xj));
      } else {
        xtb_ops(ph, 1, TK_K_POWER_W, xt, X, v, w.Q, 1, v.n, l, w.w, N * es, 2.0 * N * l, 0,
                w.part);
      }
      // compensated Y = X W on FP32 mode-major views, as the single call runs it
      void* plo = xtb32_ok(xt, v, X)
                      ? (unsigned char*)w.part + (size_t)splits * v.n * lc * asize(xt) : nullptr;
      ph.push_back(xb_op(3, TK_K_POWER_Y, xt, X, v, w.w, l, it.seed, it.tag, k, w.part, splits,
                         N * es, 2.0 * N * l, 0, 1, plo));
      ReduceJob rd{w.part, v.n, w.Q, alpha, w.Y, splits, l, lc, plo};
      ph.push_back(make_op(4, TK_K_CONVERT, BK_REDUCE, acc, 0, 0, 0, cdiv(v.n * l, 32),
                           red_bytes, (double)splits * nl, rd));
      svd_ops(ph, 5, p.sp[k], acc, w.Y, v.n, w.Q, sig, w.small, (int)p.rule, true, false,
              alpha, stt->ahist + (size_t)k * TK_MAX_Q + (t - 1),
              stt->shist + (size_t)k * TK_MAX_Q + (t - 1), w.status);
      prog.push_back(ph);
      pr->slot.push_back(step * per_step + t);
    }
    // ---- finish phase: U_k, TTM shrink
    {
      Phase ph;
      const int r = p.r[k];
      if (!fp64) {
        const int nblk = polish_blocks(v.n);
        GramJob gj{w.Q, (double*)w.small, v.n, r};
        ph.push_back(make_op(0, TK_K_CONVERT, BK_GRAM, X_F64, 0, 0, gram_smem(r),
                             (uint32_t)nblk, 2.0 * v.n * r * 8.0, 2.0 * v.n * r * r, gj));
        PolishJob pj{w.Q, (const double*)w.small, w.status, v.n, r, nblk};
        ph.push_back(make_op(1, TK_K_CONVERT, BK_POLISH, X_F64, 0, 0, polish_smem(r),
                             (uint32_t)nblk, 0.0, 0.0, pj));
      }
      CopyJob cu{w.Q, it.U[k], v.n, v.n, v.n, r};
      ph.push_back(make_op(2, TK_K_CONVERT, BK_COPY, xt, 0, 0, 0, cdiv(v.n * r, 256),
                           (double)v.n * r * (8.0 + es), 0.0, cu));
      if (qd[k]) {
        // the error pass reads the returned factor (rounded to A's dtype)
        CopyJob cq{w.Q, qd[k], v.n, v.n, v.n, r};
        ph.push_back(make_op(2, TK_K_CONVERT, BK_COPY, X_F64, 0, fp64 ? 0 : 1, 0,
                             cdiv(v.n * r, 256), (double)v.n * r * 16.0, 0.0, cq));
      }
      void* out = (step == d - 1) ? it.core : w.g[pp];
      // the TTM reads the returned factor (FP32 for an FP32 tensor)
      xtb_ops(ph, 3, TK_K_TTM, xt, X, v, w.Q, 1, v.n, r, out, (N + N / v.n * r) * es,
              2.0 * N * r, p.rot ? 1 : 0, w.part, fp64 ? nullptr : (const float*)it.U[k],
              /*comp=*/true);
      prog.push_back(ph);
      pr->slot.push_back(step * per_step + TK_MAX_Q + 1);
      X = out;
      pp ^= 1;
      cur[k] = r;
    }
  }
  // ---- error phase (tucker_error on the returned core and factors)
  if (it.rel_err) {
    Phase ph;
    std::vector<int64_t> dims(p.r.begin(), p.r.end());
    const void* Xe = it.core;
    void* tb[2] = {base + ex.tb[0], base + ex.tb[1]};
    for (int k = 0; k < d - 1; ++k) {
      const View v = view_of(dims, k);
      const int m = (int)p.n[k];
      const double cin = (double)v.P * v.n * v.S;
      xtb_ops(ph, k, TK_K_ERROR, xt, Xe, v, qd[k], p.n[k], 1, m, tb[k & 1],
              (cin + cin / v.n * m) * es, 2.0 * cin / v.n * m * v.n, 0, nullptr,
              fp64 ? nullptr : (const float*)it.U[k], /*comp=*/true);
      Xe = tb[k & 1];
      dims[k] = p.n[k];
    }
    const View vl = view_of(dims, d - 1);
    const int m = (int)p.n[d - 1];
    const int mt = xtb_tile(m);
    const int egx = (int)cdiv(vl.cols(), 128);
    const double Nf = (double)vl.P * (double)m;
    double* ep = (double*)(base + ex.ep);
    if (err32_ok(xt, vl)) {
      const int gx = (int)cdiv(vl.P, 128);
      Err32Job ej{Xe, vl.P, (const float*)it.U[d - 1], p.n[d - 1], 1, it.A.data, ep, (int)vl.n,
                  m, gx};
      // the same kernel body and blocks as the single call (err32_blocks)
      const bool rowtile = err32c_ok(vl);
      ph.push_back(make_op(d - 1, TK_K_ERROR, BK_ERR32, xt, 0, rowtile ? 1 : 0,
                           rowtile ? err32c_smem((int)vl.n) : 0,
                           (uint32_t)err32_blocks(vl, m), Nf * es + (double)vl.P * vl.n * es,
                           2.0 * Nf * vl.n, ej));
    } else {
      XtbJob ej{Xe, vl.P, vl.n, vl.S, qd[d - 1], p.n[d - 1], 1, nullptr, it.A.data, ep, m, egx};
      ph.push_back(make_op(d - 1, TK_K_ERROR, BK_XTB, xt, mt, 1, 0, (uint32_t)egx * cdiv(m, mt),
                           Nf * es + (double)vl.P * vl.n * es, 2.0 * Nf * vl.n, ej));
    }
    ErrFinalJob fj{ep, it.rel_err, ex.eblocks};
    ph.push_back(make_op(d, TK_K_ERROR, BK_ERRFIN, X_F64, 0, 0, 0, 1, 0.0, 0.0, fj));
    prog.push_back(ph);
    pr->slot.push_back(TK_MAX_D * per_step);
  }
  return TK_OK;
}

// ---------------------------------------------------------------------------
// Merging.
// ---------------------------------------------------------------------------
static bool key_less(const Op* a, const Op* b) {
  if (a->pos != b->pos) return a->pos < b->pos;
  if (a->prof != b->prof) return a->prof < b->prof;
  if (a->key.kind != b->key.kind) return a->key.kind < b->key.kind;
  if (a->key.xt != b->key.xt) return a->key.xt < b->key.xt;
  if (a->key.tile != b->key.tile) return a->key.tile < b->key.tile;
  return a->key.flag < b->key.flag;
}

static bool key_eq(const Op* a, const Op* b) { return !key_less(a, b) && !key_less(b, a); }

static size_t blob_take(std::vector<unsigned char>& blob, size_t bytes) {
  // 64-byte aligned: job structs may hold TMA tensor maps
  const size_t off = (blob.size() + 63) & ~(size_t)63;
  blob.resize(off + bytes);
  return off;
}

void merge_ops(const std::vector<const Op*>& ops_in, std::vector<unsigned char>& blob,
               std::vector<LaunchRec>& out) {
  std::vector<const Op*> ops(ops_in);
  std::stable_sort(ops.begin(), ops.end(), key_less);
  size_t i = 0;
  while (i < ops.size()) {
    size_t j = i + 1;
    while (j < ops.size() && key_eq(ops[i], ops[j])) ++j;
    LaunchRec r;
    std::memset(&r, 0, sizeof(r));
    r.b = ops[i]->key;
    r.prof = ops[i]->prof;
    const size_t js = job_size(r.b.kind);
    const int nj = (int)(j - i);
    r.jobs_off = blob_take(blob, js * nj);
    r.start_off = blob_take(blob, sizeof(uint32_t) * nj);
    uint32_t total = 0;
    size_t smem = 0;
    for (int t = 0; t < nj; ++t) {
      const Op* o = ops[i + t];
      std::memcpy(blob.data() + r.jobs_off + js * t, o->job, js);
      std::memcpy(blob.data() + r.start_off + sizeof(uint32_t) * t, &total, sizeof(uint32_t));
      total += o->blocks;
      smem = std::max(smem, o->key.smem);
      r.bytes += o->bytes;
      r.flops += o->flops;
    }
    r.b.njobs = nj;
    r.b.total = total;
    r.b.smem = smem;
    out.push_back(r);
    i = j;
  }
}

void resolve(std::vector<LaunchRec>& recs, const unsigned char* dev_blob) {
  for (auto& r : recs) {
    r.b.jobs = dev_blob + r.jobs_off;
    r.b.start = (const uint32_t*)(dev_blob + r.start_off);
  }
}

cudaError_t issue(const LaunchRec& r, cudaStream_t st, bool profile) {
  if (profile) {
    ProfScope ps(r.prof, r.bytes, r.flops, st);
    return launch_batch(r.b, st);
  }
  return launch_batch(r.b, st);
}

}  // namespace tk
