// FP32 mode-major contractions on CUDA cores (FFMA), register-tiled.
//
// For a mode-major view (P == 1: X_(k) is n x cols, column j contiguous) and
// FP32 data, the two products of the power step, the sketch and the TTM run
// here instead of the generic strided kernels of k_contract.cu:
//   k_xtb32  out[j, c] = sum_i X[i, j] B[i, c]       (W = X^T Q; TTM)
//   k_xb32   part[s][i][c] = sum_{j in split s} X[i, j] B[j, c]
//            (Y = X W, or Y = X Omega_k with Omega generated in registers)
// Each thread accumulates an 8 x 4 tile; a warp is laid out 8 (rows) x 4
// (outputs) so that every shared-memory read is a 16-byte vector hitting at
// most 128 distinct bytes (one wavefront); tiles of X are staged through
// registers into a double-buffered shared-memory slab, so global loads of
// the next slab overlap the FMAs of the current one.  Summation order per
// output is fixed (i or j ascending within a block), so results are
// deterministic and independent of what else runs.
#include <algorithm>

#include "tk_batch.h"
#include "tk_common.cuh"
#include "tk_internal.h"

namespace tk {

namespace c32 {

constexpr int KS = 16;   // contraction rows staged per slab

// ---------------------------------------------------------------------------
// out[j, c] = sum_i X[i + n j] B[i*b_ri + c*b_cm],  block (bx, by):
// columns j0 = bx*MJ.., outputs c0 = by*MC..  (MJ = 64 WJ, MC = 16 WC).
// out is written in the (1, m, cols) layout out[c + m j], or with tout in
// the (cols, m) layout out[j + cols c] (the mode just contracted moves last).
// ---------------------------------------------------------------------------
// COMP: slab-compensated accumulation over the rows, as in xb32_body below:
// each slab of KS rows is summed from zero and folded into a (hi, lo) pair by
// TwoSum, and the output is hi + lo rounded once.  Used for the TTM, whose
// output is the next mode's tensor and (after the last mode) the core: an
// uncompensated FP32 sum over n_k rows of a positive, smooth tensor carries
// errors of several units of roundoff of its large entries, which in the
// later modes reach the size of the weak directions the factors must keep.
template <int WJ, int WC, typename BT, bool COMP = false>
__device__ __forceinline__ void xtb32_body(const float* __restrict__ X, int64_t n, int64_t cols,
                                           const BT* __restrict__ B, int64_t b_ri,
                                           int64_t b_cm, int m, float* __restrict__ out,
                                           int tout, int64_t ib, int64_t ie, unsigned bx,
                                           unsigned by) {
  constexpr int MJ = 64 * WJ, MC = 16 * WC, T = 32 * WJ * WC;
  constexpr int XPT = KS * MJ / T;          // X elements each thread stages per slab
  constexpr int BPT = (KS * MC + T - 1) / T;
  // slabs in flight in registers: two where the staging registers allow;
  // one with the compensated sums, which then fit two CTAs per SM (<= 128
  // registers: 16 warps per SM instead of 8 to hide the FMA chains' latency)
  constexpr int PF = XPT <= 8 && !COMP ? 2 : 1;
  __shared__ __align__(16) float Xs[2][KS][MJ + 4];
  __shared__ __align__(16) float Bs[2][KS][MC];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wj = w % WJ, wc = w / WJ;
  const int lj = lane >> 2, lc = lane & 3;
  const int64_t j0 = (int64_t)bx * MJ;
  const int c0 = (int)by * MC;
  const int ja = wj * 64 + lj * 4;          // thread's columns: ja..ja+3, ja+32..ja+35
  const int cb = wc * 16 + lc * 4;          // thread's outputs: cb..cb+3

  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
  float cmp[COMP ? 8 : 1][4];
#pragma unroll
  for (int a = 0; a < (COMP ? 8 : 1); ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) cmp[a][q] = 0.f;

  // slab t (rows ib + t KS ..) travels in register set t % PF, then shared
  // buffer t & 1
  float xr[PF][XPT], br[PF][BPT];
  auto load = [&](int p, int64_t i0) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      const int ii = e % KS, jj = e / KS;
      const int64_t i = i0 + ii, j = j0 + jj;
      xr[p][r] = (i < ie && j < cols) ? __ldg(X + j * n + i) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < BPT; ++r) {
      const int e = tid + r * T;
      float v = 0.f;
      if (e < KS * MC) {
        const int c = e % MC, ii = e / MC;
        const int64_t i = i0 + ii;
        if (i < ie && c0 + c < m) v = (float)B[i * b_ri + (int64_t)(c0 + c) * b_cm];
      }
      br[p][r] = v;
    }
  };
  auto store = [&](int p, int buf) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      Xs[buf][e % KS][e / KS] = xr[p][r];
    }
#pragma unroll
    for (int r = 0; r < BPT; ++r) {
      const int e = tid + r * T;
      if (e < KS * MC) Bs[buf][e / MC][e % MC] = br[p][r];
    }
  };

  const int nsl = ie > ib ? (int)((ie - ib + KS - 1) / KS) : 0;
  if (nsl > 0) {
    load(0, ib);
    store(0, 0);
  }
  if (PF == 2) {
    if (1 < nsl) load(1, ib + KS);
    if (2 < nsl) load(0, ib + 2 * KS);
  }
  __syncthreads();
  for (int s = 0; s < nsl; ++s) {
    const int buf = s & 1;
    if (PF == 1 && s + 1 < nsl) load(0, ib + (int64_t)(s + 1) * KS);
    float sl[COMP ? 8 : 1][4];
    if constexpr (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) sl[a][q] = 0.f;
    }
#pragma unroll
    for (int ii = 0; ii < KS; ++ii) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][ii][ja]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][ii][ja + 32]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][ii][cb]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if constexpr (COMP) sl[a][q] = fmaf(av[a], bv[q], sl[a][q]);
          else acc[a][q] = fmaf(av[a], bv[q], acc[a][q]);
        }
      if constexpr (COMP) {
        // the first row is a slab of its own: when one term dominates (the
        // leading index of a core being expanded), the running sum of a
        // 16-row slab would be rounded at its scale 15 more times
        if (ii == 0 && s == 0) {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[a][q] = sl[a][q];
              sl[a][q] = 0.f;
            }
        }
      }
    }
    if constexpr (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float x = sl[a][q];
          const float t = __fadd_rn(acc[a][q], x);
          const float z = __fsub_rn(t, acc[a][q]);
          const float se = __fadd_rn(__fsub_rn(acc[a][q], __fsub_rn(t, z)), __fsub_rn(x, z));
          acc[a][q] = t;
          cmp[a][q] = __fadd_rn(cmp[a][q], se);
        }
    }
    if (PF == 1) {
      if (s + 1 < nsl) store(0, (s + 1) & 1);
    } else if (s + 1 < nsl) {
      // slab s+1 to shared memory; its register set takes slab s+3
      const int64_t nxt = ib + (int64_t)(s + 3) * KS;
      if (((s + 1) & 1) == 0) {
        store(0, (s + 1) & 1);
        if (s + 3 < nsl) load(0, nxt);
      } else {
        store(PF - 1, (s + 1) & 1);
        if (s + 3 < nsl) load(PF - 1, nxt);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t j = j0 + ja + (a < 4 ? a : 28 + a);
    if (j >= cols) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + cb + q;
      float v = acc[a][q];
      if constexpr (COMP) v = __fadd_rn(acc[a][q], cmp[a][q]);
      if (c < m) out[tout ? j + cols * c : (int64_t)c + (int64_t)m * j] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// part[(split*n + i)*lc + c] = sum_{j in split} X[i + n j] B(j, c), block
// (bx, by, bz): rows i0 = bx*MI.., outputs c0 = by*MC.., split bz over
// columns [bz*cps, (bz+1)*cps).  B(j, c) = W[c + l j] or Omega_k(jk, c), where
// jk = j / ka + kb (j % ka) maps the layout's column order to the unfolding's
// (ka = columns, kb = 1 for the natural layout).
// ---------------------------------------------------------------------------
// COMP: slab-compensated accumulation.  Each slab of KS columns is summed in
// FP32 from zero and folded into a (hi, lo) pair by TwoSum (correctly rounded
// adds, so nothing is contracted); the pair is written as two partial planes,
// hi to part and lo to part_lo.  Sequential FP32 sums over ~10^6 columns
// carry rounding errors of the size of their running sums, which for the
// weak directions of Y = X W are many times the result; with the fold only
// the slab sums' own rounding (a few products' worth) is left.
template <int WI, int WC, bool OMEGA, bool COMP = false, bool SHADOW = false>
__device__ __forceinline__ void xb32_body(const float* __restrict__ X, int64_t n, int64_t cols,
                                          const float* __restrict__ W, int l, int lc,
                                          uint64_t seed, uint32_t tag, int mode, int64_t cps,
                                          int64_t ka, int64_t kb, float* __restrict__ part,
                                          unsigned bx, unsigned by, unsigned bz,
                                          float* __restrict__ part_lo = nullptr,
                                          __nv_bfloat16* __restrict__ shadow = nullptr) {
  constexpr int MI = 64 * WI, MC = 16 * WC, T = 32 * WI * WC;
  constexpr int XPT = KS * MI / T;
  constexpr int BPT = (KS * MC + T - 1) / T;
  constexpr int OPT = (KS * (MC / 4) + T - 1) / T;   // Omega groups of 4 per thread
  __shared__ __align__(16) float Xs[2][KS][MI + 4];
  __shared__ __align__(16) float Bs[2][KS][MC];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wi = w % WI, wc = w / WI;
  const int li = lane >> 2, lcn = lane & 3;
  const int64_t i0 = (int64_t)bx * MI;
  const int c0 = (int)by * MC;
  const int64_t jb = (int64_t)bz * cps;
  const int64_t je = min(cols, jb + cps);
  const int ia = wi * 64 + li * 4;
  const int cb = wc * 16 + lcn * 4;

  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
  float cmp[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) cmp[a][q] = 0.f;

  float xr[XPT], br[OMEGA ? 4 * OPT : BPT];
  // shadow: the sketch pass also writes the bfloat16 copy of X (round to
  // nearest even), each element once (from the blocks of the first output
  // tile), so the precision form needs no separate conversion pass
  const bool wshadow = SHADOW && by == 0;
  auto load = [&](int64_t j0) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      const int ii = e % MI, jj = e / MI;
      const int64_t i = i0 + ii, j = j0 + jj;
      const bool in = i < n && j < je;
      xr[r] = in ? __ldg(X + j * n + i) : 0.f;
      if constexpr (SHADOW) {
        if (wshadow && in) shadow[j * n + i] = __float2bfloat16_rn(xr[r]);
      }
    }
    if (OMEGA) {
#pragma unroll
      for (int r = 0; r < OPT; ++r) {
        const int e = tid + r * T;
        float w4[4] = {0.f, 0.f, 0.f, 0.f};
        if (e < KS * (MC / 4)) {
          const int jj = e % KS, g = e / KS;
          const int64_t j = j0 + jj;
          // Omega's row is the column's index in the unfolding's own order:
          // column j = a + ka*b of this layout is row b + kb*a
          if (j < je && c0 + 4 * g < l)
            omega4((uint64_t)(j / ka + kb * (j % ka)), (c0 >> 2) + g, mode, tag, seed, w4);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) br[4 * r + q] = w4[q];
      }
    } else {
#pragma unroll
      for (int r = 0; r < BPT; ++r) {
        const int e = tid + r * T;
        float v = 0.f;
        if (e < KS * MC) {
          const int c = e % MC, jj = e / MC;
          const int64_t j = j0 + jj;
          if (j < je && c0 + c < l) v = W[(int64_t)(c0 + c) + (int64_t)l * j];
        }
        br[r] = v;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      Xs[buf][e / MI][e % MI] = xr[r];
    }
    if (OMEGA) {
#pragma unroll
      for (int r = 0; r < OPT; ++r) {
        const int e = tid + r * T;
        if (e < KS * (MC / 4)) {
          const int jj = e % KS, g = e / KS;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            Bs[buf][jj][4 * g + q] = (c0 + 4 * g + q < l) ? br[4 * r + q] : 0.f;
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < BPT; ++r) {
        const int e = tid + r * T;
        if (e < KS * MC) Bs[buf][e / MC][e % MC] = br[r];
      }
    }
  };

  const int nsl = je > jb ? (int)((je - jb + KS - 1) / KS) : 0;
  if (nsl > 0) {
    load(jb);
    store(0);
  }
  __syncthreads();
  for (int s = 0; s < nsl; ++s) {
    const int buf = s & 1;
    if (s + 1 < nsl) load(jb + (int64_t)(s + 1) * KS);
    float sl[8][4];
    if (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) sl[a][q] = 0.f;
    }
#pragma unroll
    for (int jj = 0; jj < KS; ++jj) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][jj][ia]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][jj][ia + 32]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][jj][cb]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (COMP) sl[a][q] = fmaf(av[a], bv[q], sl[a][q]);
          else acc[a][q] = fmaf(av[a], bv[q], acc[a][q]);
        }
    }
    if (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = __fadd_rn(acc[a][q], sl[a][q]);
          const float z = __fsub_rn(t, acc[a][q]);
          const float se = __fadd_rn(__fsub_rn(acc[a][q], __fsub_rn(t, z)),
                                     __fsub_rn(sl[a][q], z));
          acc[a][q] = t;
          cmp[a][q] = __fadd_rn(cmp[a][q], se);
        }
    }
    if (s + 1 < nsl) store(buf ^ 1);
    __syncthreads();
  }
  float* dst = part + (int64_t)bz * n * lc;
  float* dlo = COMP ? part_lo + (int64_t)bz * n * lc : nullptr;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + ia + (a < 4 ? a : 28 + a);
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + cb + q;
      if (c >= lc) continue;
      if (COMP) {
        const float hi = __fadd_rn(acc[a][q], cmp[a][q]);
        dst[i * lc + c] = hi;
        dlo[i * lc + c] = __fadd_rn(__fsub_rn(acc[a][q], hi), cmp[a][q]);
      } else {
        dst[i * lc + c] = acc[a][q];
      }
    }
  }
}

// Y = X_(k) W partials (W given, no bfloat16 copy) with X and W staged by
// cp.async into a ring of XB_NS shared-memory slabs: the copies of slab
// s + XB_NS - 1 are in flight while slab s is summed, and no registers hold
// staged data.  Same slabs, same order and same arithmetic as xb32_body, so
// the results are bitwise equal.  Needs n and l multiples of 4 (16-byte
// aligned rows) and dynamic shared memory xb32_cpa_smem(WI, WC).
constexpr int XB_NS = 3;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

template <int WI, int WC, bool COMP>
__device__ __forceinline__ void xb32_cpa_body(const float* __restrict__ X, int64_t n,
                                              int64_t cols, const float* __restrict__ W, int l,
                                              int lc, int64_t cps, float* __restrict__ part,
                                              unsigned bx, unsigned by, unsigned bz,
                                              float* __restrict__ part_lo) {
  constexpr int MI = 64 * WI, MC = 16 * WC, T = 32 * WI * WC;
  extern __shared__ __align__(16) float xb_dsm[];
  float* Xs = xb_dsm;                         // [XB_NS][KS][MI]
  float* Bs = xb_dsm + XB_NS * KS * MI;       // [XB_NS][KS][MC]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wi = w % WI, wc = w / WI;
  const int li = lane >> 2, lcn = lane & 3;
  const int64_t i0 = (int64_t)bx * MI;
  const int c0 = (int)by * MC;
  const int64_t jb = (int64_t)bz * cps;
  const int64_t je = min(cols, jb + cps);
  const int ia = wi * 64 + li * 4;
  const int cb = wc * 16 + lcn * 4;

  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
  float cmp[COMP ? 8 : 1][4];
#pragma unroll
  for (int a = 0; a < (COMP ? 8 : 1); ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) cmp[a][q] = 0.f;

  // slab at columns j0.. into ring slot st; entries past n, l or je are zero
  auto issue = [&](int st, int64_t j0) {
    constexpr int XC = KS * MI / 4, BC = KS * MC / 4;
    float* xs = Xs + st * KS * MI;
    float* bs = Bs + st * KS * MC;
#pragma unroll
    for (int e = tid; e < XC; e += T) {
      const int jj = e / (MI / 4), q4 = e % (MI / 4);
      const int64_t j = j0 + jj, i = i0 + 4 * q4;
      const bool in = j < je && i < n;
      cp_async16((uint32_t)__cvta_generic_to_shared(xs + jj * MI + 4 * q4),
                 in ? (const void*)(X + j * n + i) : (const void*)X, in ? 16 : 0);
    }
#pragma unroll
    for (int e = tid; e < BC; e += T) {
      const int jj = e / (MC / 4), q4 = e % (MC / 4);
      const int64_t j = j0 + jj;
      const int c = c0 + 4 * q4;
      const bool in = j < je && c < l;
      cp_async16((uint32_t)__cvta_generic_to_shared(bs + jj * MC + 4 * q4),
                 in ? (const void*)(W + (int64_t)l * j + c) : (const void*)W, in ? 16 : 0);
    }
  };

  const int nsl = je > jb ? (int)((je - jb + KS - 1) / KS) : 0;
#pragma unroll
  for (int st = 0; st < XB_NS - 1; ++st) {
    if (st < nsl) issue(st, jb + (int64_t)st * KS);
    cp_async_commit();
  }
  for (int s = 0; s < nsl; ++s) {
    cp_async_wait<XB_NS - 2>();
    __syncthreads();     // slab s landed for every thread; slot (s - 1) % XB_NS is free
    {
      const int nx = s + XB_NS - 1;
      if (nx < nsl) issue(nx % XB_NS, jb + (int64_t)nx * KS);
      cp_async_commit();
    }
    const float* xs = Xs + (s % XB_NS) * KS * MI;
    const float* bs = Bs + (s % XB_NS) * KS * MC;
    float sl[COMP ? 8 : 1][4];
    if constexpr (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) sl[a][q] = 0.f;
    }
#pragma unroll
    for (int jj = 0; jj < KS; ++jj) {
      const float4 a0 = *reinterpret_cast<const float4*>(xs + jj * MI + ia);
      const float4 a1 = *reinterpret_cast<const float4*>(xs + jj * MI + ia + 32);
      const float4 b = *reinterpret_cast<const float4*>(bs + jj * MC + cb);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if constexpr (COMP) sl[a][q] = fmaf(av[a], bv[q], sl[a][q]);
          else acc[a][q] = fmaf(av[a], bv[q], acc[a][q]);
        }
    }
    if constexpr (COMP) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = __fadd_rn(acc[a][q], sl[a][q]);
          const float z = __fsub_rn(t, acc[a][q]);
          const float se = __fadd_rn(__fsub_rn(acc[a][q], __fsub_rn(t, z)),
                                     __fsub_rn(sl[a][q], z));
          acc[a][q] = t;
          cmp[a][q] = __fadd_rn(cmp[a][q], se);
        }
    }
  }
  cp_async_wait<0>();
  float* dst = part + (int64_t)bz * n * lc;
  float* dlo = COMP ? part_lo + (int64_t)bz * n * lc : nullptr;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + ia + (a < 4 ? a : 28 + a);
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + cb + q;
      if (c >= lc) continue;
      if constexpr (COMP) {
        const float hi = __fadd_rn(acc[a][q], cmp[a][q]);
        dst[i * lc + c] = hi;
        dlo[i * lc + c] = __fadd_rn(__fsub_rn(acc[a][q], hi), cmp[a][q]);
      } else {
        dst[i * lc + c] = acc[a][q];
      }
    }
  }
}

template <int WI, int WC, bool COMP>
__global__ void __launch_bounds__(32 * WI * WC)
k_xb32_cpa(const float* __restrict__ X, int64_t n, int64_t cols, const float* __restrict__ W,
           int l, int lc, int64_t cps, float* __restrict__ part, float* __restrict__ part_lo) {
  xb32_cpa_body<WI, WC, COMP>(X, n, cols, W, l, lc, cps, part, blockIdx.x, blockIdx.y,
                              blockIdx.z, part_lo);
}

template <int WJ, int WC, typename BT, bool COMP = false>
__global__ void __launch_bounds__(32 * WJ * WC, COMP ? 2 : 1)
k_xtb32(const float* __restrict__ X, int64_t n, int64_t cols, const BT* __restrict__ B,
        int64_t b_ri, int64_t b_cm, int m, float* __restrict__ out, int tout, int64_t kps,
        float* __restrict__ part) {
  // split z of the rows writes its partial sums to part (layout c + m j)
  const int64_t ib = (int64_t)blockIdx.z * kps, ie = min(n, ib + kps);
  float* o = part ? part + (int64_t)blockIdx.z * cols * m : out;
  xtb32_body<WJ, WC, BT, COMP>(X, n, cols, B, b_ri, b_cm, m, o, part ? 0 : tout, ib, ie,
                               blockIdx.x, blockIdx.y);
}

// out = sum over the ks row splits of the partials, in a fixed order.
__device__ __forceinline__ void xtb32_red_body(const float* __restrict__ part, int ks,
                                               int64_t cols, int m, int tout,
                                               float* __restrict__ out, unsigned bx) {
  const int64_t e = (int64_t)bx * 256 + threadIdx.x;
  if (e >= cols * m) return;
  float s = 0.f;
  for (int z = 0; z < ks; ++z) s += part[(int64_t)z * cols * m + e];
  const int64_t c = e % m, j = e / m;
  out[tout ? j + cols * c : e] = s;
}

__global__ void __launch_bounds__(256)
k_xtb32_red(const float* __restrict__ part, int ks, int64_t cols, int m, int tout,
            float* __restrict__ out) {
  xtb32_red_body(part, ks, cols, m, tout, out, blockIdx.x);
}

__global__ void __launch_bounds__(256)
k_xtb32_red_batch(const Xtb32RedJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                  int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const Xtb32RedJob J = jobs[j];
    xtb32_red_body((const float*)J.part, J.ks, J.cols, J.m, J.tout, (float*)J.out,
                   b - __ldg(start + j));
  }
}

template <int WI, int WC, bool OMEGA, bool COMP = false, bool SHADOW = false>
__global__ void __launch_bounds__(32 * WI * WC)
k_xb32(const float* __restrict__ X, int64_t n, int64_t cols, const float* __restrict__ W, int l,
       int lc, uint64_t seed, uint32_t tag, int mode, int64_t cps, int64_t ka, int64_t kb,
       float* __restrict__ part, float* __restrict__ part_lo,
       __nv_bfloat16* __restrict__ shadow) {
  xb32_body<WI, WC, OMEGA, COMP, SHADOW>(X, n, cols, W, l, lc, seed, tag, mode, cps, ka, kb,
                                         part, blockIdx.x, blockIdx.y, blockIdx.z, part_lo,
                                         shadow);
}

template <int WJ, int WC, bool COMP>
__global__ void __launch_bounds__(32 * WJ * WC, COMP ? 2 : 1)
k_xtb32_batch(const Xtb32Job* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
              uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const Xtb32Job J = jobs[j];
    const uint32_t lb = b - __ldg(start + j);
    const uint32_t gxy = (uint32_t)J.gx * (uint32_t)J.gy, z = lb / gxy, r = lb % gxy;
    const int64_t ib = (int64_t)z * J.kps, ie = min(J.n, ib + J.kps);
    float* o = J.part ? (float*)J.part + (int64_t)z * J.cols * J.m : (float*)J.out;
    xtb32_body<WJ, WC, float, COMP>((const float*)J.X, J.n, J.cols, J.B, J.b_ri, J.b_cm, J.m, o,
                       J.part ? 0 : J.tout, ib, ie, r % (uint32_t)J.gx, r / (uint32_t)J.gx);
    __syncthreads();
  }
}

template <int WI, int WC, bool OMEGA, bool COMP = false>
__global__ void __launch_bounds__(32 * WI * WC)
k_xb32_batch(const Xb32Job* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
             uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const Xb32Job J = jobs[j];
    const uint32_t lb = b - __ldg(start + j);
    const uint32_t gxy = (uint32_t)J.gx * (uint32_t)J.gy;
    const uint32_t r = lb % gxy;
    xb32_body<WI, WC, OMEGA, COMP>((const float*)J.X, J.n, J.cols, (const float*)J.W, J.l,
                                   J.lc, J.seed, J.tag, J.mode, J.cps, J.ka, J.kb,
                                   (float*)J.part, r % (uint32_t)J.gx, r / (uint32_t)J.gx,
                                   lb / gxy, (float*)J.part_lo);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Last-mode expansion fused with the error sums (relative error, Section 5):
// for S == 1, a_hat(p, c) = sum_{i < K} T[p + P i] B(i, c) with B(i, c) =
// Bm[i*b_ri + c*b_cm]; the block adds (A[p + P c] - a_hat)^2 and A^2 over its
// 128 x 64 tile (p, c) and writes the two sums to err[2 blk], blk = by gx + bx.
// a_hat is never stored.  Thread tile 8 p x 4 c (lanes 8 x 4, warps 2 x 4).
// ---------------------------------------------------------------------------
template <typename BT>
__device__ __forceinline__ void err32_body(const float* __restrict__ Tt, int64_t P, int K,
                                           const BT* __restrict__ Bm, int64_t b_ri,
                                           int64_t b_cm, int m, const float* __restrict__ A,
                                           double* __restrict__ err, unsigned bx, unsigned by,
                                           unsigned gx) {
  constexpr int MP = 128, MC = 64, T = 256;
  constexpr int XPT = KS * MP / T;                  // 8
  constexpr int BPT = KS * MC / T;                  // 4
  __shared__ __align__(16) float Ts[2][KS][MP + 4];
  __shared__ __align__(16) float Bs[2][KS][MC];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wp = w & 1, wc = w >> 1;
  const int lp = lane >> 2, lc = lane & 3;
  const int64_t p0 = (int64_t)bx * MP;
  const int c0 = (int)by * MC;
  const int pa = wp * 64 + lp * 4;
  const int cb = wc * 16 + lc * 4;
  // The accumulator starts at a(p, c) and every product is subtracted from
  // it, so it holds the running residual a - sum_{i<t} T(p,i) B(i,c): after
  // the leading term it is already at the scale of the remaining terms, and
  // the roundings are relative to that, not to a_hat.  (Summing a_hat first
  // and subtracting at the end rounds every FMA at the scale of a_hat, which
  // on the workloads here is ~1e6 times the residual.)
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t p = p0 + pa + (a < 4 ? a : 28 + a);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + cb + q;
      acc[a][q] = (p < P && c < m) ? __ldg(A + p + P * c) : 0.f;
    }
  }
  float tr[XPT], br[BPT];
  auto load = [&](int i0) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      const int pp = e % MP, ii = e / MP;
      const int64_t p = p0 + pp;
      const int i = i0 + ii;
      tr[r] = (p < P && i < K) ? __ldg(Tt + p + P * i) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < BPT; ++r) {
      const int e = tid + r * T;
      const int c = e % MC, ii = e / MC;
      const int i = i0 + ii;
      br[r] = (i < K && c0 + c < m) ? (float)Bm[(int64_t)i * b_ri + (int64_t)(c0 + c) * b_cm]
                                    : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < XPT; ++r) {
      const int e = tid + r * T;
      Ts[buf][e / MP][e % MP] = tr[r];
    }
#pragma unroll
    for (int r = 0; r < BPT; ++r) {
      const int e = tid + r * T;
      Bs[buf][e / MC][e % MC] = br[r];
    }
  };
  const int nsl = (K + KS - 1) / KS;
  load(0);
  store(0);
  __syncthreads();
  for (int s = 0; s < nsl; ++s) {
    const int buf = s & 1;
    if (s + 1 < nsl) load((s + 1) * KS);
    // rows past K in the last slab are zero: skipping them leaves every sum
    // unchanged (K = r_d is often far from a multiple of KS)
    const int rows = min(KS, K - s * KS);
#pragma unroll
    for (int ii = 0; ii < KS; ++ii) {
      if (ii >= rows) break;
      const float4 a0 = *reinterpret_cast<const float4*>(&Ts[buf][ii][pa]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Ts[buf][ii][pa + 32]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][ii][cb]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {-b.x, -b.y, -b.z, -b.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(av[a], bv[q], acc[a][q]);
    }
    if (s + 1 < nsl) store(buf ^ 1);
    __syncthreads();
  }
  // squared differences: per-thread FP32 sums of 32 terms, then FP64
  float e2t = 0.f, a2t = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = c0 + cb + q;
    if (c >= m) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t p = p0 + pa + (a < 4 ? a : 28 + a);
      if (p >= P) continue;
      const float av = __ldg(A + p + P * c);
      const float dv = acc[a][q];
      e2t = fmaf(dv, dv, e2t);
      a2t = fmaf(av, av, a2t);
    }
  }
  double e2 = (double)e2t, a2 = (double)a2t;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    red[0][w] = e2;
    red[1][w] = a2;
  }
  __syncthreads();
  if (tid == 0) {
    double se = 0.0, sa = 0.0;
    for (int k = 0; k < 8; ++k) {
      se += red[0][k];
      sa += red[1][k];
    }
    const int64_t blk = (int64_t)by * gx + bx;
    err[2 * blk] = se;
    err[2 * blk + 1] = sa;
  }
  __syncthreads();
}

template <typename BT>
__global__ void __launch_bounds__(256)
k_err32(const float* __restrict__ Tt, int64_t P, int K, const BT* __restrict__ Bm,
        int64_t b_ri, int64_t b_cm, int m, const float* __restrict__ A,
        double* __restrict__ err) {
  err32_body<BT>(Tt, P, K, Bm, b_ri, b_cm, m, A, err, blockIdx.x, blockIdx.y, gridDim.x);
}

// The same tiles with the output blocks of one row tile adjacent in launch
// order (grid x = output blocks, y = row tiles): they share the row tile of
// T, which then comes from L2 instead of being read from HBM once per
// output block.  Tiles, sums and partial slots are those of k_err32.
template <typename BT>
__global__ void __launch_bounds__(256)
k_err32_t(const float* __restrict__ Tt, int64_t P, int K, const BT* __restrict__ Bm,
          int64_t b_ri, int64_t b_cm, int m, const float* __restrict__ A,
          double* __restrict__ err) {
  err32_body<BT>(Tt, P, K, Bm, b_ri, b_cm, m, A, err, blockIdx.y, blockIdx.x, gridDim.y);
}

// The same residual sums with one CTA per row tile and ERR_CT consecutive
// output tiles (K <= ERR_KMAX): T's row tile (K x 128) and B's rows for the
// CTA's 256 outputs are staged in shared memory once, and each output tile's
// A block is loaded into registers while the previous tile is summed.  Every
// residual entry and every per-thread FP32 sum of squares is formed exactly
// as in err32_body (same terms, same order); only the FP64 sums over the
// output tiles are grouped per CTA.  Block lb of the launch is row tile
// lb / groups, output group lb % groups (groups = ceil(m / (64 ERR_CT))).
// Dynamic shared memory: err32c_smem(K).
constexpr int ERR_CT = 4;
constexpr int ERR_KMAX = 64;

template <typename BT>
__device__ __forceinline__ void err32c_body(const float* __restrict__ Tt, int64_t P, int K,
                                            const BT* __restrict__ Bm, int64_t b_ri,
                                            int64_t b_cm, int m, const float* __restrict__ A,
                                            double* __restrict__ err, uint32_t lb) {
  constexpr int MP = 128, MC = 64, T = 256, TS = MP + 4, BW = ERR_CT * MC;
  extern __shared__ __align__(16) float err_dsm[];
  float* Ts = err_dsm;                // [K][TS]
  float* Bs = err_dsm + K * TS;       // [K][BW]
  __shared__ double red[2][8];
  const int groups = (m + BW - 1) / BW;
  const int64_t ptile = lb / (uint32_t)groups;
  const int g = (int)(lb % (uint32_t)groups);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wp = w & 1, wc = w >> 1;
  const int lp = lane >> 2, lcn = lane & 3;
  const int64_t p0 = ptile * MP;
  const int cg0 = g * BW;
  const int pa = wp * 64 + lp * 4;
  const int cb = wc * 16 + lcn * 4;

  // A block of output tile ct, as err32_body's accumulator starts
  float an[8][4];
  auto load_a = [&](int ct) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t p = p0 + pa + (a < 4 ? a : 28 + a);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = cg0 + ct * MC + cb + q;
        an[a][q] = (p < P && c < m) ? __ldg(A + p + P * c) : 0.f;
      }
    }
  };
  load_a(0);
  for (int e = tid; e < K * MP; e += T) {
    const int i = e / MP, pp = e % MP;
    const int64_t p = p0 + pp;
    Ts[i * TS + pp] = p < P ? __ldg(Tt + p + P * i) : 0.f;
  }
  for (int e = tid; e < K * BW; e += T) {
    const int i = e / BW, cc = e % BW;
    const int c = cg0 + cc;
    Bs[i * BW + cc] = c < m ? (float)Bm[(int64_t)i * b_ri + (int64_t)c * b_cm] : 0.f;
  }
  __syncthreads();
  double e2 = 0.0, a2 = 0.0;
  for (int ct = 0; ct < ERR_CT; ++ct) {
    const int cbase = cg0 + ct * MC;
    if (cbase >= m) break;             // uniform over the CTA
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][q] = an[a][q];
    if (ct + 1 < ERR_CT && cbase + MC < m) load_a(ct + 1);
    // squares of a over the tile, in the order of err32_body's second read
    float a2t = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (cbase + cb + q >= m) continue;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (p0 + pa + (a < 4 ? a : 28 + a) >= P) continue;
        a2t = fmaf(acc[a][q], acc[a][q], a2t);
      }
    }
    // the running residual a - sum_{i<t} T(p,i) B(i,c), terms in ascending i
    const float* bcol = Bs + ct * MC + cb;
#pragma unroll 4
    for (int i = 0; i < K; ++i) {
      const float4 a0 = *reinterpret_cast<const float4*>(Ts + i * TS + pa);
      const float4 a1 = *reinterpret_cast<const float4*>(Ts + i * TS + pa + 32);
      const float4 b = *reinterpret_cast<const float4*>(bcol + i * BW);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {-b.x, -b.y, -b.z, -b.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(av[a], bv[q], acc[a][q]);
    }
    float e2t = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (cbase + cb + q >= m) continue;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (p0 + pa + (a < 4 ? a : 28 + a) >= P) continue;
        e2t = fmaf(acc[a][q], acc[a][q], e2t);
      }
    }
    e2 += (double)e2t;
    a2 += (double)a2t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    red[0][w] = e2;
    red[1][w] = a2;
  }
  __syncthreads();
  if (tid == 0) {
    double se = 0.0, sa = 0.0;
    for (int k = 0; k < 8; ++k) {
      se += red[0][k];
      sa += red[1][k];
    }
    err[2 * (int64_t)lb] = se;
    err[2 * (int64_t)lb + 1] = sa;
  }
  __syncthreads();
}

template <typename BT>
__global__ void __launch_bounds__(256, 2)
k_err32c(const float* __restrict__ Tt, int64_t P, int K, const BT* __restrict__ Bm,
         int64_t b_ri, int64_t b_cm, int m, const float* __restrict__ A,
         double* __restrict__ err) {
  err32c_body<BT>(Tt, P, K, Bm, b_ri, b_cm, m, A, err, blockIdx.x);
}

__global__ void __launch_bounds__(256, 2)
k_err32c_batch(const Err32Job* __restrict__ jobs, const uint32_t* __restrict__ start,
               int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const Err32Job J = jobs[j];
    err32c_body<float>((const float*)J.T, J.P, J.K, J.B, J.b_ri, J.b_cm, J.m,
                       (const float*)J.A, J.err, b - __ldg(start + j));
  }
}

__global__ void __launch_bounds__(256)
k_err32_batch(const Err32Job* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
              uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const Err32Job J = jobs[j];
    const uint32_t lb = b - __ldg(start + j);
    // output blocks of one row tile adjacent (they share its rows of T)
    const uint32_t gy = (uint32_t)((J.m + 63) / 64);
    err32_body<float>((const float*)J.T, J.P, J.K, J.B, J.b_ri, J.b_cm, J.m, (const float*)J.A,
                       J.err, lb / gy, lb % gy, (uint32_t)J.gx);
  }
}

}  // namespace c32

// ---------------------------------------------------------------------------
// Shapes.  Outputs per block: 16 WC (WC = 1, 2, 4 for up to 16, 32, 64
// outputs; more outputs take several blocks along y).  Rows per block for
// k_xb32: 64 WI with WI = 1, 2 or 4 by n.
// ---------------------------------------------------------------------------
static int wc_of(int m) { return m <= 16 ? 1 : (m <= 32 ? 2 : 4); }
static int wi_of(int64_t n) { return n <= 64 ? 1 : (n <= 128 ? 2 : 4); }
static int wj_of(int wc) { return wc == 4 ? 2 : 4; }

bool xtb32_ok(XType xt, View v, const void* X) {
  return xt == X_F32 && v.P == 1 && v.n >= 1 && v.cols() >= 1 && X != nullptr;
}

Xtb32Shape xtb32_shape(View v, int m, bool allow_split) {
  Xtb32Shape s;
  s.wc = wc_of(m);
  s.wj = wj_of(s.wc);
  s.gx = (int)((v.cols() + 64 * s.wj - 1) / (64 * s.wj));
  s.gy = (m + 16 * s.wc - 1) / (16 * s.wc);
  s.threads = 32 * s.wj * s.wc;
  // few column tiles: split the rows too (partials + a fixed-order sum),
  // so that about two CTAs per SM work; each split keeps >= 64 rows
  s.ks = 1;
  const int64_t tiles = (int64_t)s.gx * s.gy;
  if (allow_split && tiles < num_sms()) {
    const int64_t want = (2LL * num_sms() + tiles - 1) / tiles;
    const int64_t maxk = std::max<int64_t>(1, v.n / 64);
    s.ks = (int)std::max<int64_t>(1, std::min(want, maxk));
    s.ks = tune_splits(TUNE_XTB32, v.n, m, v.cols(), s.ks, (int)maxk);
  }
  int64_t kps = (v.n + s.ks - 1) / s.ks;
  kps = (kps + c32::KS - 1) / c32::KS * c32::KS;
  s.kps = kps;
  s.ks = (int)((v.n + kps - 1) / kps);
  return s;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// scratch: the row-split partials (when the rows are split), then B in FP32
// (n x m): converting B once here instead of per element in every CTA
size_t xtb32_b32_offset(View v, int m) {
  const Xtb32Shape s = xtb32_shape(v, m, true);
  return s.ks > 1 ? al256((size_t)s.ks * v.cols() * m * sizeof(float)) : 0;
}
size_t xtb32_scratch(View v, int m) {
  return xtb32_b32_offset(v, m) + al256((size_t)v.n * m * sizeof(float));
}

Xb32Shape xb32_shape(View v, int l, int splits_req) {
  Xb32Shape s;
  s.lc = xb_lc(l);
  s.wc = wc_of(std::min(s.lc, 64));
  s.wi = wi_of(v.n);
  s.gx = (int)((v.n + 64 * s.wi - 1) / (64 * s.wi));
  s.gy = (s.lc + 16 * s.wc - 1) / (16 * s.wc);
  int64_t splits = splits_req;
  if (splits <= 0) {
    // about 3 CTAs per SM in total, at least 4 slabs of columns per split
    const int64_t target = 3LL * num_sms();
    splits = (target + (int64_t)s.gx * s.gy - 1) / ((int64_t)s.gx * s.gy);
    const int64_t maxs = std::max<int64_t>(1, (v.cols() + 4 * c32::KS - 1) / (4 * c32::KS));
    splits = std::max<int64_t>(1, std::min(splits, maxs));
    splits = tune_splits(TUNE_XB32, v.n, s.lc, v.cols(), (int)splits,
                         (int)std::min<int64_t>(maxs, 1 << 20));
  }
  int64_t cps = (v.cols() + splits - 1) / splits;
  cps = (cps + c32::KS - 1) / c32::KS * c32::KS;
  // every split writes its partial block (splits past the last column write
  // zeros), so the reduction may sum exactly `splits` blocks
  s.splits = (int)splits;
  s.cps = cps;
  s.threads = 32 * s.wi * s.wc;
  return s;
}

template <int WJ, int WC, typename BT, bool COMP>
static void xtb32_go(const float* X, View v, const BT* B, int64_t b_ri, int64_t b_cm, int m,
                     float* out, int tout, float* part, const Xtb32Shape& s, cudaStream_t st) {
  c32::k_xtb32<WJ, WC, BT, COMP><<<dim3(s.gx, s.gy, s.ks), 32 * WJ * WC, 0, st>>>(
      X, v.n, v.cols(), B, b_ri, b_cm, m, out, tout, s.kps, s.ks > 1 ? part : nullptr);
}

template <typename BT, bool COMP>
static void xtb32_wcc(const float* X, View v, const BT* B, int64_t b_ri, int64_t b_cm, int m,
                      float* out, int tout, float* part, const Xtb32Shape& s, cudaStream_t st) {
  switch (s.wc) {
    case 1: xtb32_go<4, 1, BT, COMP>(X, v, B, b_ri, b_cm, m, out, tout, part, s, st); break;
    case 2: xtb32_go<4, 2, BT, COMP>(X, v, B, b_ri, b_cm, m, out, tout, part, s, st); break;
    default: xtb32_go<2, 4, BT, COMP>(X, v, B, b_ri, b_cm, m, out, tout, part, s, st); break;
  }
}

template <typename BT>
static void xtb32_wc(const float* X, View v, const BT* B, int64_t b_ri, int64_t b_cm, int m,
                     float* out, int tout, float* part, const Xtb32Shape& s, cudaStream_t st,
                     bool comp) {
  if (comp) xtb32_wcc<BT, true>(X, v, B, b_ri, b_cm, m, out, tout, part, s, st);
  else xtb32_wcc<BT, false>(X, v, B, b_ri, b_cm, m, out, tout, part, s, st);
}

namespace c32 {
// out[i + n c] = (float) B[i b_ri + c b_cm]
__global__ void __launch_bounds__(256) k_b_to_f32(const double* __restrict__ B, int64_t b_ri,
                                                  int64_t b_cm, int64_t n, int m,
                                                  float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= n * m) return;
  const int64_t i = e % n, c = e / n;
  out[e] = (float)B[i * b_ri + c * b_cm];
}
}  // namespace c32

// With scratch (sized by xtb32_scratch), B is first rounded to FP32 once;
// without, every CTA rounds the entries it stages.  The products are the
// same either way (each FMA sees (float)B).
cudaError_t launch_xtb32(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                         int m, void* out, cudaStream_t st, int tout, void* scratch,
                         const float* B32, bool comp) {
  if (v.cols() <= 0 || m <= 0) return cudaSuccess;
  const Xtb32Shape s = xtb32_shape(v, m, scratch != nullptr);
  const float* x = (const float*)X;
  float* o = (float*)out;
  float* part = (float*)scratch;
  if (B32 != nullptr) {
    count_kernels(s.ks > 1 ? 2 : 1);
    xtb32_wc(x, v, B32, b_ri, b_cm, m, o, tout, part, s, st, comp);
  } else if (scratch == nullptr) {
    count_kernels(1);
    xtb32_wc(x, v, B, b_ri, b_cm, m, o, tout, (float*)nullptr, s, st, comp);
    return cudaGetLastError();
  } else {
    float* b32 = (float*)((unsigned char*)scratch + xtb32_b32_offset(v, m));
    count_kernels(s.ks > 1 ? 3 : 2);
    const int64_t nb = v.n * m;
    c32::k_b_to_f32<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(B, b_ri, b_cm, v.n, m, b32);
    xtb32_wc(x, v, (const float*)b32, 1, v.n, m, o, tout, part, s, st, comp);
  }
  if (s.ks > 1) {
    const int64_t tot = v.cols() * m;
    c32::k_xtb32_red<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, s.ks, v.cols(), m,
                                                                      tout, o);
  }
  return cudaGetLastError();
}

// the cp.async-staged form applies: W given, rows 16-byte aligned
static bool xb32_cpa_ok(const float* X, View v, const float* W, int l,
                        const __nv_bfloat16* shadow) {
  return W != nullptr && shadow == nullptr && (v.n % 4) == 0 && (l % 4) == 0 &&
         (((uintptr_t)X) & 15) == 0 && (((uintptr_t)W) & 15) == 0;
}

template <int WI, int WC, bool COMP>
static void xb32_cpa_go(const float* X, View v, const float* W, int l, float* part,
                        float* part_lo, const Xb32Shape& s, const dim3& grid, cudaStream_t st) {
  const size_t smem =
      (size_t)c32::XB_NS * c32::KS * (64 * WI + 16 * WC) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(c32::k_xb32_cpa<WI, WC, COMP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  c32::k_xb32_cpa<WI, WC, COMP><<<grid, 32 * WI * WC, smem, st>>>(X, v.n, v.cols(), W, l, s.lc,
                                                                  s.cps, part, part_lo);
}

template <int WI, int WC>
static void xb32_go(const float* X, View v, const float* W, int l, uint64_t seed, uint32_t tag,
                    int mode, float* part, int64_t ka, int64_t kb, const Xb32Shape& s,
                    cudaStream_t st, float* part_lo, __nv_bfloat16* shadow) {
  const dim3 grid(s.gx, s.gy, s.splits);
  if (xb32_cpa_ok(X, v, W, l, shadow)) {
    if (part_lo != nullptr) xb32_cpa_go<WI, WC, true>(X, v, W, l, part, part_lo, s, grid, st);
    else xb32_cpa_go<WI, WC, false>(X, v, W, l, part, nullptr, s, grid, st);
    return;
  }
  if (W == nullptr && shadow != nullptr)
    c32::k_xb32<WI, WC, true, false, true><<<grid, 32 * WI * WC, 0, st>>>(
        X, v.n, v.cols(), nullptr, l, s.lc, seed, tag, mode, s.cps, ka, kb, part, nullptr,
        shadow);
  else if (W == nullptr)
    c32::k_xb32<WI, WC, true><<<grid, 32 * WI * WC, 0, st>>>(X, v.n, v.cols(), nullptr, l, s.lc,
                                                             seed, tag, mode, s.cps, ka, kb, part,
                                                             nullptr, nullptr);
  else if (part_lo != nullptr)
    c32::k_xb32<WI, WC, false, true><<<grid, 32 * WI * WC, 0, st>>>(
        X, v.n, v.cols(), W, l, s.lc, seed, tag, mode, s.cps, ka, kb, part, part_lo, nullptr);
  else
    c32::k_xb32<WI, WC, false><<<grid, 32 * WI * WC, 0, st>>>(X, v.n, v.cols(), W, l, s.lc,
                                                              seed, tag, mode, s.cps, ka, kb,
                                                              part, nullptr, nullptr);
}

template <int WI>
static void xb32_wc(const float* X, View v, const float* W, int l, uint64_t seed, uint32_t tag,
                    int mode, float* part, int64_t ka, int64_t kb, const Xb32Shape& s,
                    cudaStream_t st, float* part_lo, __nv_bfloat16* shadow) {
  switch (s.wc) {
    case 1: xb32_go<WI, 1>(X, v, W, l, seed, tag, mode, part, ka, kb, s, st, part_lo, shadow); break;
    case 2: xb32_go<WI, 2>(X, v, W, l, seed, tag, mode, part, ka, kb, s, st, part_lo, shadow); break;
    default: xb32_go<WI, 4>(X, v, W, l, seed, tag, mode, part, ka, kb, s, st, part_lo, shadow); break;
  }
}

cudaError_t launch_xb32(const void* X, View v, const void* W, int l, uint64_t seed, uint32_t tag,
                        int mode, void* part, int splits, cudaStream_t st, int64_t ka,
                        int64_t kb, void* part_lo, void* shadow) {
  if (ka <= 0) {   // natural layout: the identity map
    ka = v.cols();
    kb = 1;
  }
  if (v.n <= 0 || v.cols() <= 0 || l <= 0) return cudaSuccess;
  const Xb32Shape s = xb32_shape(v, l, splits);
  count_kernels(1);
  const float* x = (const float*)X;
  const float* w = (const float*)W;
  float* p = (float*)part;
  float* plo = W != nullptr ? (float*)part_lo : nullptr;
  __nv_bfloat16* sh = W == nullptr ? (__nv_bfloat16*)shadow : nullptr;
  switch (s.wi) {
    case 1: xb32_wc<1>(x, v, w, l, seed, tag, mode, p, ka, kb, s, st, plo, sh); break;
    case 2: xb32_wc<2>(x, v, w, l, seed, tag, mode, p, ka, kb, s, st, plo, sh); break;
    default: xb32_wc<4>(x, v, w, l, seed, tag, mode, p, ka, kb, s, st, plo, sh); break;
  }
  return cudaGetLastError();
}

bool err32_ok(XType xt, View v) { return xt == X_F32 && v.S == 1 && v.P >= 1; }

// the row-tile form (err32c) for K = n_k <= ERR_KMAX
bool err32c_ok(View v) { return v.n >= 1 && v.n <= c32::ERR_KMAX; }
size_t err32c_smem(int K) {
  return (size_t)K * ((128 + 4) + c32::ERR_CT * 64) * sizeof(float);
}

int err32_blocks(View v, int m) {
  if (err32c_ok(v))
    return (int)(((v.P + 127) / 128) * ((m + 64 * c32::ERR_CT - 1) / (64 * c32::ERR_CT)));
  return (int)(((v.P + 127) / 128) * ((m + 63) / 64));
}

void c32_batch_init() {
  static bool attr = false;
  if (attr) return;
  cudaFuncSetAttribute(c32::k_err32c_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)err32c_smem(c32::ERR_KMAX));
  attr = true;
}

cudaError_t launch_err32(const void* T, View v, const double* B, int64_t b_ri, int64_t b_cm,
                         int m, const void* A, double* err_part, cudaStream_t st,
                         const float* B32) {
  if (v.P <= 0 || m <= 0) return cudaSuccess;
  if (err32c_ok(v)) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(c32::k_err32c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)err32c_smem(c32::ERR_KMAX));
      cudaFuncSetAttribute(c32::k_err32c<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)err32c_smem(c32::ERR_KMAX));
      attr = true;
    }
    const unsigned nb = (unsigned)err32_blocks(v, m);
    const size_t smem = err32c_smem((int)v.n);
    count_kernels(1);
    if (B32 != nullptr)
      c32::k_err32c<float><<<nb, 256, smem, st>>>((const float*)T, v.P, (int)v.n, B32, b_ri,
                                                  b_cm, m, (const float*)A, err_part);
    else
      c32::k_err32c<double><<<nb, 256, smem, st>>>((const float*)T, v.P, (int)v.n, B, b_ri,
                                                   b_cm, m, (const float*)A, err_part);
    return cudaGetLastError();
  }
  const unsigned gx = (unsigned)((v.P + 127) / 128), gy = (unsigned)((m + 63) / 64);
  count_kernels(1);
  if (gx <= 65535u) {
    // output blocks of a row tile adjacent: T's row tile is read from HBM once
    if (B32 != nullptr)
      c32::k_err32_t<float><<<dim3(gy, gx), 256, 0, st>>>(
          (const float*)T, v.P, (int)v.n, B32, b_ri, b_cm, m, (const float*)A, err_part);
    else
      c32::k_err32_t<double><<<dim3(gy, gx), 256, 0, st>>>(
          (const float*)T, v.P, (int)v.n, B, b_ri, b_cm, m, (const float*)A, err_part);
    return cudaGetLastError();
  }
  const dim3 grid(gx, gy);
  if (B32 != nullptr)
    c32::k_err32<float><<<grid, 256, 0, st>>>((const float*)T, v.P, (int)v.n, B32, b_ri, b_cm, m,
                                              (const float*)A, err_part);
  else
    c32::k_err32<double><<<grid, 256, 0, st>>>((const float*)T, v.P, (int)v.n, B, b_ri, b_cm, m,
                                               (const float*)A, err_part);
  return cudaGetLastError();
}

// Work-list launches: tile = WC; xtb32: flag = compensated | WJ << 1; xb32:
// flag = omega | WI << 1 | compensated << 4.
cudaError_t launch_batch_c32(const BatchLaunch& b, cudaStream_t st) {
  const int wc = b.tile, wx = (b.flag >> 1) & 7, omega = b.flag & 1;
  const bool comp_y = (b.flag >> 4) & 1;
  if (b.kind == BK_XTB32RED) return run_batch(c32::k_xtb32_red_batch, b, 256, st);
  if (b.kind == BK_ERR32) {
    // flag 1: the row-tile form (err32c_ok), dynamic shared memory in smem
    if (b.flag == 1) return run_batch(c32::k_err32c_batch, b, 256, st);
    return run_batch(c32::k_err32_batch, b, 256, st);
  }
  if (b.kind == BK_XTB32) {
    const bool comp = (b.flag & 1) != 0;
    if (wc == 1)
      return comp ? run_batch(c32::k_xtb32_batch<4, 1, true>, b, 128, st)
                  : run_batch(c32::k_xtb32_batch<4, 1, false>, b, 128, st);
    if (wc == 2)
      return comp ? run_batch(c32::k_xtb32_batch<4, 2, true>, b, 256, st)
                  : run_batch(c32::k_xtb32_batch<4, 2, false>, b, 256, st);
    return comp ? run_batch(c32::k_xtb32_batch<2, 4, true>, b, 256, st)
                : run_batch(c32::k_xtb32_batch<2, 4, false>, b, 256, st);
  }
  if (b.kind != BK_XB32) return cudaErrorInvalidValue;
#define TK_XB32_CASE(WI, WC)                                                              \
  if (wx == WI && wc == WC)                                                               \
    return omega ? run_batch(c32::k_xb32_batch<WI, WC, true>, b, 32 * WI * WC, st)        \
                 : (comp_y ? run_batch(c32::k_xb32_batch<WI, WC, false, true>, b,           \
                                       32 * WI * WC, st)                                 \
                           : run_batch(c32::k_xb32_batch<WI, WC, false>, b, 32 * WI * WC, st));
  TK_XB32_CASE(1, 1)
  TK_XB32_CASE(1, 2)
  TK_XB32_CASE(1, 4)
  TK_XB32_CASE(2, 1)
  TK_XB32_CASE(2, 2)
  TK_XB32_CASE(2, 4)
  TK_XB32_CASE(4, 1)
  TK_XB32_CASE(4, 2)
  TK_XB32_CASE(4, 4)
#undef TK_XB32_CASE
  return cudaErrorInvalidValue;
}

}  // namespace tk
