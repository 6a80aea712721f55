// Fused shifted power step on tcgen05 tensor cores, bfloat16 tensor:
//   Y_part = X_(k) (X_(k)^T Q)      (Algorithm 2/3 inner loop; the shift
//                                    -alpha Q is applied by the reduction)
// for a mode-major view (P == 1): X_(k) is n x cols, column j contiguous.
//
// One HBM read of X per step.  A CTA owns a 32-wide part of the l columns
// of Q (c-part) and streams column slabs of 64 columns:
//   GEMM1  D1[j, c] = sum_i X[i, j] Q[i, c]      (M = 64 slab columns,
//          N = 32, K = n; A = the TMA tile read K-major, B = Q^T resident)
//   epilogue: D1 (TMEM) -> W^T = W_hi^T + W_lo^T as two bfloat16 tiles in shared memory
//   GEMM2  Y[i, c] += sum_j X[i, j] W[j, c]      (M = 128 rows per tile,
//          N = 32, K = 64; A = the same TMA tile read MN-major)
// Y stays in TMEM (ceil(n/128) tiles x 32 columns) for the whole launch and
// is written once as a per-CTA FP32 partial.  CTAs of different c-parts
// process the same slabs in the same order, so the second read of a slab is
// served by L2.
//
// Roles: warp 0 issues TMA, warp 1 issues MMAs (one thread) and owns TMEM,
// warps 2-5 run the epilogue.  Every wait is bounded by a time limit; on
// expiry the CTA records TK_ETIMEOUT, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "tk_common.cuh"
#include "tk_internal.h"
#include "tk_tc.cuh"

namespace tk {

namespace tc {

constexpr int NC = 32;          // Q columns per CTA (c-part width)
constexpr int BJ = 64;          // slab width (columns of X_(k))
constexpr int CHUNK_I = 64;     // rows of one TMA box (128 bytes of bf16)
constexpr int SUP_BYTES = 2 * CHUNK_I * BJ * 2;   // 128 rows x 64 cols bf16 = 16 KB
constexpr int QT_CHUNK_BYTES = NC * 128;           // 32 rows x 64 i bf16 = 4 KB
constexpr int W_BYTES = NC * 128;                  // 32 rows (c) x 64 j bf16 = 4 KB
constexpr int THREADS = 192;

struct Params {
  int n;           // rows of X_(k)
  int nt;          // 128-row tiles (superchunks) per slab
  long long cols;  // columns of X_(k)
  int nslabs;      // ceil(cols / BJ)
  int cparts;      // c-parts (l_pad / NC)
  int ring;        // superchunk slots
  int l_pad;       // row stride of the partial output
  uint32_t tmem_cols;
};

struct __align__(8) Bars {
  uint64_t full[16];
  uint64_t empty[16];
  uint64_t qfull;
  uint64_t d1_full[2];
  uint64_t d1_empty[2];
  uint64_t w_full[2];
  uint64_t w_empty[2];
  uint64_t y_done;
  uint64_t drain;
};

__global__ void __launch_bounds__(THREADS, 1)
k_power_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
           Params pr, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int nq = pr.nt * 2;                       // Q^T chunks of 64 rows
  unsigned char* sQ = sm;                         // nq x 4 KB
  unsigned char* sRing = sQ + nq * QT_CHUNK_BYTES;   // ring x 16 KB
  unsigned char* sW = sRing + pr.ring * SUP_BYTES;   // W_hi^T: 2 x 4 KB, then W_lo^T: 2 x 4 KB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpart = blockIdx.x % pr.cparts;
  const int group = blockIdx.x / pr.cparts;
  const int ngroups = gridDim.x / pr.cparts;
  // slabs of this CTA: group, group + ngroups, ...
  const int my_slabs = group < pr.nslabs ? (pr.nslabs - 1 - group) / ngroups + 1 : 0;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < pr.ring; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    mbar_init(smem_u32(&bars.qfull), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars.d1_full[b]), 1);
      mbar_init(smem_u32(&bars.d1_empty[b]), 4);
      mbar_init(smem_u32(&bars.w_full[b]), 4);
      mbar_init(smem_u32(&bars.w_empty[b]), 1);
    }
    mbar_init(smem_u32(&bars.y_done), 1);
    mbar_init(smem_u32(&bars.drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(pr.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t d1col0 = (uint32_t)(pr.nt * NC);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && my_slabs > 0) {
      asm volatile("prefetch.tensormap [%0];" :: "l"((uint64_t)&tmX) : "memory");
      const uint32_t qb = smem_u32(&bars.qfull);
      mbar_expect_tx(qb, (uint32_t)(nq * QT_CHUNK_BYTES));
      for (int ch = 0; ch < nq; ++ch)
        tma_load_2d(smem_u32(sQ + ch * QT_CHUNK_BYTES), &tmQ, ch * CHUNK_I, cpart * NC, qb);
      long long issued = 0;
      int slot = 0;
      uint32_t use = 0;
      for (int k = 0; k < my_slabs && !abort_flag; ++k) {
        const int slab = group + k * ngroups;
        for (int t = 0; t < pr.nt; ++t, ++issued) {
          if (t > 0 || k > 0) {
            if (++slot == pr.ring) { slot = 0; ++use; }
          }
          if (!mbar_wait(smem_u32(&bars.empty[slot]), (use & 1) ^ 1, &abort_flag)) break;
          const uint32_t fb = smem_u32(&bars.full[slot]);
          mbar_expect_tx(fb, SUP_BYTES);
          const uint32_t dst = smem_u32(sRing + slot * SUP_BYTES);
          tma_load_2d(dst, &tmX, t * 128, slab * BJ, fb);
          tma_load_2d(dst + SUP_BYTES / 2, &tmX, t * 128 + CHUNK_I, slab * BJ, fb);
        }
        if (abort_flag) break;
      }
      // drain: every issued copy must have landed before the CTA exits
      const long long first = issued > pr.ring ? issued - pr.ring : 0;
      for (long long u = first; u < issued; ++u) {
        const int slot = (int)(u % pr.ring);
        const uint32_t use = (uint32_t)(u / pr.ring);
        const uint64_t t0 = now_ns();
        while (!mbar_try(smem_u32(&bars.full[slot]), use & 1) && now_ns() - t0 < WAIT_NS) {
        }
      }
      const uint64_t t0 = now_ns();
      while (!mbar_try(qb, 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && my_slabs > 0) {
      const uint32_t ID1 = idesc_bf16(64, NC, 0, 0);
      const uint32_t ID2 = idesc_bf16(128, NC, 1, 0);
      bool ok = mbar_wait(smem_u32(&bars.qfull), 0, &abort_flag);
      fence_after();
      int slot = -1;
      uint32_t use = 0;
      const uint64_t dring1 = desc_sw128(smem_u32(sRing), 16, 1024);
      const uint64_t dring2 = desc_sw128(smem_u32(sRing), SUP_BYTES / 2, 1024);
      const uint64_t dq = desc_sw128(smem_u32(sQ), 16, 1024);
      int slots[16];
      for (int k = 0; k < my_slabs && ok; ++k) {
        const int b = k & 1;
        const uint32_t v = (uint32_t)(k >> 1);
        const uint32_t d1 = tmem + d1col0 + (uint32_t)(b * NC);
        if (!mbar_wait(smem_u32(&bars.d1_empty[b]), (v & 1) ^ 1, &abort_flag)) { ok = false; break; }
        fence_after();
        // GEMM1: D1 = X_slab^T Q_part  (K over the n rows)
        for (int t = 0; t < pr.nt; ++t) {
          if (++slot == pr.ring) { slot = 0; ++use; }
          slots[t] = slot;
          if (!mbar_wait(smem_u32(&bars.full[slot]), use & 1, &abort_flag)) { ok = false; break; }
          fence_after();
          const uint64_t da0 = desc_off(dring1, (uint32_t)slot * SUP_BYTES);
          const uint64_t db0 = desc_off(dq, (uint32_t)(2 * t) * QT_CHUNK_BYTES);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(d1, desc_off(da0, h * (SUP_BYTES / 2) + kk * 32),
                       desc_off(db0, h * QT_CHUNK_BYTES + kk * 32), ID1, (t | h | kk) != 0);
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars.d1_full[b]));
        // GEMM2: Y_tile(t) += X_tile(t) W   (K over the 64 slab columns)
        if (!mbar_wait(smem_u32(&bars.w_full[b]), v & 1, &abort_flag)) { ok = false; break; }
        fence_after();
        const uint64_t dwh = desc_sw128(smem_u32(sW + b * W_BYTES), 16, 1024);
        const uint64_t dwl = desc_sw128(smem_u32(sW + (2 + b) * W_BYTES), 16, 1024);
        for (int t = 0; t < pr.nt; ++t) {
          const uint64_t da0 = desc_off(dring2, (uint32_t)slots[t] * SUP_BYTES);
          const uint32_t yt = tmem + (uint32_t)(t * NC);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // W = W_hi + W_lo (bfloat16 pair, ~16 bits): Y += X W_hi + X W_lo
            mma_bf16(yt, desc_off(da0, kk * 2048), desc_off(dwh, kk * 32), ID2, (k | kk) != 0);
            mma_bf16(yt, desc_off(da0, kk * 2048), desc_off(dwl, kk * 32), ID2, 1);
          }
          mma_commit(smem_u32(&bars.empty[slots[t]]));
        }
        mma_commit(smem_u32(&bars.w_empty[b]));
      }
      mma_commit(smem_u32(&bars.y_done));
      // drain: all MMAs issued by this thread complete before TMEM is freed
      mma_commit(smem_u32(&bars.drain));
      const uint64_t t0 = now_ns();
      while (!mbar_try(smem_u32(&bars.drain), 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---------------- epilogue warps 2..5 ----------------
    const int q = warp & 3;                     // TMEM lane quarter of this warp
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    bool ok = true;
    for (int k = 0; k < my_slabs && ok; ++k) {
      const int b = k & 1;
      const uint32_t v = (uint32_t)(k >> 1);
      if (!mbar_wait(smem_u32(&bars.d1_full[b]), v & 1, &abort_flag)) { ok = false; break; }
      fence_after();
      uint32_t r[32];
      tmem_ld32(tmem + lane_off + d1col0 + (uint32_t)(b * NC), r);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.d1_empty[b]));
      if (!mbar_wait(smem_u32(&bars.w_empty[b]), (v & 1) ^ 1, &abort_flag)) { ok = false; break; }
      // M = 64 accumulator: lanes 0..15 of quarter q hold slab columns j = 16 q + lane
      if (lane < 16) {
        const int j = 16 * q + lane;
        unsigned char* wb = sW + b * W_BYTES;
        unsigned char* wl = sW + (2 + b) * W_BYTES;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int off = c * 128 + ((((2 * j) >> 4) ^ (c & 7)) << 4) + ((2 * j) & 15);
          const float w = __uint_as_float(r[c]);
          const __nv_bfloat16 h = __float2bfloat16_rn(w);
          *reinterpret_cast<__nv_bfloat16*>(wb + off) = h;
          *reinterpret_cast<__nv_bfloat16*>(wl + off) =
              __float2bfloat16_rn(__fsub_rn(w, __bfloat162float(h)));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.w_full[b]));
    }
    // write this CTA's Y partial: rows 128 t + 32 q + lane, columns of this c-part
    const bool have = my_slabs > 0 && ok && mbar_wait(smem_u32(&bars.y_done), 0, &abort_flag);
    if (have) fence_after();
    for (int t = 0; t < pr.nt; ++t) {
      uint32_t r[32];
      if (have) tmem_ld32(tmem + lane_off + (uint32_t)(t * NC), r);
      const int i = t * 128 + q * 32 + lane;
      if (i < pr.n) {
        float* dst = part + ((long long)group * pr.n + i) * pr.l_pad + cpart * NC;
#pragma unroll
        for (int c = 0; c < NC; c += 4) {
          float4 v4;
          v4.x = have ? __uint_as_float(r[c]) : 0.f;
          v4.y = have ? __uint_as_float(r[c + 1]) : 0.f;
          v4.z = have ? __uint_as_float(r[c + 2]) : 0.f;
          v4.w = have ? __uint_as_float(r[c + 3]) : 0.f;
          *reinterpret_cast<float4*>(dst + c) = v4;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) atomicExch(err, (int)TK_ETIMEOUT);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(pr.tmem_cols) : "memory");
  }
}

// Q (n x l, FP64, column-major) -> Q^T (l_pad x n_pad) bfloat16, zero padded.
__global__ void k_qt_bf16(const double* __restrict__ Q, int n, int l, int n_pad, int l_pad,
                          __nv_bfloat16* __restrict__ qt) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_pad * l_pad) return;
  const int i = (int)(idx % n_pad), c = (int)(idx / n_pad);
  const float v = (i < n && c < l) ? (float)Q[i + (long long)n * c] : 0.f;
  qt[idx] = __float2bfloat16_rn(v);
}

// ===========================================================================
// Cluster variant: a pair of CTAs (one cluster) shares each slab.  CTA rank r
// owns rows [r*half, (r+1)*half) of X_(k) and of Q (all 64 columns of Q), so
// every byte of X is read from HBM exactly once and each CTA holds a
// double-buffered half slab:
//   GEMM1  D1_r[j, c] = sum_{i in half r} X[i, j] Q[i, c]   (M = 64, N = 64)
//   the two partials are exchanged through distributed shared memory and
//   summed (own + peer, the same order in both CTAs: identical W), then
//   rounded to bfloat16 into one of two W buffers;
//   GEMM2  Y[i, c] += sum_j X[i, j] W[j, c] for the CTA's rows (M = 128).
// With two W buffers the epilogue prepares W for slab k + 1 while GEMM2 of
// slab k still reads W for slab k.
// GEMM1 and GEMM2 are issued from two different warps, so waiting for the
// next slab's data never delays the current slab's GEMM2.
// Roles: warp 0 TMA, warp 1 GEMM1 issuer + TMEM owner, warp 2 GEMM2 issuer,
// warps 3..6 epilogue (exchange, W, Y write-back).
// ===========================================================================
constexpr int NC2 = 64;
constexpr int THREADS2 = 224;
constexpr int XBUF_BYTES = BJ * NC2 * 4;        // 64 x 64 FP32 partial = 16 KB
constexpr int W2_BYTES = BJ * 128;              // 64 rows (j) x 64 c bf16 = 8 KB per buffer
constexpr int QT2_CHUNK_BYTES = NC2 * 128;      // 64 rows (c) x 64 i bf16 = 8 KB

// (a, b) -> bfloat16 roundings (a in the low half), packed in one word.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

struct Params2 {
  int n;           // rows of X_(k)
  int half;        // rows per CTA (multiple of 128)
  int nth;         // 128-row tiles per CTA
  long long cols;
  int nslabs;
  int l_pad;       // row stride of the partial output (64)
  uint32_t tmem_cols;
};

struct __align__(8) Bars2 {
  uint64_t full[12];
  uint64_t empty[12];
  uint64_t qfull;
  uint64_t d1_full[2];
  uint64_t d1_empty[2];
  uint64_t w_full[2];
  uint64_t w_empty[2];
  uint64_t xfull;       // peer's partial has landed in my exchange buffer
  uint64_t peer_free;   // the peer has consumed its exchange buffer
  uint64_t y_done;
  uint64_t drain1, drain2;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS2, 1)
k_power_tc2(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
            Params2 pr, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ Bars2 bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int nq = pr.nth * 2;                           // Q^T chunks of 64 rows
  const int ring = 2 * pr.nth;                         // two half-slab buffers
  unsigned char* sQ = sm;                              // nq x 8 KB
  unsigned char* sRing = sQ + nq * QT2_CHUNK_BYTES;    // ring x 16 KB
  unsigned char* sW = sRing + ring * SUP_BYTES;        // W: 2 x 8 KB
  float* sX = reinterpret_cast<float*>(sW + 2 * W2_BYTES);  // 16 KB exchange buffer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  const int cid = blockIdx.x >> 1;
  const int nclusters = gridDim.x >> 1;
  const int my_slabs = cid < pr.nslabs ? (pr.nslabs - 1 - cid) / nclusters + 1 : 0;
  const int row0 = (int)rank * pr.half;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < ring; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    mbar_init(smem_u32(&bars.qfull), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars.d1_full[b]), 1);
      mbar_init(smem_u32(&bars.d1_empty[b]), 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars.w_full[b]), 4);
      mbar_init(smem_u32(&bars.w_empty[b]), 1);
    }
    // xfull: one local arrival per phase carrying the expected 16 KB that the
    // peer's asynchronous stores complete
    mbar_init(smem_u32(&bars.xfull), 1);
    mbar_init(smem_u32(&bars.peer_free), 4);
    if (my_slabs > 0) mbar_expect_tx(smem_u32(&bars.xfull), (uint32_t)XBUF_BYTES);
    mbar_init(smem_u32(&bars.y_done), 1);
    mbar_init(smem_u32(&bars.drain1), 1);
    mbar_init(smem_u32(&bars.drain2), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(pr.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  cluster_sync();              // barriers of both CTAs initialised before any remote arrive
  fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t d1col0 = (uint32_t)(pr.nth * NC2);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && my_slabs > 0) {
      const uint32_t qb = smem_u32(&bars.qfull);
      mbar_expect_tx(qb, (uint32_t)(nq * QT2_CHUNK_BYTES));
      for (int ch = 0; ch < nq; ++ch)
        tma_load_2d(smem_u32(sQ + ch * QT2_CHUNK_BYTES), &tmQ, row0 + ch * CHUNK_I, 0, qb);
      // slab k uses slots (k & 1) nth .. (k & 1) nth + nth - 1 (ring == 2 nth),
      // the (k >> 1)-th time each
      long long issued = 0;
      for (int k = 0; k < my_slabs && !abort_flag; ++k) {
        const int slab = cid + k * nclusters;
        const uint32_t use = (uint32_t)(k >> 1);
        for (int t = 0; t < pr.nth; ++t, ++issued) {
          const int slot = (k & 1) * pr.nth + t;
          if (!mbar_wait(smem_u32(&bars.empty[slot]), (use & 1) ^ 1, &abort_flag)) break;
          const uint32_t fb = smem_u32(&bars.full[slot]);
          mbar_expect_tx(fb, SUP_BYTES);
          const uint32_t dst = smem_u32(sRing + slot * SUP_BYTES);
          tma_load_2d(dst, &tmX, row0 + t * 128, slab * BJ, fb);
          tma_load_2d(dst + SUP_BYTES / 2, &tmX, row0 + t * 128 + CHUNK_I, slab * BJ, fb);
        }
        if (abort_flag) break;
      }
      const long long first = issued > ring ? issued - ring : 0;
      for (long long u = first; u < issued; ++u) {
        const int kk = (int)(u / pr.nth);
        const int slot = (kk & 1) * pr.nth + (int)(u - (long long)kk * pr.nth);
        const uint32_t use = (uint32_t)(kk >> 1);
        const uint64_t t0 = now_ns();
        while (!mbar_try(smem_u32(&bars.full[slot]), use & 1) && now_ns() - t0 < WAIT_NS) {
        }
      }
      const uint64_t t0 = now_ns();
      while (!mbar_try(qb, 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else if (warp == 1) {
    // ---------------- GEMM1 issuer: D1 = X_half^T Q_half ----------------
    if (lane == 0 && my_slabs > 0) {
      const uint32_t ID1 = idesc_bf16(64, NC2, 0, 0);
      bool ok = mbar_wait(smem_u32(&bars.qfull), 0, &abort_flag);
      fence_after();
      // descriptors of the first ring slot and of Q^T; the others are at
      // constant offsets (one add each: the issue loop stays short)
      const uint64_t dring = desc_sw128(smem_u32(sRing), 16, 1024);
      const uint64_t dq = desc_sw128(smem_u32(sQ), 16, 1024);
      for (int k = 0; k < my_slabs && ok; ++k) {
        const int b = k & 1;
        const uint32_t v = (uint32_t)(k >> 1);
        const uint32_t d1 = tmem + d1col0 + (uint32_t)(b * NC2);
        if (!mbar_wait(smem_u32(&bars.d1_empty[b]), (v & 1) ^ 1, &abort_flag)) { ok = false; break; }
        fence_after();
        for (int t = 0; t < pr.nth; ++t) {
          const int slot = b * pr.nth + t;
          if (!mbar_wait(smem_u32(&bars.full[slot]), v & 1, &abort_flag)) { ok = false; break; }
          fence_after();
          const uint64_t da0 = desc_off(dring, (uint32_t)slot * SUP_BYTES);
          const uint64_t db0 = desc_off(dq, (uint32_t)(2 * t) * QT2_CHUNK_BYTES);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(d1, desc_off(da0, h * (SUP_BYTES / 2) + kk * 32),
                       desc_off(db0, h * QT2_CHUNK_BYTES + kk * 32), ID1, (t | h | kk) != 0);
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars.d1_full[b]));
      }
      mma_commit(smem_u32(&bars.drain1));
      const uint64_t t0 = now_ns();
      while (!mbar_try(smem_u32(&bars.drain1), 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else if (warp == 2) {
    // ---------------- GEMM2 issuer: Y_tile += X_tile W ----------------
    if (lane == 0 && my_slabs > 0) {
      const uint32_t ID2 = idesc_bf16(128, NC2, 1, 1);
      const uint64_t dring = desc_sw128(smem_u32(sRing), SUP_BYTES / 2, 1024);
      const uint64_t dw = desc_sw128(smem_u32(sW), 1024, 1024);
      bool ok = true;
      for (int k = 0; k < my_slabs && ok; ++k) {
        const int b = k & 1;
        if (!mbar_wait(smem_u32(&bars.w_full[b]), (uint32_t)(k >> 1) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint64_t dwb = desc_off(dw, (uint32_t)b * W2_BYTES);
        for (int t = 0; t < pr.nth; ++t) {
          const int slot = b * pr.nth + t;
          const uint64_t da0 = desc_off(dring, (uint32_t)slot * SUP_BYTES);
          const uint32_t yt = tmem + (uint32_t)(t * NC2);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(yt, desc_off(da0, kk * 2048), desc_off(dwb, kk * 2048), ID2, (k | kk) != 0);
          mma_commit(smem_u32(&bars.empty[slot]));
        }
        mma_commit(smem_u32(&bars.w_empty[b]));
      }
      mma_commit(smem_u32(&bars.y_done));
      mma_commit(smem_u32(&bars.drain2));
      const uint64_t t0 = now_ns();
      while (!mbar_try(smem_u32(&bars.drain2), 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---------------- epilogue warps 3..6 ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int j = 16 * q + (lane & 15);                 // D1 row of this lane (lane < 16)
    const uint32_t xrow_peer = mapa(smem_u32(sX + j * NC2), peer);
    const uint32_t peer_xfull = mapa(smem_u32(&bars.xfull), peer);
    const uint32_t peer_free = mapa(smem_u32(&bars.peer_free), peer);
    bool ok = true;
    for (int k = 0; k < my_slabs && ok; ++k) {
      const int b = k & 1;
      const uint32_t v = (uint32_t)(k >> 1);
      if (!mbar_wait(smem_u32(&bars.d1_full[b]), v & 1, &abort_flag)) { ok = false; break; }
      fence_after();
      uint32_t r0[32], r1[32];
      tmem_ld32(tmem + lane_off + d1col0 + (uint32_t)(b * NC2), r0);
      tmem_ld32(tmem + lane_off + d1col0 + (uint32_t)(b * NC2) + 32, r1);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.d1_empty[b]));
      // send my partial row j to the peer once its exchange buffer is free
      if (!mbar_wait_cluster(smem_u32(&bars.peer_free), (k & 1) ^ 1, &abort_flag)) {
        ok = false;
        break;
      }
      // chunk ch (four floats) of row j sits at chunk ch ^ (j & 15) of the row
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 32; c += 4)
          st_async_v4(xrow_peer + (((c >> 2) ^ (j & 15)) << 4), r0[c], r0[c + 1], r0[c + 2],
                      r0[c + 3], peer_xfull);
#pragma unroll
        for (int c = 0; c < 32; c += 4)
          st_async_v4(xrow_peer + (((8 + (c >> 2)) ^ (j & 15)) << 4), r1[c], r1[c + 1], r1[c + 2],
                      r1[c + 3], peer_xfull);
      }
      // the peer's partial for my rows (its 16 KB completes my xfull phase)
      if (!mbar_wait_cluster(smem_u32(&bars.xfull), k & 1, &abort_flag)) { ok = false; break; }
      // own partial + peer's, in the same order in both CTAs (identical W)
      if (lane < 16) {
        const float* px = sX + j * NC2;
#pragma unroll
        for (int ch = 0; ch < 16; ++ch) {
          uint32_t* rr = ch < 8 ? r0 : r1;
          const int c0 = (ch & 7) * 4;
          const float4 pa = *reinterpret_cast<const float4*>(px + ((ch ^ (j & 15)) << 2));
          rr[c0] = __float_as_uint(__uint_as_float(rr[c0]) + pa.x);
          rr[c0 + 1] = __float_as_uint(__uint_as_float(rr[c0 + 1]) + pa.y);
          rr[c0 + 2] = __float_as_uint(__uint_as_float(rr[c0 + 2]) + pa.z);
          rr[c0 + 3] = __float_as_uint(__uint_as_float(rr[c0 + 3]) + pa.w);
        }
      }
      __syncwarp();
      if (lane == 0) {
        // re-arm xfull for the next slab before the peer may send it
        if (q == 0 && k + 1 < my_slabs) mbar_expect_tx(smem_u32(&bars.xfull), (uint32_t)XBUF_BYTES);
        mbar_arrive_remote(peer_free);      // my exchange buffer may be refilled
      }
      // W of this slab into buffer b once GEMM2 of slab k - 2 has read it
      if (!mbar_wait(smem_u32(&bars.w_empty[b]), (v & 1) ^ 1, &abort_flag)) { ok = false; break; }
      if (lane < 16) {
        unsigned char* wrow = sW + b * W2_BYTES + j * 128;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          uint32_t* rr = ch < 4 ? r0 : r1;
          const int c0 = (ch & 3) * 8;
          uint4 w4;
          w4.x = bf16x2_bits(__uint_as_float(rr[c0]), __uint_as_float(rr[c0 + 1]));
          w4.y = bf16x2_bits(__uint_as_float(rr[c0 + 2]), __uint_as_float(rr[c0 + 3]));
          w4.z = bf16x2_bits(__uint_as_float(rr[c0 + 4]), __uint_as_float(rr[c0 + 5]));
          w4.w = bf16x2_bits(__uint_as_float(rr[c0 + 6]), __uint_as_float(rr[c0 + 7]));
          *reinterpret_cast<uint4*>(wrow + ((ch ^ (j & 7)) << 4)) = w4;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.w_full[b]));
    }
    // write this CTA's rows of the Y partial
    const bool have = my_slabs > 0 && ok && mbar_wait(smem_u32(&bars.y_done), 0, &abort_flag);
    if (have) fence_after();
    for (int t = 0; t < pr.nth; ++t) {
      uint32_t y0[32], y1[32];
      if (have) {
        tmem_ld32(tmem + lane_off + (uint32_t)(t * NC2), y0);
        tmem_ld32(tmem + lane_off + (uint32_t)(t * NC2) + 32, y1);
      }
      const int i = row0 + t * 128 + q * 32 + lane;
      if (i < pr.n) {
        float* dst = part + ((long long)cid * pr.n + i) * pr.l_pad;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          float4 a4, b4;
          a4.x = have ? __uint_as_float(y0[c]) : 0.f;
          a4.y = have ? __uint_as_float(y0[c + 1]) : 0.f;
          a4.z = have ? __uint_as_float(y0[c + 2]) : 0.f;
          a4.w = have ? __uint_as_float(y0[c + 3]) : 0.f;
          b4.x = have ? __uint_as_float(y1[c]) : 0.f;
          b4.y = have ? __uint_as_float(y1[c + 1]) : 0.f;
          b4.z = have ? __uint_as_float(y1[c + 2]) : 0.f;
          b4.w = have ? __uint_as_float(y1[c + 3]) : 0.f;
          *reinterpret_cast<float4*>(dst + c) = a4;
          *reinterpret_cast<float4*>(dst + 32 + c) = b4;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  cluster_sync();              // no CTA leaves while its peer may still touch its memory
  if (abort_flag && threadIdx.x == 0) atomicExch(err, (int)TK_ETIMEOUT);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(pr.tmem_cols) : "memory");
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
                 uint32_t box_inner, uint32_t box_outer) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct TcShape {
  int nt, nq, l_pad, cparts, ring;
  uint32_t tmem_cols;
  size_t smem;
};

bool tc_shape(int64_t n, int l, TcShape* s) {
  if (n < 8 || (n % 8) != 0 || l < 1 || l > TK_MAX_L) return false;
  s->nt = (int)((n + 127) / 128);
  if (s->nt > 16) return false;                 // MMA thread keeps 16 slot ids
  s->nq = 2 * s->nt;
  s->l_pad = (l + tc::NC - 1) / tc::NC * tc::NC;
  s->cparts = s->l_pad / tc::NC;
  const uint32_t need = (uint32_t)(s->nt * tc::NC + 2 * tc::NC);
  uint32_t cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512) return false;
  s->tmem_cols = cols;
  const size_t fixed = (size_t)s->nq * tc::QT_CHUNK_BYTES + 4 * tc::W_BYTES + 1024;
  const size_t budget = 227 * 1024 - 2048;   // static smem (barriers) kept aside
  if (fixed + (size_t)(s->nt + 1) * tc::SUP_BYTES > budget) return false;
  int ring = (int)((budget - fixed) / tc::SUP_BYTES);
  ring = std::min(ring, 16);
  ring = std::min(ring, 2 * s->nt + 2);
  s->ring = ring;
  s->smem = fixed + (size_t)ring * tc::SUP_BYTES;
  return true;
}


// Cluster variant shape (n in [512, 1024], l <= 64).
struct Tc2Shape {
  int nth, half, nq, ring, nt;
  uint32_t tmem_cols;
  size_t smem;
};

bool tc2_shape(int64_t n, int l, Tc2Shape* s) {
  if (n < 512 || n > 1024 || (n % 8) != 0 || l < 1 || l > tc::NC2) return false;
  s->nt = (int)((n + 127) / 128);
  s->nth = (s->nt + 1) / 2;
  s->half = s->nth * 128;
  s->nq = 2 * s->nth;
  s->ring = 2 * s->nth;
  const uint32_t need = (uint32_t)(s->nth * tc::NC2 + 2 * tc::NC2);
  uint32_t cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512 || s->ring > 12) return false;
  s->tmem_cols = cols;
  s->smem = (size_t)s->nq * tc::QT2_CHUNK_BYTES + (size_t)s->ring * tc::SUP_BYTES +
            2 * tc::W2_BYTES + tc::XBUF_BYTES + 1024;   // two W buffers
  return s->smem <= 227 * 1024 - 2048;
}

bool use_cluster(View v, int l) {
  Tc2Shape s2;
  return tc2_shape(v.n, l, &s2);
}

}  // namespace

bool power_tc_supported(View v, int l, const void* X) {
  TcShape s;
  return v.P == 1 && tc_shape(v.n, l, &s) && (((uintptr_t)X) & 15) == 0 &&
         v.cols() < (1LL << 31) && get_encode() != nullptr;
}

int power_tc_lpad(View v, int l) {
  return use_cluster(v, l) ? tc::NC2 : (l + tc::NC - 1) / tc::NC * tc::NC;
}

int power_tc_groups(View v, int l) {
  const long long nslabs = (v.cols() + tc::BJ - 1) / tc::BJ;
  if (use_cluster(v, l)) {
    long long cl = num_sms() / 2;
    return (int)std::max(1LL, std::min(cl, nslabs));
  }
  TcShape s;
  if (!tc_shape(v.n, l, &s)) return 0;
  const int per_sm = (int)(512 / s.tmem_cols);
  long long groups = (long long)num_sms() * per_sm / s.cparts;
  groups = std::max(1LL, std::min(groups, nslabs));
  return (int)groups;
}

size_t power_tc_scratch(View v, int l) {
  TcShape s;
  if (!tc_shape(v.n, l, &s)) return 0;
  return (size_t)s.nt * 128 * std::max(s.l_pad, tc::NC2) * sizeof(__nv_bfloat16) + 256;
}

cudaError_t launch_power_tc(const void* X, View v, const double* Q, int l, void* scratch,
                            float* part, int groups, int* err, cudaStream_t st) {
  TcShape s;
  if (!tc_shape(v.n, l, &s)) return cudaErrorInvalidValue;
  const int n_pad = s.nt * 128;
  const bool cluster = use_cluster(v, l);
  const int l_pad = cluster ? tc::NC2 : s.l_pad;
  __nv_bfloat16* qt = (__nv_bfloat16*)scratch;
  {
    const long long tot = (long long)n_pad * l_pad;
    count_kernels(1);
    tc::k_qt_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Q, (int)v.n, l, n_pad, l_pad,
                                                                  qt);
  }
  CUtensorMap mx, mq;
  if (!make_map_2d(&mx, X, (uint64_t)v.n, (uint64_t)v.cols(), 64, tc::BJ)) return cudaErrorUnknown;
  if (cluster) {
    Tc2Shape s2;
    tc2_shape(v.n, l, &s2);
    if (!make_map_2d(&mq, qt, (uint64_t)n_pad, (uint64_t)l_pad, 64, tc::NC2))
      return cudaErrorUnknown;
    tc::Params2 pr;
    pr.n = (int)v.n;
    pr.half = s2.half;
    pr.nth = s2.nth;
    pr.cols = v.cols();
    pr.nslabs = (int)((v.cols() + tc::BJ - 1) / tc::BJ);
    pr.l_pad = l_pad;
    pr.tmem_cols = s2.tmem_cols;
    static bool attr2 = false;
    if (!attr2) {
      cudaFuncSetAttribute(tc::k_power_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024 - 2048);
      attr2 = true;
    }
    // one CTA per SM: the shared-memory request keeps a second one away
    const size_t smem = std::max(s2.smem, (size_t)120 * 1024);
    count_kernels(1);
    tc::k_power_tc2<<<2 * groups, tc::THREADS2, smem, st>>>(mx, mq, pr, part, err);
    return cudaGetLastError();
  }
  if (!make_map_2d(&mq, qt, (uint64_t)n_pad, (uint64_t)s.l_pad, 64, tc::NC))
    return cudaErrorUnknown;
  tc::Params pr;
  pr.n = (int)v.n;
  pr.nt = s.nt;
  pr.cols = v.cols();
  pr.nslabs = (int)((v.cols() + tc::BJ - 1) / tc::BJ);
  pr.cparts = s.cparts;
  pr.ring = s.ring;
  pr.l_pad = s.l_pad;
  pr.tmem_cols = s.tmem_cols;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_power_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024 - 2048);
    attr = true;
  }
  // occupancy: at most 512 / tmem_cols CTAs per SM (TMEM), enforced through
  // the shared-memory request
  const int per_sm = (int)(512 / s.tmem_cols);
  size_t smem = s.smem;
  if (per_sm == 1) smem = std::max(smem, (size_t)120 * 1024);
  else if (per_sm == 2) smem = std::max(smem, (size_t)80 * 1024);
  else smem = std::max(smem, (size_t)(230 * 1024 / (per_sm + 1)));
  count_kernels(1);
  tc::k_power_tc<<<groups * s.cparts, tc::THREADS, smem, st>>>(mx, mq, pr, part, err);
  return cudaGetLastError();
}

}  // namespace tk
