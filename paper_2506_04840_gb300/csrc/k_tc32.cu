// tcgen05 kind::tf32 building blocks for the FP32 contractions.
//
// tucker_debug_tf32_mma: one 128 x 64 x 32 product D = A B on the tensor
// cores (four K = 8 instructions accumulating in TMEM), with A taken from
// shared memory (K-major) or from tensor memory.  A test entry point: it
// fixes, on the GPU itself, how the kind::tf32 instruction treats FP32
// operand bits below TF32 precision (they are dropped: truncation) and how
// its FP32 accumulator rounds (toward zero, within and between
// instructions), which the 3xTF32 split of the FP32 kernels and the
// accumulation-length choices depend on.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "tk_common.cuh"
#include "tk_internal.h"
#include "tk_batch.h"
#include "tk_plan.h"
#include "tk_tc.cuh"

namespace tk {
namespace tc {

// element (r, k) of a K-major tile with 128-byte swizzle: rows of 32 FP32 K
// values (128 B), 8-row atoms of 1 KB
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k * 4) >> 4) ^ (r & 7)) << 4) +
                    ((k * 4) & 15));
}
__global__ void __launch_bounds__(128, 1)
k_tf32_probe(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ D,
             int mode, int* __restrict__ err) {
  __shared__ __align__(1024) unsigned char sA[16384];
  __shared__ __align__(1024) unsigned char sB[8192];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(128u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // stage A (row tid) and B (rows n = tid / 2 halves) into shared memory
  const int m = tid;
  for (int k = 0; k < 32; ++k) {
    const float a = A[m * 32 + k];
    *reinterpret_cast<float*>(sA + kmaj_off(m, k)) = a;
  }
  for (int e = tid; e < 64 * 32; e += 128) {
    const int n = e / 32, k = e % 32;
    *reinterpret_cast<float*>(sB + kmaj_off(n, k)) = B[k * 64 + n];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  if (mode == 1) {
    uint32_t r[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) r[k] = __float_as_uint(A[m * 32 + k]);
    tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + 64u, r);
    tmem_st_wait();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (tid == 0) {
    const uint32_t id = idesc_tf32(128, 64, 0, 0);
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t db = desc_sw128(smem_u32(sB) + kk * 32, 16, 1024);
      if (mode == 1) {
        mma_tf32_ts(tmem, tmem + 64u + (uint32_t)(kk * 8), db, id, kk > 0);
      } else {
        const uint64_t da = desc_sw128(smem_u32(sA) + kk * 32, 16, 1024);
        mma_tf32_ss(tmem, da, db, id, kk > 0);
      }
    }
    mma_commit(smem_u32(&bar));
  }
  const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag);
  fence_after();
  if (ok) {
    uint32_t r0[32], r1[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), r0);
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, r1);
#pragma unroll
    for (int n = 0; n < 32; ++n) {
      D[m * 64 + n] = __uint_as_float(r0[n]);
      D[m * 64 + 32 + n] = __uint_as_float(r1[n]);
    }
  }
  fence_before();
  __syncthreads();
  if (tid == 0 && abort_flag) atomicExch(err, (int)TK_ETIMEOUT);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(128u) : "memory");
  }
}

}  // namespace tc

// ===========================================================================
// W = X^T B on tcgen05 tensor cores in 3xTF32, for a mode-major FP32 view
// (X_(k) is n x cols, column j contiguous):
//   out[j, c] = sum_i X[i, j] B[i, c],   c < m <= 64
// (the first half W = X_(k)^T Q of a shifted power step, Algorithms 2/3).
// Each FP32 operand x is split as x = x_hi + x_lo with x_hi = x with its low
// 13 mantissa bits cleared (exactly a TF32 value) and x_lo = x - x_hi (exact
// in FP32, at most 13 significant bits); the product is taken as
//   X_hi B_hi + X_hi B_lo + X_lo B_hi
// (the X_lo B_lo term is below FP32 rounding), all three on the tensor
// cores with FP32 accumulation in TMEM.  X_hi is the tile TMA brought into
// shared memory as it stands (kind::tf32 reads the upper 19 bits of each
// 32-bit operand); X_lo is formed by converter warps and placed in TMEM,
// where the third product reads its A operand.  B arrives split, as B_hi^T
// and B_lo^T planes, from a small preparation kernel.
//
// Work unit: 256 columns (two M = 128 tiles) over all n rows; a persistent
// grid strides over units.  Stage: 32 rows (K) of both tiles + the matching
// 32 rows of B_hi^T and B_lo^T, 48 KB, four stages in flight.  TMEM: two
// accumulator sets (units alternate) of 2 x 64 columns, and X_lo for every
// stage (4 x 2 x 32 columns): 512 columns.
// Roles: warp 0 TMA, warp 1 MMA issue + TMEM, warps 2-5 X_lo converters,
// warps 6-9 epilogue (TMEM -> global).  Every wait is bounded; on expiry the
// CTA records TK_ETIMEOUT, drains its copies and MMAs, frees TMEM, returns.
// ===========================================================================
namespace tc {

constexpr int X_THREADS = 320;
constexpr int X_NS = 4;                         // stages
constexpr int X_KC = 32;                        // rows per stage (128 B of FP32)
constexpr int X_TM = 2;                         // M tiles per unit
constexpr int X_ATILE = 128 * X_KC * 4;         // 16 KB
constexpr int X_BHALF = 64 * X_KC * 4;          // 8 KB
constexpr int X_STAGE = X_TM * X_ATILE + 2 * X_BHALF;   // 48 KB
constexpr uint32_t X_LO0 = 256;                 // first TMEM column of X_lo

}  // namespace tc

namespace tc {

struct __align__(8) XtbBars {
  uint64_t full[X_NS];
  uint64_t conv[X_NS];
  uint64_t empty[X_NS];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t drain;
};

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// The units of all jobs form one sequence (job j's units start at start[j];
// start == NULL: a single job); a CTA takes units blockIdx.x, + gridDim.x, ...
// Each unit's arithmetic depends on its own job only, so a problem's result is
// the same alone and in a batch.  Tensor maps in a job table (global memory)
// are acquired for the tensormap proxy before their first use.
__device__ __forceinline__ void xtb_locate(const Tc32XtbJob* jobs, const uint32_t* start,
                                           int njobs, long long u, int* jb, long long* lu) {
  if (start == nullptr) {
    *jb = 0;
    *lu = u;
    return;
  }
  const int j = batch_job(start, njobs, (uint32_t)u);
  *jb = j;
  *lu = u - (long long)__ldg(start + j);
}

__device__ __forceinline__ void xtb_body(const Tc32XtbJob* jobs, const uint32_t* start,
                                         int njobs, long long total, bool table) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ XtbBars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long my_units =
      (long long)blockIdx.x < total ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < X_NS; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.conv[s]), 4);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars.accf[b]), 1);
      mbar_init(smem_u32(&bars.acce[b]), 4);
    }
    mbar_init(smem_u32(&bars.drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(512u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && my_units > 0) {
      long long it = 0;
      int cur = -1;
      for (long long ul = 0; ul < my_units && !abort_flag; ++ul) {
        int jb;
        long long u;
        xtb_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &u);
        const Tc32XtbJob* J = jobs + jb;
        if (jb != cur) {
          cur = jb;
          if (table) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;"
                         :: "l"((uint64_t)&J->mx) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;"
                         :: "l"((uint64_t)&J->mb) : "memory");
          }
        }
        const int nk = J->nk;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = (int)(it % X_NS);
          const uint32_t use = (uint32_t)(it / X_NS);
          if (!mbar_wait(smem_u32(&bars.empty[s]), (use & 1) ^ 1, &abort_flag)) break;
          const uint32_t fb = smem_u32(&bars.full[s]);
          mbar_expect_tx(fb, (uint32_t)X_STAGE);
          const uint32_t dst = smem_u32(sm + s * X_STAGE);
#pragma unroll
          for (int t = 0; t < X_TM; ++t)
            tma_load_2d(dst + t * X_ATILE, &J->mx, kc * X_KC, (int)(u * 256 + t * 128), fb);
          tma_load_2d(dst + X_TM * X_ATILE, &J->mb, kc * X_KC, 0, fb);
          tma_load_2d(dst + X_TM * X_ATILE + X_BHALF, &J->mb, kc * X_KC, 64, fb);
        }
      }
      // every issued copy lands before the CTA exits
      const long long first = it > X_NS ? it - X_NS : 0;
      for (long long v = first; v < it; ++v) {
        const int s = (int)(v % X_NS);
        const uint32_t use = (uint32_t)(v / X_NS);
        const uint64_t t0 = now_ns();
        while (!mbar_try(smem_u32(&bars.full[s]), use & 1) && now_ns() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && my_units > 0) {
      const uint32_t ID = idesc_tf32(128, 64, 0, 0);
      // stage 0's descriptors; the others are at constant offsets
      const uint64_t dsm = desc_sw128(smem_u32(sm), 16, 1024);
      long long it = 0;
      bool ok = true;
      for (long long ul = 0; ul < my_units && ok; ++ul) {
        int jb;
        long long u;
        xtb_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &u);
        const int nk = jobs[jb].nk;
        const int b = (int)(ul & 1);
        const uint32_t v = (uint32_t)(ul >> 1);
        if (!mbar_wait(smem_u32(&bars.acce[b]), (v & 1) ^ 1, &abort_flag)) { ok = false; break; }
        fence_after();
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = (int)(it % X_NS);
          const uint32_t use = (uint32_t)(it / X_NS);
          if (!mbar_wait(smem_u32(&bars.conv[s]), use & 1, &abort_flag)) { ok = false; break; }
          fence_after();
          const uint64_t d0 = desc_off(dsm, (uint32_t)s * X_STAGE);
#pragma unroll
          for (int t = 0; t < X_TM; ++t) {
            const uint32_t d = tmem + (uint32_t)((b * X_TM + t) * 64);
            const uint32_t lo = tmem + X_LO0 + (uint32_t)((s * X_TM + t) * 32);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t da = desc_off(d0, t * X_ATILE + kk * 32);
              const uint64_t dbh = desc_off(d0, X_TM * X_ATILE + kk * 32);
              const uint64_t dbl = desc_off(d0, X_TM * X_ATILE + X_BHALF + kk * 32);
              mma_tf32_ss(d, da, dbh, ID, (kc | kk) != 0);
              mma_tf32_ss(d, da, dbl, ID, 1);
              mma_tf32_ts(d, lo + (uint32_t)(kk * 8), dbh, ID, 1);
            }
          }
          mma_commit(smem_u32(&bars.empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars.accf[b]));
      }
      // every MMA this thread issued completes before TMEM is freed
      mma_commit(smem_u32(&bars.drain));
      const uint64_t t0 = now_ns();
      while (!mbar_try(smem_u32(&bars.drain), 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else if (warp < 6) {
    // ---------------- X_lo converters (TMEM lanes = the tile's columns) ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int jj = q * 32 + lane;
    long long it = 0;
    bool ok = true;
    for (long long ul = 0; ul < my_units && ok; ++ul) {
      int jb;
      long long u;
      xtb_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &u);
      const int nk = jobs[jb].nk;
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int s = (int)(it % X_NS);
        const uint32_t use = (uint32_t)(it / X_NS);
        if (!mbar_wait(smem_u32(&bars.full[s]), use & 1, &abort_flag)) { ok = false; break; }
#pragma unroll
        for (int t = 0; t < X_TM; ++t) {
          const unsigned char* row = sm + s * X_STAGE + t * X_ATILE + jj * 128;
          uint32_t r[32];
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const float4 v4 = *reinterpret_cast<const float4*>(row + ((ch ^ (jj & 7)) << 4));
            r[4 * ch + 0] = __float_as_uint(__fsub_rn(v4.x, tf32_hi(v4.x)));
            r[4 * ch + 1] = __float_as_uint(__fsub_rn(v4.y, tf32_hi(v4.y)));
            r[4 * ch + 2] = __float_as_uint(__fsub_rn(v4.z, tf32_hi(v4.z)));
            r[4 * ch + 3] = __float_as_uint(__fsub_rn(v4.w, tf32_hi(v4.w)));
          }
          tmem_st32(tmem + lane_off + X_LO0 + (uint32_t)((s * X_TM + t) * 32), r);
        }
        tmem_st_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars.conv[s]));
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int jj = q * 32 + lane;
    for (long long ul = 0; ul < my_units; ++ul) {
      int jb;
      long long u;
      xtb_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &u);
      const Tc32XtbJob& pr = jobs[jb];
      float* __restrict__ out = pr.out;
      const int b = (int)(ul & 1);
      const uint32_t v = (uint32_t)(ul >> 1);
      if (!mbar_wait(smem_u32(&bars.accf[b]), v & 1, &abort_flag)) break;
      fence_after();
#pragma unroll 1
      for (int t = 0; t < X_TM; ++t) {
        uint32_t r0[32], r1[32];
        tmem_ld32(tmem + lane_off + (uint32_t)((b * X_TM + t) * 64), r0);
        tmem_ld32(tmem + lane_off + (uint32_t)((b * X_TM + t) * 64) + 32u, r1);
        if (t == X_TM - 1) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars.acce[b]));
        }
        const long long j = u * 256 + t * 128 + jj;
        if (j >= pr.cols) continue;
        if (pr.out_mode == 0) {
          float* o = out + (long long)pr.m * j;
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < pr.m) o[c] = __uint_as_float(c < 32 ? r0[c] : r1[c - 32]);
        } else if (pr.out_mode == 1) {
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < pr.m) out[j + pr.cols * c] = __uint_as_float(c < 32 ? r0[c] : r1[c - 32]);
        } else {
#pragma unroll
          for (int c = 0; c < 64; ++c) {
            const float w = __uint_as_float(c < 32 ? r0[c] : r1[c - 32]);
            const float h = tf32_hi(w);
            out[j + pr.ld * c] = h;
            out[j + pr.ld * (64 + c)] = __fsub_rn(w, h);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0 && my_units > 0) {
    // the problem of this CTA's first unit records the timeout
    int jb;
    long long u;
    xtb_locate(jobs, start, njobs, (long long)blockIdx.x, &jb, &u);
    atomicExch(jobs[jb].err, (int)TK_ETIMEOUT);
  }
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(512u) : "memory");
  }
}

__global__ void __launch_bounds__(X_THREADS, 1)
k_tc32_xtb(const __grid_constant__ Tc32XtbJob job) {
  xtb_body(&job, nullptr, 1, job.units, false);
}

// Work-list form (batches, the server): the jobs' units one after another.
__global__ void __launch_bounds__(X_THREADS, 1)
k_tc32_xtb_batch(const Tc32XtbJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                 int njobs, uint32_t total) {
  xtb_body(jobs, start, njobs, (long long)total, true);
}

// B (n x m, FP64, b(i, c) = B[i b_ri + c b_cm]) -> the planes B2[c][i] =
// hi(b), B2[64 + c][i] = lo(b) (FP32, 128 x n_pad, zero padded), hi = the FP32
// value of b with its low 13 mantissa bits cleared, lo = b - hi rounded to
// FP32.  Block bx of the job covers entries 256 bx ...
__device__ __forceinline__ void split_b_body(const Tc32SplitJob& J, unsigned bx) {
  const long long e = (long long)bx * 256 + threadIdx.x;
  if (e >= 64LL * J.n_pad) return;
  const int i = (int)(e % J.n_pad), c = (int)(e / J.n_pad);
  float h = 0.f, l = 0.f;
  if (i < J.n && c < J.m) {
    const double b = J.B[(int64_t)i * J.b_ri + (int64_t)c * J.b_cm];
    h = tf32_hi((float)b);
    l = (float)(b - (double)h);
  }
  J.B2[(long long)c * J.n_pad + i] = h;
  J.B2[(long long)(64 + c) * J.n_pad + i] = l;
}

__global__ void __launch_bounds__(256) k_split_b(const __grid_constant__ Tc32SplitJob job) {
  split_b_body(job, blockIdx.x);
}

__global__ void __launch_bounds__(256)
k_split_b_batch(const Tc32SplitJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    split_b_body(jobs[j], b - __ldg(start + j));
  }
}

}  // namespace tc


// ===========================================================================
// The sketch Y_part = X_(k) Omega_k on tcgen05 tensor cores in 3xTF32, for an
// FP32 mode-major view (Algorithms 2/3, first product of each mode):
//   part[g][i][c] = sum_{j in column group g} X[i, j] Omega_k(jk, c)
// with Omega_k generated in the kernel from the library's Philox
// definition, jk the column's index in the unfolding's order.  X arrives
// MN-major (rows contiguous) and kind::tf32 takes its A operand K-major only,
// so converter warps move each X tile into tensor memory as x_hi (low 13
// mantissa bits cleared) and x_lo = x - x_hi; Omega's hi/lo split goes to
// shared memory K-major.  D += X_hi W_hi + X_hi W_lo + X_lo W_hi, all three
// with A from tensor memory.  FP32 accumulation in TMEM rounds toward zero;
// the sketch only fixes the starting subspace of the power steps, and the
// column groups (a few thousand columns) are summed in FP64 afterwards.
//
// Work unit: 256 rows (two M = 128 tiles) x one column group; stage: 32
// columns (8 TMA boxes of 32 rows x 32 columns, 32 KB) + Omega hi/lo (16 KB),
// three stages.  TMEM: the unit's accumulators (2 x 64 columns) and per stage
// the two tiles' X_hi | X_lo (2 x 64 columns): 512.  Roles: warp 0 TMA, warp 1
// MMA issue + TMEM, warps 2-5 X converters (and the bfloat16 copy), warps 6-9
// Omega generation for each stage and, at the end of a unit, its partials.
// ===========================================================================
namespace tc {

constexpr int S_THREADS = 320;
constexpr int S_NS = 3;
constexpr int S_BOX = 32 * 32 * 4;                  // 4 KB: 32 rows x 32 columns
constexpr int S_ATILE = 4 * S_BOX;                  // 16 KB: 128 rows
constexpr int S_BHALF = 64 * 32 * 4;                // 8 KB
constexpr int S_STAGE = 2 * S_ATILE + 2 * S_BHALF;  // 48 KB
constexpr uint32_t S_A0 = 128;                      // first TMEM column of the A regions

__device__ __forceinline__ void sketch_locate(const Tc32SketchJob* jobs, const uint32_t* start,
                                              int njobs, long long u, int* jb, int* rb, int* g,
                                              long long* j0, int* nst) {
  int j = 0;
  long long lu = u;
  if (start != nullptr) {
    j = batch_job(start, njobs, (uint32_t)u);
    lu = u - (long long)__ldg(start + j);
  }
  const Tc32SketchJob& J = jobs[j];
  *jb = j;
  *rb = (int)(lu % J.nrb);
  *g = (int)(lu / J.nrb);
  *j0 = (long long)(*g) * J.cpg;
  const long long je = min(J.cols, *j0 + J.cpg);
  *nst = (int)((je - *j0 + 31) / 32);
}

__device__ __forceinline__ void sketch_body(const Tc32SketchJob* jobs, const uint32_t* start,
                                            int njobs, long long total, bool table) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ XtbBars bars;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long my_units =
      (long long)blockIdx.x < total ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S_NS; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.conv[s]), 8);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    mbar_init(smem_u32(&bars.accf[0]), 1);
    mbar_init(smem_u32(&bars.acce[0]), 4);
    mbar_init(smem_u32(&bars.drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(512u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer (X only) ----------------
    if (lane == 0 && my_units > 0) {
      long long it = 0;
      int cur = -1;
      for (long long ul = 0; ul < my_units && !abort_flag; ++ul) {
        int jb, rb, g, nst;
        long long j0;
        sketch_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &rb, &g,
                      &j0, &nst);
        const Tc32SketchJob* J = jobs + jb;
        if (jb != cur) {
          cur = jb;
          if (table)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;"
                         :: "l"((uint64_t)&J->mx) : "memory");
        }
        for (int ks = 0; ks < nst; ++ks, ++it) {
          const int s = (int)(it % S_NS);
          const uint32_t use = (uint32_t)(it / S_NS);
          if (!mbar_wait(smem_u32(&bars.empty[s]), (use & 1) ^ 1, &abort_flag)) break;
          const uint32_t fb = smem_u32(&bars.full[s]);
          mbar_expect_tx(fb, (uint32_t)(2 * S_ATILE));
          const uint32_t dst = smem_u32(sm + s * S_STAGE);
          const int jc = (int)(j0 + (long long)ks * 32);
#pragma unroll
          for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int bx = 0; bx < 4; ++bx)
              tma_load_2d(dst + t * S_ATILE + bx * S_BOX, &J->mx, rb * 256 + t * 128 + bx * 32,
                          jc, fb);
        }
      }
      const long long first = it > S_NS ? it - S_NS : 0;
      for (long long v = first; v < it; ++v) {
        const int s = (int)(v % S_NS);
        const uint32_t use = (uint32_t)(v / S_NS);
        const uint64_t t0 = now_ns();
        while (!mbar_try(smem_u32(&bars.full[s]), use & 1) && now_ns() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: A from TMEM, B (Omega) from shared memory ----------------
    if (lane == 0 && my_units > 0) {
      const uint32_t ID = idesc_tf32(128, 64, 0, 0);
      // stage 0's Omega descriptor; the others are at constant offsets
      const uint64_t dsm = desc_sw128(smem_u32(sm + 2 * S_ATILE), 16, 1024);
      int s = S_NS - 1;
      uint32_t use = ~0u;
      bool ok = true;
      for (long long ul = 0; ul < my_units && ok; ++ul) {
        int jb, rb, g, nst;
        long long j0;
        sketch_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &rb, &g,
                      &j0, &nst);
        if (!mbar_wait(smem_u32(&bars.acce[0]), ((uint32_t)ul & 1) ^ 1, &abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        for (int ks = 0; ks < nst; ++ks) {
          if (++s == S_NS) { s = 0; }
          if (s == 0) ++use;
          if (!mbar_wait(smem_u32(&bars.conv[s]), use & 1, &abort_flag)) { ok = false; break; }
          fence_after();
          const uint64_t d0 = desc_off(dsm, (uint32_t)s * S_STAGE);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const uint32_t d = tmem + (uint32_t)(t * 64);
            const uint32_t ah = tmem + S_A0 + (uint32_t)((s * 2 + t) * 64);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t dbh = desc_off(d0, kk * 32);
              const uint64_t dbl = desc_off(d0, S_BHALF + kk * 32);
              mma_tf32_ts(d, ah + (uint32_t)(kk * 8), dbh, ID, (ks | kk) != 0);
              mma_tf32_ts(d, ah + (uint32_t)(kk * 8), dbl, ID, 1);
              mma_tf32_ts(d, ah + 32u + (uint32_t)(kk * 8), dbh, ID, 1);
            }
          }
          mma_commit(smem_u32(&bars.empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars.accf[0]));
      }
      mma_commit(smem_u32(&bars.drain));
      const uint64_t t0 = now_ns();
      while (!mbar_try(smem_u32(&bars.drain), 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else if (warp < 6) {
    // ---------------- converters: X -> TMEM (hi | lo) and the bfloat16 copy ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    long long it = 0;
    bool ok = true;
    for (long long ul = 0; ul < my_units && ok; ++ul) {
      int jb, rb, g, nst;
      long long j0;
      sketch_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &rb, &g,
                    &j0, &nst);
      // the job's fields in registers: the copy's stores below may not be
      // assumed apart from the job table, which would reload them per store
      const Tc32SketchJob& J = jobs[jb];
      __nv_bfloat16* const shadow = J.shadow;
      const int jn = J.n, jl = J.l, jmode = J.mode;
      const uint32_t jcols = (uint32_t)J.cols, jka = (uint32_t)J.ka, jkb = (uint32_t)J.kb;
      const uint32_t jtag = J.tag;
      const uint64_t jseed = J.seed;
      for (int ks = 0; ks < nst; ++ks, ++it) {
        const int s = (int)(it % S_NS);
        const uint32_t use = (uint32_t)(it / S_NS);
        if (!mbar_wait(smem_u32(&bars.full[s]), use & 1, &abort_flag)) { ok = false; break; }
        unsigned char* st0 = sm + s * S_STAGE;
#pragma unroll 1
        for (int t = 0; t < 2; ++t) {
          // TMEM lane 32 q + lane = row 32 q + lane of tile t = row `lane` of box q
          const unsigned char* box = st0 + t * S_ATILE + q * S_BOX;
          uint32_t hi[32], lo[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = *reinterpret_cast<const float*>(
                box + j * 128 + ((((lane >> 2) ^ (j & 7))) << 4) + (lane & 3) * 4);
            const float h = tf32_hi(x);
            hi[j] = __float_as_uint(h);
            lo[j] = __float_as_uint(__fsub_rn(x, h));
          }
          const uint32_t ta = tmem + lane_off + S_A0 + (uint32_t)((s * 2 + t) * 64);
          tmem_st32(ta, hi);
          tmem_st32(ta + 32u, lo);
          if (shadow != nullptr) {
            // the precision form's bfloat16 copy of X, written as the pass reads X
            const int i = rb * 256 + t * 128 + q * 32 + lane;
            const long long jb0 = j0 + (long long)ks * 32;
            if (i < jn) {
              __nv_bfloat16* dst = shadow + jb0 * jn + i;
              const int jmax = (int)min(32LL, (long long)jcols - jb0);
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < jmax)
                  dst[(long long)j * jn] =
                      __float2bfloat16_rn(__uint_as_float(hi[j]) + __uint_as_float(lo[j]));
            }
          }
        }
        {
          // the last of Omega's four chains of this stage (groups 12..15;
          // the Omega warps take 0..11): balances the two kinds of warps
          unsigned char* bt = st0 + 2 * S_ATILE;
          const int ctid = (warp - 2) * 32 + lane;
          const int jj = lane;
          const uint32_t jg = (uint32_t)(j0 + (long long)ks * 32 + jj);
          const uint32_t jq = jg / jka;
          const uint64_t orow = (uint64_t)jq + (uint64_t)jkb * (jg - jq * jka);
          const int gq = (ctid >> 5) + 12;    // 12..15
          float w4[4] = {0.f, 0.f, 0.f, 0.f};
          if (jg < jcols && 4 * gq < jl) omega4(orow, gq, jmode, jtag, jseed, w4);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 4 * gq + e;
            const float w = c < jl ? w4[e] : 0.f;
            const float h = tf32_hi(w);
            const uint32_t off = (uint32_t)((c >> 3) * 1024 + (c & 7) * 128 +
                                            ((((jj * 4) >> 4) ^ (c & 7)) << 4) + ((jj * 4) & 15));
            *reinterpret_cast<float*>(bt + off) = h;
            *reinterpret_cast<float*>(bt + S_BHALF + off) = __fsub_rn(w, h);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tmem_st_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars.conv[s]));
      }
    }
  } else {
    // ---------------- Omega -> shared for each k-step, then the unit's partial rows ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int ctid = (warp - 6) * 32 + lane;     // 0..127
    long long it = 0;
    bool ok = true;
    for (long long ul = 0; ul < my_units && ok; ++ul) {
      int jb, rb, g, nst;
      long long j0;
      sketch_locate(jobs, start, njobs, (long long)blockIdx.x + ul * gridDim.x, &jb, &rb, &g,
                    &j0, &nst);
      const Tc32SketchJob& J = jobs[jb];
      {
        const int jl = J.l, jmode = J.mode;
        const uint32_t jcols = (uint32_t)J.cols, jka = (uint32_t)J.ka, jkb = (uint32_t)J.kb;
        const uint32_t jtag = J.tag;
        const uint64_t jseed = J.seed;
        for (int ks = 0; ks < nst; ++ks, ++it) {
          const int s = (int)(it % S_NS);
          const uint32_t use = (uint32_t)(it / S_NS);
          // stage s is free again (its copy has landed after the MMAs released it)
          if (!mbar_wait(smem_u32(&bars.full[s]), use & 1, &abort_flag)) { ok = false; break; }
          unsigned char* st0 = sm + s * S_STAGE;
          // Omega rows j0 + 32 ks + jj (layout order), groups of four columns
          unsigned char* bt = st0 + 2 * S_ATILE;
          const int jj = ctid & 31;
          // column of the unfolding and its Omega row (columns < 2^31)
          const uint32_t jg = (uint32_t)(j0 + (long long)ks * 32 + jj);
          const uint32_t jq = jg / jka;
          const uint64_t orow = (uint64_t)jq + (uint64_t)jkb * (jg - jq * jka);
          // four independent generator chains per thread, interleaved (one
          // such warp per SM sub-partition: latency is hidden by ILP)
#pragma unroll
          for (int r4 = 0; r4 < 3; ++r4) {
            const int gq = (ctid >> 5) + 4 * r4;    // 0..11 (12..15: the converters)
            float w4[4] = {0.f, 0.f, 0.f, 0.f};
            if (jg < jcols && 4 * gq < jl) omega4(orow, gq, jmode, jtag, jseed, w4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c = 4 * gq + e;
              const float w = c < jl ? w4[e] : 0.f;
              const float h = tf32_hi(w);
              const uint32_t off = (uint32_t)((c >> 3) * 1024 + (c & 7) * 128 +
                                              ((((jj * 4) >> 4) ^ (c & 7)) << 4) + ((jj * 4) & 15));
              *reinterpret_cast<float*>(bt + off) = h;
              *reinterpret_cast<float*>(bt + S_BHALF + off) = __fsub_rn(w, h);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars.conv[s]));
        }
      }
      if (!ok) break;
      if (!mbar_wait(smem_u32(&bars.accf[0]), (uint32_t)ul & 1, &abort_flag)) break;
      fence_after();
      uint32_t r0[32], r1[32], r2[32], r3[32];
      tmem_ld32(tmem + lane_off, r0);
      tmem_ld32(tmem + lane_off + 32u, r1);
      tmem_ld32(tmem + lane_off + 64u, r2);
      tmem_ld32(tmem + lane_off + 96u, r3);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.acce[0]));
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int i = rb * 256 + t * 128 + q * 32 + lane;
        if (i >= J.n) continue;
        const uint32_t* a = t == 0 ? r0 : r2;
        const uint32_t* b = t == 0 ? r1 : r3;
        float4* o = reinterpret_cast<float4*>(J.part + ((long long)g * J.n + i) * 64);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          o[c] = make_float4(__uint_as_float(a[4 * c]), __uint_as_float(a[4 * c + 1]),
                             __uint_as_float(a[4 * c + 2]), __uint_as_float(a[4 * c + 3]));
#pragma unroll
        for (int c = 0; c < 8; ++c)
          o[8 + c] = make_float4(__uint_as_float(b[4 * c]), __uint_as_float(b[4 * c + 1]),
                                 __uint_as_float(b[4 * c + 2]), __uint_as_float(b[4 * c + 3]));
      }
    }
  }
  fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0 && my_units > 0) {
    int jb, rb, g, nst;
    long long j0;
    sketch_locate(jobs, start, njobs, (long long)blockIdx.x, &jb, &rb, &g, &j0, &nst);
    atomicExch(jobs[jb].err, (int)TK_ETIMEOUT);
  }
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(512u) : "memory");
  }
}

__global__ void __launch_bounds__(S_THREADS, 1)
k_tc32_sketch(const __grid_constant__ Tc32SketchJob job) {
  sketch_body(&job, nullptr, 1, job.units, false);
}

__global__ void __launch_bounds__(S_THREADS, 1)
k_tc32_sketch_batch(const Tc32SketchJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                    int njobs, uint32_t total) {
  sketch_body(jobs, start, njobs, (long long)total, true);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2D FP32 map (inner dimension contiguous, row stride `stride` elements),
// box 32 (inner, 128 B) x box_outer, 128-byte swizzle.
bool map_f32(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t stride,
             uint32_t box_outer) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {stride * 4};
  cuuint32_t box[2] = {32, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tc32_ok(View v, int m, const void* X) {
  return v.P == 1 && v.n >= 1 && (v.n % 4) == 0 && v.cols() >= 1 && m >= 1 && m <= 64 &&
         (((uintptr_t)X) & 15) == 0 && v.n < (1 << 30) && v.cols() < (1LL << 31) &&
         encode_fn() != nullptr;
}

size_t tc32_xtb_scratch(View v) {
  const int64_t n_pad = (v.n + 31) / 32 * 32;
  return (size_t)128 * n_pad * sizeof(float) + 256;
}

bool tc32_xtb_jobs(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm, int m,
                   float* out, int out_mode, int64_t ld, void* scratch, int* err,
                   Tc32SplitJob* sj, Tc32XtbJob* xj) {
  if (!tc32_ok(v, m, X)) return false;
  const int n = (int)v.n;
  const int n_pad = (n + 31) / 32 * 32;
  float* B2 = (float*)scratch;
  *sj = Tc32SplitJob{B, b_ri, b_cm, B2, n, m, n_pad};
  std::memset(xj, 0, sizeof(*xj));
  if (!map_f32(&xj->mx, X, (uint64_t)n, (uint64_t)v.cols(), (uint64_t)n, 128)) return false;
  if (!map_f32(&xj->mb, B2, (uint64_t)n_pad, 128, (uint64_t)n_pad, 64)) return false;
  xj->out = out;
  xj->err = err;
  xj->cols = v.cols();
  xj->units = (v.cols() + 255) / 256;
  xj->ld = ld;
  xj->n = n;
  xj->nk = n_pad / 32;
  xj->m = m;
  xj->out_mode = out_mode;
  return true;
}

uint32_t tc32_split_blocks(const Tc32SplitJob& j) {
  return (uint32_t)((64LL * j.n_pad + 255) / 256);
}

size_t tc32_xtb_smem() { return (size_t)tc::X_NS * tc::X_STAGE + 1024; }

static void tc32_attrs() {
  static bool done = false;
  if (done) return;
  const int smem = (int)tc32_xtb_smem();
  cudaFuncSetAttribute(tc::k_tc32_xtb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(tc::k_tc32_xtb_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  done = true;
}

cudaError_t launch_tc32_xtb(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                            int m, float* out, int out_mode, int64_t ld, void* scratch, int* err,
                            cudaStream_t st) {
  Tc32SplitJob sj;
  Tc32XtbJob xj;
  if (!tc32_xtb_jobs(X, v, B, b_ri, b_cm, m, out, out_mode, ld, scratch, err, &sj, &xj))
    return cudaErrorInvalidValue;
  count_kernels(1);
  tc::k_split_b<<<tc32_split_blocks(sj), 256, 0, st>>>(sj);
  tc32_attrs();
  const long long grid = std::min<long long>(xj.units, (long long)num_sms());
  count_kernels(1);
  tc::k_tc32_xtb<<<(unsigned)grid, tc::X_THREADS, tc32_xtb_smem(), st>>>(xj);
  return cudaGetLastError();
}


int tc32_sketch_groups(View v) {
  // about eight units per SM; column groups of at least 32 columns
  const long long nrb = (v.n + 255) / 256;
  const long long want = std::max<long long>(1, 8LL * num_sms() / nrb);
  long long cpg = (v.cols() + want - 1) / want;
  cpg = std::max<long long>(32, (cpg + 31) / 32 * 32);
  return (int)((v.cols() + cpg - 1) / cpg);
}

size_t tc32_sketch_part_bytes(View v) {
  return (size_t)tc32_sketch_groups(v) * v.n * 64 * sizeof(float) + 256;
}

size_t tc32_sketch_smem() { return (size_t)tc::S_NS * tc::S_STAGE + 1024; }

bool tc32_sketch_job(const void* X, View v, int l, uint64_t seed, uint32_t tag, int mode,
                     int64_t ka, int64_t kb, float* part, int* err, void* shadow,
                     Tc32SketchJob* j) {
  if (!tc32_ok(v, l, X)) return false;
  std::memset(j, 0, sizeof(*j));
  if (!map_f32(&j->mx, X, (uint64_t)v.n, (uint64_t)v.cols(), (uint64_t)v.n, 32)) return false;
  const int groups = tc32_sketch_groups(v);
  const long long cpg0 = (v.cols() + groups - 1) / groups;
  j->part = part;
  j->err = err;
  j->shadow = (__nv_bfloat16*)shadow;
  j->cols = v.cols();
  j->cpg = (cpg0 + 31) / 32 * 32;
  j->groups = (int)((v.cols() + j->cpg - 1) / j->cpg);
  j->n = (int)v.n;
  j->nrb = (int)((v.n + 255) / 256);
  j->units = (long long)j->nrb * j->groups;
  if (ka <= 0) {
    ka = v.cols();
    kb = 1;
  }
  j->ka = ka;
  j->kb = kb;
  j->seed = seed;
  j->tag = tag;
  j->l = l;
  j->mode = mode;
  return true;
}

static void tc32_sketch_attrs() {
  static bool done = false;
  if (done) return;
  const int smem = (int)tc32_sketch_smem();
  cudaFuncSetAttribute(tc::k_tc32_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(tc::k_tc32_sketch_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem);
  done = true;
}

cudaError_t launch_tc32_sketch(const Tc32SketchJob& j, cudaStream_t st) {
  tc32_sketch_attrs();
  const long long grid = std::min<long long>(j.units, (long long)num_sms());
  count_kernels(1);
  tc::k_tc32_sketch<<<(unsigned)grid, tc::S_THREADS, tc32_sketch_smem(), st>>>(j);
  return cudaGetLastError();
}


cudaError_t launch_batch_tc32(const BatchLaunch& b, cudaStream_t st) {
  if (b.total == 0 || b.njobs == 0) return cudaSuccess;
  if (b.kind == BK_TC32SPLIT) return run_batch(tc::k_split_b_batch, b, 256, st);
  if (b.kind == BK_TC32SKETCH) {
    tc32_sketch_attrs();
    const unsigned grid = (unsigned)std::min<long long>((long long)b.total, (long long)num_sms());
    count_kernels(1);
    tc::k_tc32_sketch_batch<<<grid, tc::S_THREADS, tc32_sketch_smem(), st>>>(
        (const Tc32SketchJob*)b.jobs, b.start, b.njobs, b.total);
    return cudaGetLastError();
  }
  if (b.kind != BK_TC32XTB) return cudaErrorInvalidValue;
  tc32_attrs();
  const unsigned grid = (unsigned)std::min<long long>((long long)b.total, (long long)num_sms());
  count_kernels(1);
  tc::k_tc32_xtb_batch<<<grid, tc::X_THREADS, tc32_xtb_smem(), st>>>(
      (const Tc32XtbJob*)b.jobs, b.start, b.njobs, b.total);
  return cudaGetLastError();
}

}  // namespace tk

using namespace tk;

extern "C" tk_status tucker_debug_tf32_mma(const float* A, const float* B, float* D, int mode,
                                           void* stream) {
  if (!A || !B || !D || mode < 0 || mode > 1) return TK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&err, sizeof(int), st);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    count_kernels(1);
    tc::k_tf32_probe<<<1, 128, 0, st>>>(A, B, D, mode, err);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return from_cuda(e);
  return h ? (tk_status)h : TK_OK;
}

