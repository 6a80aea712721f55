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
          const uint32_t base = smem_u32(sm + s * X_STAGE);
#pragma unroll
          for (int t = 0; t < X_TM; ++t) {
            const uint32_t d = tmem + (uint32_t)((b * X_TM + t) * 64);
            const uint32_t lo = tmem + X_LO0 + (uint32_t)((s * X_TM + t) * 32);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t da = desc_sw128(base + t * X_ATILE + kk * 32, 16, 1024);
              const uint64_t dbh = desc_sw128(base + X_TM * X_ATILE + kk * 32, 16, 1024);
              const uint64_t dbl = desc_sw128(base + X_TM * X_ATILE + X_BHALF + kk * 32, 16, 1024);
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

cudaError_t launch_batch_tc32(const BatchLaunch& b, cudaStream_t st) {
  if (b.total == 0 || b.njobs == 0) return cudaSuccess;
  if (b.kind == BK_TC32SPLIT) return run_batch(tc::k_split_b_batch, b, 256, st);
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

