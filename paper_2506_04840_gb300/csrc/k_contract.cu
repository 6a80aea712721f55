// Strided mode-k contractions on CUDA cores (FFMA / DFMA), unfolding-free.
//
//  k_xb   : partial products of Y = X_(k) B, B = Omega_k (generated in
//           registers from Philox, Algorithm 2/3 sketch) or B = W stored in
//           the (P, l, S) layout (second half of the power step
//           X_(k)(X_(k)^T Q)).
//  k_xtb  : out = X x_k B^T, i.e. out[j, c] = sum_i X_(k)[i, j] B[i, c],
//           written in the (P, m, S) layout.  This is the mode-k product of
//           Section 2 with B^T, used for W = X_(k)^T Q, for the TTM shrink
//           G <- G x_k U_k^T of Algorithms 2/3, and (with B = U^T) for the
//           expansion G x_k U_k of the relative error.
//  k_xtb_err : the last expansion fused with sum (A - A_hat)^2 and sum A^2
//           (Section 5, RE), so A_hat is never stored.
//
// X(p, i, s) sits at p + P*(i + n*s); column j = p + P*s of X_(k).
#include <algorithm>

#include "tk_batch.h"
#include "tk_common.cuh"
#include "tk_internal.h"

namespace tk {

constexpr int XB_TJ = 32;   // column chunk of k_xb (FP32 accumulation; FP64 uses 16)
template <typename TA> struct xb_tj { static constexpr int value = sizeof(TA) == 8 ? 16 : XB_TJ; };

// Block (bx, by) of the product: rows bx*TI.., columns of split by.
template <typename TX, int LC, int TM, bool OMEGA>
__device__ __forceinline__ void xb_body(const TX* __restrict__ X, int64_t P, int64_t n, int64_t S,
                                        const typename acc_of<TX>::type* __restrict__ W, int l,
                                        uint64_t seed, uint32_t tag, int mode,
                                        int64_t cols_per_split,
                                        typename acc_of<TX>::type* __restrict__ part,
                                        unsigned bx, unsigned by) {
  typedef typename acc_of<TX>::type TA;
  constexpr int TN = LC / 16;
  constexpr int TI = 16 * TM;
  constexpr int TJ = xb_tj<TA>::value;
  __shared__ TA Xs[TJ][TI + 1];
  __shared__ TA Bs[TJ][LC];
  __shared__ int64_t offx[TJ];
  __shared__ int64_t offw[TJ];

  const int tid = threadIdx.x;
  const int ti = tid & 15, tc = tid >> 4;
  const int64_t i0 = (int64_t)bx * TI;
  const int64_t ncols = P * S;
  const int64_t jb = (int64_t)by * cols_per_split;
  const int64_t je = min(ncols, jb + cols_per_split);

  TA acc[TM][TN];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int q = 0; q < TN; ++q) acc[m][q] = (TA)0;

  for (int64_t j0 = jb; j0 < je; j0 += TJ) {
    if (tid < TJ) {
      const int64_t j = j0 + tid;
      if (j < je) {
        const int64_t s = j / P, p = j - s * P;
        offx[tid] = p + P * n * s;
        offw[tid] = p + P * (int64_t)l * s;
      } else {
        offx[tid] = -1;
        offw[tid] = -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < TI * TJ; e += TK_THREADS) {
      int ii, jj;
      if (P == 1) { ii = e % TI; jj = e / TI; } else { jj = e % TJ; ii = e / TJ; }
      const int64_t i = i0 + ii;
      const int64_t o = offx[jj];
      TA v = (TA)0;
      if (o >= 0 && i < n) v = load_as<TA>(X + o + P * i);
      Xs[jj][ii] = v;
    }
    if (OMEGA) {
      for (int e = tid; e < TJ * (LC / 4); e += TK_THREADS) {
        const int jj = e % TJ, g = e / TJ;
        float w4[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t j = j0 + jj;
        if (j < je && 4 * g < l) omega4((uint64_t)j, g, mode, tag, seed, w4);
#pragma unroll
        for (int q = 0; q < 4; ++q) Bs[jj][4 * g + q] = (4 * g + q < l) ? (TA)w4[q] : (TA)0;
      }
    } else {
      for (int e = tid; e < TJ * LC; e += TK_THREADS) {
        int jj, c;
        if (P == 1) { c = e % LC; jj = e / LC; } else { jj = e % TJ; c = e / TJ; }
        const int64_t o = offw[jj];
        TA v = (TA)0;
        if (o >= 0 && c < l) v = W[o + P * c];
        Bs[jj][c] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      TA a[TM], b[TN];
#pragma unroll
      for (int m = 0; m < TM; ++m) a[m] = Xs[jj][ti + 16 * m];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[jj][tc + 16 * q];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int q = 0; q < TN; ++q) acc[m][q] = fma(a[m], b[q], acc[m][q]);
    }
    __syncthreads();
  }
  TA* dst = part + (int64_t)by * n * LC;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int64_t i = i0 + ti + 16 * m;
    if (i < n) {
#pragma unroll
      for (int q = 0; q < TN; ++q) dst[i * LC + tc + 16 * q] = acc[m][q];
    }
  }
}

template <typename TX, int LC, int TM, bool OMEGA>
__global__ void __launch_bounds__(TK_THREADS)
k_xb(const TX* __restrict__ X, int64_t P, int64_t n, int64_t S,
     const typename acc_of<TX>::type* __restrict__ W, int l, uint64_t seed, uint32_t tag,
     int mode, int64_t cols_per_split, typename acc_of<TX>::type* __restrict__ part) {
  xb_body<TX, LC, TM, OMEGA>(X, P, n, S, W, l, seed, tag, mode, cols_per_split, part, blockIdx.x,
                             blockIdx.y);
}

// Y[i, c] = sum over splits of part[split][i][c] (- alpha Q[i, c]).  A block
// of 256 threads owns 32 consecutive outputs (c fastest: coalesced reads of
// the partials); its 8 warps take every 8th split and the 8 warp sums are
// added in a fixed order.
template <typename TA>
__device__ __forceinline__ void reduce_body(const TA* __restrict__ part, int splits, int64_t n,
                                            int l, int lc, const double* __restrict__ Q,
                                            const double* __restrict__ alpha,
                                            double* __restrict__ Y, unsigned bx,
                                            const TA* __restrict__ part_lo = nullptr) {
  __shared__ double red[8][32];
  const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t idx = (int64_t)bx * 32 + o;
  const bool valid = idx < n * l;
  const int c = valid ? (int)(idx % l) : 0;
  const int64_t i = valid ? idx / l : 0;
  double s0 = 0.0, s1 = 0.0;
  if (valid) {
    const TA* src = part + i * lc + c;
    const int64_t stride = n * lc;
    int sp = g;
    for (; sp + 8 < splits; sp += 16) {
      s0 += (double)src[(int64_t)sp * stride];
      s1 += (double)src[(int64_t)(sp + 8) * stride];
    }
    if (sp < splits) s0 += (double)src[(int64_t)sp * stride];
    if (part_lo != nullptr) {
      const TA* lo = part_lo + i * lc + c;
      for (sp = g; sp < splits; sp += 8) s1 += (double)lo[(int64_t)sp * stride];
    }
  }
  red[g][o] = s0 + s1;
  __syncthreads();
  if (g == 0 && valid) {
    double s = ((red[0][o] + red[1][o]) + (red[2][o] + red[3][o])) +
               ((red[4][o] + red[5][o]) + (red[6][o] + red[7][o]));
    if (Q != nullptr) s -= alpha[0] * Q[i + n * c];
    Y[i + n * c] = s;
  }
  __syncthreads();
}

template <typename TA>
__global__ void __launch_bounds__(256)
k_reduce(const TA* __restrict__ part, int splits, int64_t n, int l, int lc,
         const double* __restrict__ Q, const double* __restrict__ alpha, double* __restrict__ Y,
         const TA* __restrict__ part_lo) {
  reduce_body<TA>(part, splits, n, l, lc, Q, alpha, Y, blockIdx.x, part_lo);
}

// out[j, c] = sum_i X(p, i, s) B(i, c) for a tile of TJ columns and LC
// outputs.  EPI = 0 stores out in the (P, m, S) layout; EPI = 1 (S == 1)
// compares with A(p, c) and accumulates the two squared sums.
// Block (bx, by) of a gx-wide grid: columns bx*TJ.., outputs by*LC..
template <typename TX, int LC, int EPI>
__device__ __forceinline__ void xtb_body(const TX* __restrict__ X, int64_t P, int64_t n,
                                         int64_t S, const double* __restrict__ B, int64_t b_ri,
                                         int64_t b_cm, int m,
                                         typename acc_of<TX>::type* __restrict__ out,
                                         const typename acc_of<TX>::type* __restrict__ A,
                                         double* __restrict__ err_part, unsigned bx, unsigned by,
                                         unsigned gx) {
  typedef typename acc_of<TX>::type TA;
  constexpr int TN = LC / 16;
  constexpr int TMJ = 8;
  constexpr int TJ = 16 * TMJ;
  constexpr int TK = sizeof(TA) == 8 ? 8 : 16;
  __shared__ TA Xs[TK][TJ + 1];
  __shared__ TA Bs[TK][LC];
  __shared__ int64_t offx[TJ];
  __shared__ double red[2][TK_THREADS / 32];

  const int tid = threadIdx.x;
  // lanes run along the contiguous output dimension when writing
  const bool cfast = (EPI == 0) && (P == 1);
  const int tj = cfast ? (tid >> 4) : (tid & 15);
  const int tc = cfast ? (tid & 15) : (tid >> 4);
  const int64_t ncols = P * S;
  const int64_t j0 = (int64_t)bx * TJ;
  const int c0 = by * LC;

  if (tid < TJ) {
    const int64_t j = j0 + tid;
    if (j < ncols) {
      const int64_t s = j / P, p = j - s * P;
      offx[tid] = p + P * n * s;
    } else {
      offx[tid] = -1;
    }
  }
  // FP32, EPI = 0: each slab of TK rows is summed from zero and folded into
  // an (acc, cmp) pair by TwoSum (the compensation of the FP32 mode-major
  // kernels), so strided TTMs and the error pass's expansions keep their
  // results to about one rounding.
  // EPI = 1 accumulates the residual instead: the accumulator starts at
  // A(p, c) and the products are subtracted, so it is rounded at the scale of
  // what remains to be subtracted rather than of a_hat (the error pass).
  constexpr bool COMP = sizeof(TA) == 4 && EPI == 0;
  TA acc[TMJ][TN], cmp[TMJ][TN];
  __syncthreads();
#pragma unroll
  for (int a = 0; a < TMJ; ++a)
#pragma unroll
    for (int q = 0; q < TN; ++q) {
      cmp[a][q] = (TA)0;
      acc[a][q] = (TA)0;
      if (EPI == 1) {
        const int64_t j = j0 + tj + 16 * a;   // S == 1: j = p
        const int c = c0 + tc + 16 * q;
        if (j < ncols && c < m) acc[a][q] = A[j + P * (int64_t)c];
      }
    }

  for (int64_t ib = 0; ib < n; ib += TK) {
    for (int e = tid; e < TK * TJ; e += TK_THREADS) {
      int ii, jj;
      if (P == 1) { ii = e % TK; jj = e / TK; } else { jj = e % TJ; ii = e / TJ; }
      const int64_t i = ib + ii;
      const int64_t o = offx[jj];
      TA v = (TA)0;
      if (o >= 0 && i < n) v = load_as<TA>(X + o + P * i);
      Xs[ii][jj] = v;
    }
    for (int e = tid; e < TK * LC; e += TK_THREADS) {
      int ii, c;
      if (b_cm == 1) { c = e % LC; ii = e / LC; } else { ii = e % TK; c = e / TK; }
      const int64_t i = ib + ii;
      TA v = (TA)0;
      if (i < n && c0 + c < m) v = (TA)B[i * b_ri + (int64_t)(c0 + c) * b_cm];
      Bs[ii][c] = v;
    }
    __syncthreads();
    TA sl[TMJ][TN];
#pragma unroll
    for (int x = 0; x < TMJ; ++x)
#pragma unroll
      for (int q = 0; q < TN; ++q) sl[x][q] = COMP ? (TA)0 : acc[x][q];
#pragma unroll
    for (int ii = 0; ii < TK; ++ii) {
      TA a[TMJ], b[TN];
#pragma unroll
      for (int q = 0; q < TMJ; ++q) a[q] = Xs[ii][tj + 16 * q];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = EPI == 1 ? -Bs[ii][tc + 16 * q] : Bs[ii][tc + 16 * q];
#pragma unroll
      for (int x = 0; x < TMJ; ++x)
#pragma unroll
        for (int q = 0; q < TN; ++q) sl[x][q] = fma(a[x], b[q], sl[x][q]);
      if constexpr (COMP) {
        // the first row is a slab of its own (a dominant leading term would
        // otherwise set the rounding scale of its whole slab)
        if (ii == 0 && ib == 0) {
#pragma unroll
          for (int x = 0; x < TMJ; ++x)
#pragma unroll
            for (int q = 0; q < TN; ++q) {
              acc[x][q] = sl[x][q];
              sl[x][q] = (TA)0;
            }
        }
      }
    }
#pragma unroll
    for (int x = 0; x < TMJ; ++x)
#pragma unroll
      for (int q = 0; q < TN; ++q) {
        if constexpr (COMP) {
          const TA t = __fadd_rn(acc[x][q], sl[x][q]);
          const TA z = __fsub_rn(t, acc[x][q]);
          const TA se = __fadd_rn(__fsub_rn(acc[x][q], __fsub_rn(t, z)), __fsub_rn(sl[x][q], z));
          acc[x][q] = t;
          cmp[x][q] = __fadd_rn(cmp[x][q], se);
        } else {
          acc[x][q] = sl[x][q];
        }
      }
    __syncthreads();
  }
  if constexpr (COMP) {
#pragma unroll
    for (int x = 0; x < TMJ; ++x)
#pragma unroll
      for (int q = 0; q < TN; ++q) acc[x][q] = __fadd_rn(acc[x][q], cmp[x][q]);
  }

  if (EPI == 0) {
#pragma unroll
    for (int x = 0; x < TMJ; ++x) {
      const int64_t j = j0 + tj + 16 * x;
      if (j >= ncols) continue;
      const int64_t s = j / P, p = j - s * P;
#pragma unroll
      for (int q = 0; q < TN; ++q) {
        const int c = c0 + tc + 16 * q;
        if (c < m) out[p + P * ((int64_t)c + (int64_t)m * s)] = acc[x][q];
      }
    }
  } else {
    // per-thread sums of TMJ*TN terms in the accumulation type (FP64 FMAs
    // run at a small fraction of the FP32 rate on this GPU), then FP64
    // across threads and blocks
    TA e2t = (TA)0, a2t = (TA)0;
#pragma unroll
    for (int x = 0; x < TMJ; ++x) {
      const int64_t j = j0 + tj + 16 * x;   // S == 1: j = p
      if (j >= ncols) continue;
#pragma unroll
      for (int q = 0; q < TN; ++q) {
        const int c = c0 + tc + 16 * q;
        if (c < m) {
          const TA av = A[j + P * (int64_t)c];
          const TA dv = acc[x][q];   // the residual (accumulated from A)
          e2t = fma(dv, dv, e2t);
          a2t = fma(av, av, a2t);
        }
      }
    }
    double e2 = (double)e2t, a2 = (double)a2t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = e2;
      red[1][tid >> 5] = a2;
    }
    __syncthreads();
    if (tid == 0) {
      double se = 0.0, sa = 0.0;
      for (int w = 0; w < TK_THREADS / 32; ++w) {
        se += red[0][w];
        sa += red[1][w];
      }
      const int64_t b = (int64_t)by * gx + bx;
      err_part[2 * b] = se;
      err_part[2 * b + 1] = sa;
    }
  }
}

template <typename TX, int LC, int EPI>
__global__ void __launch_bounds__(TK_THREADS)
k_xtb(const TX* __restrict__ X, int64_t P, int64_t n, int64_t S, const double* __restrict__ B,
      int64_t b_ri, int64_t b_cm, int m, typename acc_of<TX>::type* __restrict__ out,
      const typename acc_of<TX>::type* __restrict__ A, double* __restrict__ err_part) {
  xtb_body<TX, LC, EPI>(X, P, n, S, B, b_ri, b_cm, m, out, A, err_part, blockIdx.x, blockIdx.y,
                        gridDim.x);
}

__device__ __forceinline__ void error_final_body(const double* __restrict__ part, int blocks,
                                                 double* __restrict__ rel) {
  __shared__ double se[TK_THREADS], sa[TK_THREADS];
  double e = 0.0, a = 0.0;
  for (int b = threadIdx.x; b < blocks; b += TK_THREADS) {
    e += part[2 * b];
    a += part[2 * b + 1];
  }
  se[threadIdx.x] = e;
  sa[threadIdx.x] = a;
  __syncthreads();
  for (int o = TK_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      se[threadIdx.x] += se[threadIdx.x + o];
      sa[threadIdx.x] += sa[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) rel[0] = sa[0] > 0.0 ? sqrt(se[0] / sa[0]) : 0.0;
}

__global__ void __launch_bounds__(TK_THREADS)
k_error_final(const double* __restrict__ part, int blocks, double* __restrict__ rel) {
  error_final_body(part, blocks, rel);
}

// ---------------------------------------------------------------------------
// Work-list launches: a persistent grid strides over the concatenated blocks
// of all jobs; each job's block runs the single-problem body unchanged.
// ---------------------------------------------------------------------------
template <typename TX, int LC, int TM, bool OMEGA>
__global__ void __launch_bounds__(TK_THREADS)
k_xb_batch(const XbJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
           uint32_t total) {
  typedef typename acc_of<TX>::type TA;
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const XbJob J = jobs[j];
    const uint32_t lb = b - __ldg(start + j);
    xb_body<TX, LC, TM, OMEGA>((const TX*)J.X, J.P, J.n, J.S, (const TA*)J.W, J.l, J.seed, J.tag,
                               J.mode, J.cps, (TA*)J.part, lb % (uint32_t)J.gx,
                               lb / (uint32_t)J.gx);
    __syncthreads();
  }
}

template <typename TA>
__global__ void __launch_bounds__(256)
k_reduce_batch(const ReduceJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
               uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const ReduceJob J = jobs[j];
    reduce_body<TA>((const TA*)J.part, J.splits, J.n, J.l, J.lc, J.Q, J.alpha, J.Y,
                    b - __ldg(start + j), (const TA*)J.part_lo);
  }
}

template <typename TX, int LC, int EPI>
__global__ void __launch_bounds__(TK_THREADS)
k_xtb_batch(const XtbJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
            uint32_t total) {
  typedef typename acc_of<TX>::type TA;
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const XtbJob J = jobs[j];
    const uint32_t lb = b - __ldg(start + j);
    xtb_body<TX, LC, EPI>((const TX*)J.X, J.P, J.n, J.S, J.B, J.b_ri, J.b_cm, J.m, (TA*)J.out,
                          (const TA*)J.A, J.err, lb % (uint32_t)J.gx, lb / (uint32_t)J.gx,
                          (uint32_t)J.gx);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TK_THREADS)
k_error_final_batch(const ErrFinalJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                    int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const ErrFinalJob J = jobs[batch_job(start, njobs, b)];
    error_final_body(J.part, J.blocks, J.rel);
    __syncthreads();
  }
}

template <typename TX, int EPI>
static cudaError_t xtb_batch_lc(const BatchLaunch& b, cudaStream_t st) {
  switch (b.tile) {
    case 16: return run_batch(k_xtb_batch<TX, 16, EPI>, b, TK_THREADS, st);
    case 32: return run_batch(k_xtb_batch<TX, 32, EPI>, b, TK_THREADS, st);
    default: return run_batch(k_xtb_batch<TX, 64, EPI>, b, TK_THREADS, st);
  }
}

template <typename TX, bool OMEGA>
static cudaError_t xb_batch_lc(const BatchLaunch& b, cudaStream_t st) {
  switch (b.tile) {
    case 16: return run_batch(k_xb_batch<TX, 16, 8, OMEGA>, b, TK_THREADS, st);
    case 32: return run_batch(k_xb_batch<TX, 32, 8, OMEGA>, b, TK_THREADS, st);
    case 64: return run_batch(k_xb_batch<TX, 64, 8, OMEGA>, b, TK_THREADS, st);
    default: return run_batch(k_xb_batch<TX, 128, 4, OMEGA>, b, TK_THREADS, st);
  }
}

template <typename TX>
static cudaError_t xb_batch_go(const BatchLaunch& b, cudaStream_t st) {
  return b.flag ? xb_batch_lc<TX, true>(b, st) : xb_batch_lc<TX, false>(b, st);
}

cudaError_t launch_batch_contract(const BatchLaunch& b, cudaStream_t st) {
  switch (b.kind) {
    case BK_XB:
      if (b.xt == X_F64) return xb_batch_go<double>(b, st);
      if (b.xt == X_F32) return xb_batch_go<float>(b, st);
      return xb_batch_go<__nv_bfloat16>(b, st);
    case BK_REDUCE:
      if (b.xt == X_F64) return run_batch(k_reduce_batch<double>, b, 256, st);
      return run_batch(k_reduce_batch<float>, b, 256, st);
    case BK_XTB:
      if (b.xt == X_F64)
        return b.flag ? xtb_batch_lc<double, 1>(b, st) : xtb_batch_lc<double, 0>(b, st);
      if (b.xt == X_F32)
        return b.flag ? xtb_batch_lc<float, 1>(b, st) : xtb_batch_lc<float, 0>(b, st);
      if (b.flag) return cudaErrorInvalidValue;
      return xtb_batch_lc<__nv_bfloat16, 0>(b, st);
    case BK_ERRFIN:
      return run_batch(k_error_final_batch, b, TK_THREADS, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
int xb_lc(int l) { return l <= 16 ? 16 : (l <= 32 ? 32 : (l <= 64 ? 64 : 128)); }

static int xb_tm(int lc) { return lc <= 64 ? 8 : 4; }

static int xb_ti(int lc) { return 16 * xb_tm(lc); }

int xb_grid_x(View v, int l) { return (int)((v.n + xb_ti(xb_lc(l)) - 1) / xb_ti(xb_lc(l))); }

int64_t xb_cols_per_split(XType xt, View v, int splits) {
  const int64_t tj = xt == X_F64 ? 16 : XB_TJ;
  int64_t cps = (v.cols() + splits - 1) / splits;
  return (cps + tj - 1) / tj * tj;
}

int xb_splits(XType xt, View v, int l) {
  if (xtb32_ok(xt, v, (const void*)1)) return xb32_shape(v, l).splits;
  const int lc = xb_lc(l);
  const int64_t itiles = (v.n + xb_ti(lc) - 1) / xb_ti(lc);
  const int64_t target = 4LL * num_sms();
  int64_t splits = (target + itiles - 1) / itiles;
  const int64_t maxs = std::max<int64_t>(1, (v.cols() + XB_TJ - 1) / XB_TJ);
  splits = std::min(splits, maxs);
  return (int)std::max<int64_t>(1, splits);
}

template <typename TX, int LC>
static cudaError_t xb_dispatch(const void* X, View v, const void* W, int l, uint64_t seed,
                               uint32_t tag, int mode, void* part, int splits, cudaStream_t st) {
  typedef typename acc_of<TX>::type TA;
  constexpr int TM = LC <= 64 ? 8 : 4;
  const int64_t ti = 16 * TM;
  const int64_t ncols = v.cols();
  constexpr int TJ = xb_tj<TA>::value;
  int64_t cps = (ncols + splits - 1) / splits;
  cps = (cps + TJ - 1) / TJ * TJ;
  dim3 grid((unsigned)((v.n + ti - 1) / ti), (unsigned)splits);
  count_kernels(1);
  if (W == nullptr)
    k_xb<TX, LC, TM, true><<<grid, TK_THREADS, 0, st>>>((const TX*)X, v.P, v.n, v.S, nullptr, l,
                                                       seed, tag, mode, cps, (TA*)part);
  else
    k_xb<TX, LC, TM, false><<<grid, TK_THREADS, 0, st>>>((const TX*)X, v.P, v.n, v.S,
                                                        (const TA*)W, l, seed, tag, mode, cps,
                                                        (TA*)part);
  return cudaGetLastError();
}

template <typename TX>
static cudaError_t xb_lc_dispatch(const void* X, View v, const void* W, int l, uint64_t seed,
                                  uint32_t tag, int mode, void* part, int splits,
                                  cudaStream_t st) {
  switch (xb_lc(l)) {
    case 16: return xb_dispatch<TX, 16>(X, v, W, l, seed, tag, mode, part, splits, st);
    case 32: return xb_dispatch<TX, 32>(X, v, W, l, seed, tag, mode, part, splits, st);
    case 64: return xb_dispatch<TX, 64>(X, v, W, l, seed, tag, mode, part, splits, st);
    default: return xb_dispatch<TX, 128>(X, v, W, l, seed, tag, mode, part, splits, st);
  }
}

cudaError_t launch_xb(XType xt, const void* X, View v, const void* W, int l, uint64_t seed,
                      uint32_t tag, int mode, void* part, int splits, cudaStream_t st,
                      int64_t ka, int64_t kb, void* part_lo) {
  if (v.n <= 0 || v.cols() <= 0 || l <= 0) return cudaSuccess;
  if (xtb32_ok(xt, v, X))
    return launch_xb32(X, v, W, l, seed, tag, mode, part, splits, st, ka, kb, part_lo);
  if (part_lo != nullptr) return cudaErrorInvalidValue;
  if (ka > 0 && W == nullptr && ka != v.cols()) return cudaErrorInvalidValue;
  switch (xt) {
    case X_F64: return xb_lc_dispatch<double>(X, v, W, l, seed, tag, mode, part, splits, st);
    case X_F32: return xb_lc_dispatch<float>(X, v, W, l, seed, tag, mode, part, splits, st);
    default:
      return xb_lc_dispatch<__nv_bfloat16>(X, v, W, l, seed, tag, mode, part, splits, st);
  }
}

cudaError_t launch_reduce(XType xt, const void* part, int splits, int64_t n, int l, int lc,
                          const double* Q, const double* alpha, double* Y, cudaStream_t st,
                          const void* part_lo) {
  const int64_t tot = n * l;
  if (tot <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((tot + 31) / 32);
  count_kernels(1);
  if (xt == X_F64)
    k_reduce<double><<<blocks, 256, 0, st>>>((const double*)part, splits, n, l, lc, Q, alpha, Y,
                                             (const double*)part_lo);
  else
    k_reduce<float><<<blocks, 256, 0, st>>>((const float*)part, splits, n, l, lc, Q, alpha, Y,
                                            (const float*)part_lo);
  return cudaGetLastError();
}

static int xtb_lc(int m) { return m <= 16 ? 16 : (m <= 32 ? 32 : 64); }

int xtb_tile(int m) { return xtb_lc(m); }

template <typename TX, int LC, int EPI>
static cudaError_t xtb_go(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                          int m, void* out, const void* A, double* err, cudaStream_t st) {
  typedef typename acc_of<TX>::type TA;
  dim3 grid((unsigned)((v.cols() + 127) / 128), (unsigned)((m + LC - 1) / LC));
  count_kernels(1);
  k_xtb<TX, LC, EPI><<<grid, TK_THREADS, 0, st>>>((const TX*)X, v.P, v.n, v.S, B, b_ri, b_cm, m,
                                                  (TA*)out, (const TA*)A, err);
  return cudaGetLastError();
}

template <typename TX, int EPI>
static cudaError_t xtb_lc_go(const void* X, View v, const double* B, int64_t b_ri, int64_t b_cm,
                             int m, void* out, const void* A, double* err, cudaStream_t st) {
  switch (xtb_lc(m)) {
    case 16: return xtb_go<TX, 16, EPI>(X, v, B, b_ri, b_cm, m, out, A, err, st);
    case 32: return xtb_go<TX, 32, EPI>(X, v, B, b_ri, b_cm, m, out, A, err, st);
    default: return xtb_go<TX, 64, EPI>(X, v, B, b_ri, b_cm, m, out, A, err, st);
  }
}

cudaError_t launch_xtb(XType xt, const void* X, View v, const double* B, int64_t b_ri,
                       int64_t b_cm, int m, void* out, cudaStream_t st, int tout,
                       void* scratch, const float* B32, bool comp) {
  if (v.cols() <= 0 || m <= 0) return cudaSuccess;
  if (xtb32_ok(xt, v, X))
    return launch_xtb32(X, v, B, b_ri, b_cm, m, out, st, tout, scratch, B32, comp);
  if (tout) return cudaErrorInvalidValue;
  switch (xt) {
    case X_F64: return xtb_lc_go<double, 0>(X, v, B, b_ri, b_cm, m, out, nullptr, nullptr, st);
    case X_F32: return xtb_lc_go<float, 0>(X, v, B, b_ri, b_cm, m, out, nullptr, nullptr, st);
    default:
      return xtb_lc_go<__nv_bfloat16, 0>(X, v, B, b_ri, b_cm, m, out, nullptr, nullptr, st);
  }
}

int xtb_error_blocks(XType xt, View v, int m) {
  if (err32_ok(xt, v)) return err32_blocks(v, m);
  const int lc = xtb_lc(m);
  return (int)(((v.cols() + 127) / 128) * ((m + lc - 1) / lc));
}

cudaError_t launch_xtb_error(XType xt, const void* T, View v, const double* B, int64_t b_ri,
                             int64_t b_cm, int m, const void* A, double* err_part, int* blocks,
                             cudaStream_t st, const float* B32) {
  *blocks = xtb_error_blocks(xt, v, m);
  if (v.cols() <= 0 || m <= 0) return cudaSuccess;
  if (err32_ok(xt, v)) return launch_err32(T, v, B, b_ri, b_cm, m, A, err_part, st, B32);
  if (xt == X_F64) return xtb_lc_go<double, 1>(T, v, B, b_ri, b_cm, m, nullptr, A, err_part, st);
  return xtb_lc_go<float, 1>(T, v, B, b_ri, b_cm, m, nullptr, A, err_part, st);
}

cudaError_t launch_error_final(const double* err_part, int blocks, double* rel_err,
                               cudaStream_t st) {
  count_kernels(1);
  k_error_final<<<1, TK_THREADS, 0, st>>>(err_part, blocks, rel_err);
  return cudaGetLastError();
}

}  // namespace tk
