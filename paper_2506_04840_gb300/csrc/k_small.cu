// [Q, Sigma, ~] = svd(Y, 'econ') for a tall n x l matrix Y (Algorithms 2
// and 3 call it after the sketch and after every shifted power step), plus
// the adaptive shift update of Algorithms 2/3.
//
// Method (all on the device, no host round trip):
//   Householder QR Y = Q_h R;  one-sided (Hestenes) Jacobi on the columns of
//   R^T, whose accumulated rotations U_R are R's left singular vectors
//   (orthogonal even when Y is rank deficient) and whose column norms are
//   Sigma;  descending sort;  Q = Q_h U_R;  sign convention (entry of
//   largest |value| positive, lowest row on ties);  shift update.
// Paths:
//   * one CTA (k_svd_one) when Y fits in shared memory;
//   * otherwise a two-level TSQR: k_leaf_qr (row blocks) -> k_root (QR of the
//     stacked triangles, Jacobi, root Q times U_R) -> k_leaf_q (block Q times
//     the root result) -> k_sign.
// The working precision T is FP64 for FP64 tensors and FP32 for FP32/BF16
// tensors, matching the precision in which Y itself was formed.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tk_common.cuh"
#include "tk_batch.h"
#include "tk_internal.h"

namespace tk {

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Division and square root for the small solvers' scalar steps: in FP32 the
// fast intrinsics (a few ulp; the correctly rounded forms have ~5x their
// latency, which sits on every Householder step's and Jacobi rotation's
// critical path), in FP64 the correctly rounded operations.
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float ssqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double ssqrt(double x) { return sqrt(x); }

// Householder reflector for column j of A (ld m) given ssq = sum of squares of
// its entries below the diagonal; run by one warp.  LAPACK-style generation
// (beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, v = x/(alpha - beta)).
template <typename T>
__device__ __forceinline__ void make_reflector(T* A, int m, int j, T ssq, T* tau) {
  const int lane = threadIdx.x & 31;
  T* x = A + (int64_t)m * j;
  const T alpha = x[j];
  const T xnorm = ssqrt(ssq);
  T beta = alpha, tj = (T)0;
  if (xnorm > (T)0) {
    const T mx = max((T)fabs(alpha), xnorm);
    const T rmx = sdiv((T)1, mx);
    const T a1 = alpha * rmx, x1 = xnorm * rmx;
    beta = -copysign(mx * ssqrt(a1 * a1 + x1 * x1), alpha);
    tj = sdiv(beta - alpha, beta);
    const T scal = sdiv((T)1, alpha - beta);
    for (int i = j + 1 + lane; i < m; i += 32) x[i] *= scal;
  }
  __syncwarp();
  if (lane == 0) {
    x[j] = beta;
    tau[j] = tj;
  }
}

// Householder QR with look-ahead, in place, of an m x l column-major matrix
// A (ld = m) in shared memory whose entries are O(1) (the caller scales);
// reflector j is (1, A[j+1:, j]) with factor tau[j]; R is the upper
// triangle.  Column c belongs to warp c % nw; the owner of column j+1 updates
// it first and builds reflector j+1 before the step's only barrier.
template <typename T>
__device__ void householder_qr_la(T* A, int m, int l, T* tau) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp == 0) {
    T s = 0;
    for (int i = 1 + lane; i < m; i += 32) s += A[i] * A[i];
    s = warp_sum(s);
    make_reflector(A, m, 0, s, tau);
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    const T tj = tau[j];
    const T* v = A + (int64_t)m * j;
    const int own_next = (j + 1) % nw;
    // the owner of column j+1 handles it first, then the rest of its columns
    for (int c = j + 1 + ((warp - (j + 1)) % nw + nw) % nw; c < l; c += nw) {
      T* y = A + (int64_t)m * c;
      if (tj != (T)0) {
        T w = lane == 0 ? y[j] : (T)0;
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * y[i];
        w = warp_sum(w) * tj;
        if (lane == 0) y[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] -= w * v[i];
        __syncwarp();
      }
      if (c == j + 1 && warp == own_next) {
        T s = 0;
        for (int i = c + 1 + lane; i < m; i += 32) s += y[i] * y[i];
        s = warp_sum(s);
        make_reflector(A, m, c, s, tau);
      }
    }
    __syncthreads();
  }
}

// Householder QR, in place, of an m x l column-major matrix A (ld = m) in
// shared memory; reflector j is (1, A[j+1:, j]) with factor tau[j]; R is the
// upper triangle.  LAPACK-style generation (beta = -sign(alpha) ||x||,
// tau = (beta - alpha)/beta, v = x / (alpha - beta)).
template <typename T>
__device__ void householder_qr(T* A, int m, int l, T* tau) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < l; ++j) {
    if (warp == 0) {
      T* x = A + (int64_t)m * j;
      T amax = (T)0;
      for (int i = j + 1 + lane; i < m; i += 32) amax = max(amax, (T)fabs(x[i]));
      amax = warp_max(amax);
      T ssq = (T)0;
      if (amax > (T)0) {
        const T inv = sdiv((T)1, amax);
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T t = x[i] * inv;
          ssq += t * t;
        }
      }
      ssq = warp_sum(ssq);
      const T xnorm = amax * ssqrt(ssq);
      const T alpha = x[j];
      T beta = alpha, tj = (T)0;
      if (xnorm > (T)0) {
        const T mx = max((T)fabs(alpha), xnorm);
        const T rmx = sdiv((T)1, mx);
        const T a1 = alpha * rmx, x1 = xnorm * rmx;
        beta = -copysign(mx * ssqrt(a1 * a1 + x1 * x1), alpha);
        tj = sdiv(beta - alpha, beta);
        const T scal = sdiv((T)1, alpha - beta);
        for (int i = j + 1 + lane; i < m; i += 32) x[i] *= scal;
      }
      __syncwarp();
      if (lane == 0) {
        x[j] = beta;
        tau[j] = tj;
      }
    }
    __syncthreads();
    const T tj = tau[j];
    const T* v = A + (int64_t)m * j;
    if (tj != (T)0) {
      for (int c = j + 1 + warp; c < l; c += nw) {
        T* y = A + (int64_t)m * c;
        T w = lane == 0 ? y[j] : (T)0;
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * y[i];
        w = warp_sum(w) * tj;
        if (lane == 0) y[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] -= w * v[i];
      }
    }
    __syncthreads();
  }
}

// Overwrite the reflectors in A (m x l, from householder_qr) with the first
// l columns of Q_h = H_0 H_1 ... H_{l-1} [I; 0] (backward accumulation).
template <typename T>
__device__ void form_q_inplace(T* A, int m, int l, const T* tau) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = l - 1; j >= 0; --j) {
    const T tj = tau[j];
    const T* v = A + (int64_t)m * j;
    if (tj != (T)0) {
      for (int c = j + 1 + warp; c < l; c += nw) {
        T* y = A + (int64_t)m * c;
        T w = lane == 0 ? y[j] : (T)0;
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * y[i];
        w = warp_sum(w) * tj;
        if (lane == 0) y[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] -= w * v[i];
      }
    }
    __syncthreads();
    T* x = A + (int64_t)m * j;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (i < j) x[i] = (T)0;
      else if (i == j) x[i] = (T)1 - tj;
      else x[i] = -tj * x[i];
    }
    __syncthreads();
  }
}

template <typename T> __device__ __forceinline__ T jacobi_tol(int l);
template <> __device__ __forceinline__ float jacobi_tol<float>(int l) {
  return fmaxf(4e-6f, 4.0f * (float)l * 5.9604645e-8f);
}
template <> __device__ __forceinline__ double jacobi_tol<double>(int l) {
  return 4.0 * (double)l * 1.1102230246251565e-16;
}

// One-sided Jacobi on the l columns of J (l x l), accumulating the rotations
// in Vp (starts as I) when Vp is non-null.  Round-robin pairing; each pair is
// handled by a group of g lanes (g = 4 for l <= 32, 8 above) and the rounds
// are spread over up to 8 warps synchronised by the named barrier 1 (only
// those warps wait).  All threads of the block must call it; threads outside
// the Jacobi warps return at once and the caller synchronises afterwards.
// The rotation parameters use fast reciprocal square roots: c = rsqrt(1+t^2),
// s = c t is an exact plane rotation up to rounding either way.
template <typename T>
__device__ void jacobi_warp(T* J, T* Vp, int l) {
  const int m2 = l + (l & 1);
  const int npairs = m2 / 2;
  const int g = l > 32 ? 8 : 4;
  const int nwj = min((npairs * g + 31) / 32, min(8, (int)(blockDim.x >> 5)));
  const int nthr = nwj * 32;
  if ((int)threadIdx.x >= nthr) return;
  const int lane = threadIdx.x & 31;
  const int groups = nthr / g;
  const int gi = (int)threadIdx.x / g, sub = (int)threadIdx.x % g;
  __shared__ int jflag[2];
  if (threadIdx.x == 0) jflag[0] = jflag[1] = 0;
  if (nwj > 1) asm volatile("bar.sync 1, %0;" :: "r"(nthr) : "memory");
  else __syncwarp();
  const T tol = jacobi_tol<T>(l);
  const T tol2 = tol * tol;
  const int max_sweeps = sizeof(T) == 8 ? 40 : 24;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const int fb = sweep & 1;
    int rotated = 0;
    for (int rd = 0; rd < m2 - 1; ++rd) {
      for (int pr0 = 0; pr0 < npairs; pr0 += groups) {
        const int pr = pr0 + gi;
        int p = 0, q = 0;
        bool act = pr < npairs;
        if (act) {
          if (pr == 0) { p = rd; q = m2 - 1; }
          else { p = (rd + pr) % (m2 - 1); q = (rd - pr + (m2 - 1)) % (m2 - 1); }
          act = p < l && q < l;
        }
        T a = 0, bb = 0, gm = 0;
        T* xp = J + (int64_t)l * p;
        T* xq = J + (int64_t)l * q;
        if (act)
          for (int i = sub; i < l; i += g) {
            const T u = xp[i], w = xq[i];
            a += u * u;
            bb += w * w;
            gm += u * w;
          }
        for (int o = 1; o < g; o <<= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          gm += __shfl_xor_sync(0xffffffffu, gm, o);
        }
        if (act && gm != (T)0 && gm * gm > tol2 * a * bb) {
          const T zeta = sdiv(bb - a, gm + gm);
          T t;
          if (fabs(zeta) > (T)1e15) t = sdiv((T)0.5, zeta);
          else t = copysign(sdiv((T)1, fabs(zeta) + ssqrt((T)1 + zeta * zeta)), zeta);
          const T cs = rsqrt((T)1 + t * t);
          const T sn = cs * t;
          for (int i = sub; i < l; i += g) {
            const T u = xp[i], w = xq[i];
            xp[i] = cs * u - sn * w;
            xq[i] = sn * u + cs * w;
          }
          if (Vp != nullptr) {
            T* vp = Vp + (int64_t)l * p;
            T* vq = Vp + (int64_t)l * q;
            for (int i = sub; i < l; i += g) {
              const T u = vp[i], w = vq[i];
              vp[i] = cs * u - sn * w;
              vq[i] = sn * u + cs * w;
            }
          }
          rotated = 1;
        }
        if (nwj > 1) asm volatile("bar.sync 1, %0;" :: "r"(nthr) : "memory");
        else __syncwarp();
      }
      // the other sweep's flag is free once every Jacobi thread has passed
      // this sweep's first round (all have read it by then)
      if (rd == 0 && threadIdx.x == 0) jflag[fb ^ 1] = 0;
    }
    if (__any_sync(0xffffffffu, rotated) && lane == 0) jflag[fb] = 1;
    if (nwj > 1) asm volatile("bar.sync 1, %0;" :: "r"(nthr) : "memory");
    else __syncwarp();
    if (!jflag[fb]) break;
  }
}

// sg[c] = ||J(:, c)||; perm = indices sorted by descending sg (lower index
// first on ties).
// The accumulated rotations Vp drift from unit column norms by a few
// roundings per rotation; their columns are renormalised here.
template <typename T>
__device__ void sigma_perm(const T* J, int l, T* sg, int* perm, T* Vp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < l; c += nw) {
    const T* x = J + (int64_t)l * c;
    T s = 0;
    for (int i = lane; i < l; i += 32) s += x[i] * x[i];
    s = warp_sum(s);
    if (lane == 0) sg[c] = sqrt(s);
    T* v = Vp + (int64_t)l * c;
    T t = 0;
    for (int i = lane; i < l; i += 32) t += v[i] * v[i];
    t = warp_sum(t);
    const T inv = t > (T)0 ? (T)1 / sqrt(t) : (T)1;
    __syncwarp();
    for (int i = lane; i < l; i += 32) v[i] *= inv;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const T si = sg[i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      const T sj = sg[j];
      if (sj > si || (sj == si && j < i)) ++rank;
    }
    perm[rank] = i;
  }
  __syncthreads();
}

__device__ __forceinline__ void shift_update(double sl, int rule, double* alpha,
                                             double* alpha_hist, double* sigl_hist) {
  const double a0 = alpha[0];
  double an;
  if (rule == (int)TK_SHIFT_NONE) an = 0.0;
  else an = (sl > a0) ? 0.5 * (sl + a0) : a0;
  alpha[0] = an;
  if (alpha_hist) alpha_hist[0] = an;
  if (sigl_hist) sigl_hist[0] = sl;
}

// ---------------------------------------------------------------------------
// Single-CTA path: Y (n x l) fits in shared memory.
// smem: A (n*l) | J (l*l) | Vp (l*l) | sg (l) | tau (l) [| B (n*l)]
// With room for B, Q = H_0 ... H_{l-1} [U_R; 0] is formed by applying the
// reflectors to U_R directly (no separate Q_h and product).
// ---------------------------------------------------------------------------
constexpr size_t kSvdSmemBudget = 200 * 1024;

__host__ __device__ __forceinline__ bool svd_fused_fits(int64_t n, int l, size_t es) {
  return (2 * (size_t)n * l + 2 * (size_t)l * l + 2 * (size_t)l) * es <= kSvdSmemBudget;
}
template <typename T>
__device__ __forceinline__ void svd_one_body(const double* __restrict__ Y, int n, int l,
                                             double* __restrict__ Q, double* __restrict__ sigma,
                                             int shift_rule, int update_shift, int basis_only,
                                             double* __restrict__ alpha,
                                             double* __restrict__ alpha_hist,
                                             double* __restrict__ sigl_hist,
                                             int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* J = A + (int64_t)n * l;
  T* Vp = J + l * l;
  T* sg = Vp + l * l;
  T* ts = sg + l;
  __shared__ int perm[TK_MAX_L];
  __shared__ double wmax[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // scale Y to max |entry| = 1 so plain sums of squares cannot under/overflow
  // (one pass over global memory, the scaling in shared memory)
  T mx = 0;
#pragma unroll 4
  for (int64_t e = tid; e < (int64_t)n * l; e += blockDim.x) {
    const T v = (T)Y[e];
    A[e] = v;
    mx = max(mx, (T)fabs(v));
  }
  mx = warp_max(mx);
  if (lane == 0) wmax[warp] = (double)mx;
  __syncthreads();
  double gmax = 0.0;
  for (int w = 0; w < nw; ++w) gmax = fmax(gmax, wmax[w]);
  const double scale = (gmax > 0.0 && isfinite(gmax)) ? 1.0 / gmax : 1.0;
  const T sc = (T)scale;
  for (int64_t e = tid; e < (int64_t)n * l; e += blockDim.x) A[e] *= sc;
  __syncthreads();
  householder_qr_la(A, n, l, ts);
  if (basis_only) {
    // only span(Y) is needed: Q = Q_h
    form_q_inplace(A, n, l, ts);
    for (int64_t e = tid; e < (int64_t)n * l; e += blockDim.x) Q[e] = (double)A[e];
    return;
  }
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    J[e] = (c <= i) ? A[c + (int64_t)n * i] : (T)0;   // J = R^T
    Vp[e] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();
  jacobi_warp(J, Vp, l);
  __syncthreads();
  sigma_perm(J, l, sg, perm, Vp);
  if (svd_fused_fits(n, l, sizeof(T))) {
    T* Bm = ts + l;
    // B = [U_R; 0] with U_R = Vp in perm order
    for (int64_t e = tid; e < (int64_t)n * l; e += blockDim.x) {
      const int i = (int)(e % n), c = (int)(e / n);
      Bm[e] = i < l ? Vp[i + (int64_t)l * perm[c]] : (T)0;
    }
    __syncthreads();
    // B <- H_0 H_1 ... H_{l-1} B (H_{l-1} first); H_j = I - tau_j v_j v_j^T,
    // v_j = (0..0, 1, A[j+1:, j])
    for (int j = l - 1; j >= 0; --j) {
      const T tj = ts[j];
      const T* v = A + (int64_t)n * j;
      if (tj != (T)0) {
        for (int c = warp; c < l; c += nw) {
          T* y = Bm + (int64_t)n * c;
          T w = lane == 0 ? y[j] : (T)0;
          for (int i = j + 1 + lane; i < n; i += 32) w += v[i] * y[i];
          w = warp_sum(w) * tj;
          if (lane == 0) y[j] -= w;
          for (int i = j + 1 + lane; i < n; i += 32) y[i] -= w * v[i];
        }
      }
      __syncthreads();
    }
    // sign convention (entry of largest magnitude positive, lowest row on
    // ties), one warp per column, then the FP64 store
    for (int c = warp; c < l; c += nw) {
      const T* y = Bm + (int64_t)n * c;
      T best = (T)-1;
      int bi = 0;
      for (int i = lane; i < n; i += 32) {
        const T av = (T)fabs(y[i]);
        if (av > best) { best = av; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      const T sgn = y[bi] < (T)0 ? (T)-1 : (T)1;
      for (int i = lane; i < n; i += 32) Q[i + (int64_t)n * c] = (double)(sgn * y[i]);
    }
  } else {
  form_q_inplace(A, n, l, ts);
  // Q = Q_h U_R (U_R = Vp with columns in perm order), one warp per column:
  // a first pass finds the entry of largest magnitude (lowest row on ties),
  // the second recomputes the column and stores it with that entry positive
  for (int c = warp; c < l; c += nw) {
    const T* u = Vp + (int64_t)l * perm[c];
    T best = (T)-1;
    int bi = 0;
    for (int i = lane; i < n; i += 32) {
      T s = 0;
      for (int k = 0; k < l; ++k) s += A[i + (int64_t)n * k] * u[k];
      const T av = (T)fabs(s);
      if (av > best) { best = av; bi = i; }
    }
    T bval = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      T s = 0;
      for (int k = 0; k < l; ++k) s += A[bi + (int64_t)n * k] * u[k];
      bval = s;
    }
    bval = __shfl_sync(0xffffffffu, bval, 0);
    const T sgn = bval < (T)0 ? (T)-1 : (T)1;
    for (int i = lane; i < n; i += 32) {
      T s = 0;
      for (int k = 0; k < l; ++k) s += A[i + (int64_t)n * k] * u[k];
      Q[i + (int64_t)n * c] = (double)(sgn * s);
    }
  }
  }
  if (tid < l) {
    const double sv = (double)sg[perm[tid]] / scale;
    sigma[tid] = sv;
    if (!isfinite(sv)) atomicExch(status, (int)TK_EBREAKDOWN);
  }
  if (tid == 0 && update_shift)
    shift_update((double)sg[perm[l - 1]] / scale, shift_rule, alpha, alpha_hist, sigl_hist);
}

template <typename T>
__global__ void k_svd_one(const double* __restrict__ Y, int n, int l, double* __restrict__ Q,
                          double* __restrict__ sigma, int shift_rule, int update_shift,
                          int basis_only, double* __restrict__ alpha,
                          double* __restrict__ alpha_hist, double* __restrict__ sigl_hist,
                          int* __restrict__ status) {
  svd_one_body<T>(Y, n, l, Q, sigma, shift_rule, update_shift, basis_only, alpha, alpha_hist,
                  sigl_hist, status);
}

// ---------------------------------------------------------------------------
// Two-level TSQR path.
// ---------------------------------------------------------------------------
// Each kernel of the chain is a body taking its block coordinates, called by
// the single-problem kernel with blockIdx and by the work-list kernel with
// the job's own block number, so both do the same work per block.
template <typename T>
__device__ __forceinline__ void leaf_qr_body(const double* __restrict__ Y, int64_t n, int l,
                                             int MB, int Pb, T* __restrict__ V,
                                             T* __restrict__ tau, T* __restrict__ Rst, int b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* ts = A + (int64_t)MB * l;
  const int64_t r0 = (int64_t)b * MB;
  const int64_t rows = min((int64_t)MB, n - r0);
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) {
    const int64_t i = e % MB, c = e / MB;
    A[e] = i < rows ? (T)Y[(r0 + i) + n * c] : (T)0;
  }
  __syncthreads();
  householder_qr(A, MB, l, ts);
  T* Vb = V + (int64_t)b * MB * l;
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) Vb[e] = A[e];
  const int64_t ldr = (int64_t)Pb * l;
  for (int64_t e = threadIdx.x; e < (int64_t)l * l; e += blockDim.x) {
    const int i = (int)(e % l), c = (int)(e / l);
    Rst[((int64_t)b * l + i) + ldr * c] = (i <= c && i < MB) ? A[i + (int64_t)MB * c] : (T)0;
  }
  for (int j = threadIdx.x; j < l; j += blockDim.x) tau[(int64_t)b * l + j] = ts[j];
}

template <typename T>
__global__ void k_leaf_qr(const double* __restrict__ Y, int64_t n, int l, int MB, int Pb,
                          T* __restrict__ V, T* __restrict__ tau, T* __restrict__ Rst) {
  leaf_qr_body<T>(Y, n, l, MB, Pb, V, tau, Rst, blockIdx.x);
}

// smem: S (m*l) | J (l*l) | Vp (l*l) | sg (l) | tau (l), m = Pb*l
template <typename T>
__device__ __forceinline__ void root_body(const T* __restrict__ Rst, int Pb, int l,
                                          T* __restrict__ Mout, double* __restrict__ sigma,
                                          int shift_rule, int update_shift,
                                          double* __restrict__ alpha,
                                          double* __restrict__ alpha_hist,
                                          double* __restrict__ sigl_hist,
                                          int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = Pb * l;
  T* S = reinterpret_cast<T*>(smem_raw);
  T* J = S + (int64_t)m * l;
  T* Vp = J + (int64_t)l * l;
  T* sg = Vp + (int64_t)l * l;
  T* ts = sg + l;
  __shared__ int perm[TK_MAX_L];
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)m * l; e += blockDim.x) S[e] = Rst[e];
  __syncthreads();
  householder_qr(S, m, l, ts);
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    J[e] = (c <= i) ? S[c + (int64_t)m * i] : (T)0;
    Vp[e] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();
  jacobi_warp(J, Vp, l);
  __syncthreads();
  sigma_perm(J, l, sg, perm, Vp);
  form_q_inplace(S, m, l, ts);
  for (int i = tid; i < m; i += blockDim.x) {
    for (int c = 0; c < l; ++c) {
      const T* u = Vp + (int64_t)l * perm[c];
      T s = 0;
      for (int k = 0; k < l; ++k) s += S[i + (int64_t)m * k] * u[k];
      Mout[i + (int64_t)m * c] = s;
    }
  }
  if (tid < l) {
    const double sv = (double)sg[perm[tid]];
    sigma[tid] = sv;
    if (!isfinite(sv)) atomicExch(status, (int)TK_EBREAKDOWN);
  }
  if (tid == 0 && update_shift)
    shift_update((double)sg[perm[l - 1]], shift_rule, alpha, alpha_hist, sigl_hist);
}

template <typename T>
__global__ void k_root(const T* __restrict__ Rst, int Pb, int l, T* __restrict__ Mout,
                       double* __restrict__ sigma, int shift_rule, int update_shift,
                       double* __restrict__ alpha, double* __restrict__ alpha_hist,
                       double* __restrict__ sigl_hist, int* __restrict__ status) {
  root_body<T>(Rst, Pb, l, Mout, sigma, shift_rule, update_shift, alpha, alpha_hist, sigl_hist,
               status);
}

// smem: B (MB*l) block reflectors -> block Q | M (l*l) | tau (l)
template <typename T>
__device__ __forceinline__ void leaf_q_body(const T* __restrict__ V, const T* __restrict__ tau,
                                            const T* __restrict__ Mout, int64_t n, int l, int MB,
                                            int Pb, double* __restrict__ Q,
                                            double* __restrict__ colmax,
                                            int* __restrict__ colidx, int b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* B = reinterpret_cast<T*>(smem_raw);
  T* M = B + (int64_t)MB * l;
  T* ts = M + (int64_t)l * l;
  const int m = Pb * l;
  const int64_t r0 = (int64_t)b * MB;
  const int64_t rows = min((int64_t)MB, n - r0);
  const T* Vb = V + (int64_t)b * MB * l;
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) B[e] = Vb[e];
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    M[e] = Mout[((int64_t)b * l + i) + (int64_t)m * c];
  }
  for (int j = threadIdx.x; j < l; j += blockDim.x) ts[j] = tau[(int64_t)b * l + j];
  __syncthreads();
  form_q_inplace(B, MB, l, ts);
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    for (int c = 0; c < l; ++c) {
      const T* u = M + (int64_t)l * c;
      T s = 0;
      for (int k = 0; k < l; ++k) s += B[i + (int64_t)MB * k] * u[k];
      Q[(r0 + i) + n * c] = (double)s;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < l; c += nw) {
    double best = -1.0;
    int bi = 0;                      // a valid row even if every entry is NaN
    for (int i = lane; i < rows; i += 32) {
      const double v = fabs(Q[(r0 + i) + n * c]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      colmax[(int64_t)b * l + c] = best;
      colidx[(int64_t)b * l + c] = (int)(r0 + bi);
    }
  }
}

template <typename T>
__global__ void k_leaf_q(const T* __restrict__ V, const T* __restrict__ tau,
                         const T* __restrict__ Mout, int64_t n, int l, int MB, int Pb,
                         double* __restrict__ Q, double* __restrict__ colmax,
                         int* __restrict__ colidx) {
  leaf_q_body<T>(V, tau, Mout, n, l, MB, Pb, Q, colmax, colidx, blockIdx.x);
}

// column c of Q takes the sign that makes its largest entry (over all leaves)
// positive
__device__ __forceinline__ void sign_body(double* __restrict__ Q, int64_t n, int l, int Pb,
                                          const double* __restrict__ colmax,
                                          const int* __restrict__ colidx, int c) {
  __shared__ double sgn;
  if (threadIdx.x == 0) {
    double best = -1.0;
    int idx = 0;
    for (int b = 0; b < Pb; ++b) {
      const double v = colmax[(int64_t)b * l + c];
      if (v > best) { best = v; idx = colidx[(int64_t)b * l + c]; }
    }
    sgn = (idx >= 0 && idx < n && Q[(int64_t)idx + n * c] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn < 0.0)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Q[i + n * c] = -Q[i + n * c];
}

__global__ void k_sign(double* __restrict__ Q, int64_t n, int l, int Pb,
                       const double* __restrict__ colmax, const int* __restrict__ colidx) {
  sign_body(Q, n, l, Pb, colmax, colidx, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Re-orthonormalisation of a factor computed in FP32 arithmetic (FP64
// storage): one CholeskyQR step U <- U R^{-1}, R^T R = G = U^T U, taken to
// first order.  U is orthonormal to FP32 rounding, so G = I + E with
// |E| ~ 1e-6; R = I + F + O(|E|^2) with F the upper triangle of E (diagonal
// halved) and R^{-1} = I - F + O(|E|^2).  The O(1e-12) remainder is far
// below the FP32 rounding of the returned factor, and the correction U F
// (itself ~1e-6 |U|) needs only FP32 arithmetic; G and the update are FP64.
// ---------------------------------------------------------------------------
constexpr int kPolishRows = 64;

__device__ __forceinline__ void gram_part_body(const double* __restrict__ U, int64_t n, int r,
                                               double* __restrict__ part, unsigned bx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ub = reinterpret_cast<double*>(smem_raw);     // kPolishRows x r
  const int b = (int)bx;
  const int64_t r0 = (int64_t)b * kPolishRows;
  const int rows = (int)min((int64_t)kPolishRows, n - r0);
  for (int e = threadIdx.x; e < kPolishRows * r; e += blockDim.x) {
    const int i = e % kPolishRows, c = e / kPolishRows;
    Ub[e] = i < rows ? U[(r0 + i) + n * c] : 0.0;
  }
  __syncthreads();
  double* G = part + (int64_t)b * r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double s = 0.0;
    for (int t = 0; t < rows; ++t) s += Ub[t + kPolishRows * i] * Ub[t + kPolishRows * j];
    G[e] = s;
  }
}

__global__ void k_gram_part(const double* __restrict__ U, int64_t n, int r,
                            double* __restrict__ part) {
  gram_part_body(U, n, r, part, blockIdx.x);
}

// smem: F (r*r, FP32) | block rows (kPolishRows*r, FP64)
__device__ __forceinline__ void polish_body(double* __restrict__ U, int64_t n, int r, int nblk,
                                            const double* __restrict__ part,
                                            int* __restrict__ status, unsigned bx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* F = reinterpret_cast<float*>(smem_raw);
  double* Ub = reinterpret_cast<double*>(smem_raw + (((size_t)r * r * sizeof(float) + 15) & ~(size_t)15));
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)bx * kPolishRows;
  const int rows = (int)min((int64_t)kPolishRows, n - r0);
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    double g = 0.0;
    for (int b = 0; b < nblk; ++b) g += part[(int64_t)b * r * r + e];
    const int i = e % r, c = e / r;
    const double dev = g - (i == c ? 1.0 : 0.0);
    // a factor this far from orthonormal is not a rounding-level correction
    if (!(fabs(dev) <= 0.25)) bad = 1;
    F[e] = i < c ? (float)dev : (i == c ? (float)(0.5 * dev) : 0.f);
  }
  for (int e = tid; e < kPolishRows * r; e += blockDim.x) {
    const int i = e % kPolishRows, c = e / kPolishRows;
    Ub[e] = i < rows ? U[(r0 + i) + n * c] : 0.0;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0 && bx == 0) atomicExch(status, (int)TK_EBREAKDOWN);
    return;
  }
  // u(c) <- u(c) - sum_{k <= c} u(k) F(k, c)
  for (int e = tid; e < kPolishRows * r; e += blockDim.x) {
    const int i = e % kPolishRows, c = e / kPolishRows;
    if (i >= rows) continue;
    float s = 0.f;
    for (int k = 0; k <= c; ++k) s = fmaf((float)Ub[i + kPolishRows * k], F[k + r * c], s);
    U[(r0 + i) + n * c] = Ub[e] - (double)s;
  }
}

__global__ void k_polish(double* __restrict__ U, int64_t n, int r, int nblk,
                         const double* __restrict__ part, int* __restrict__ status) {
  polish_body(U, n, r, nblk, part, status, blockIdx.x);
}

size_t polish_scratch(int64_t n, int r) {
  return (size_t)((n + kPolishRows - 1) / kPolishRows) * r * r * sizeof(double);
}

cudaError_t launch_polish(double* U, int64_t n, int r, void* scratch, int* status,
                          cudaStream_t st) {
  if (n <= 0 || r <= 0) return cudaSuccess;
  const int nblk = (int)((n + kPolishRows - 1) / kPolishRows);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gram_part, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_polish, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_kernels(2);
  k_gram_part<<<nblk, 256, (size_t)kPolishRows * r * sizeof(double), st>>>(U, n, r,
                                                                           (double*)scratch);
  k_polish<<<nblk, 256, polish_smem(r), st>>>(
      U, n, r, nblk, (const double*)scratch, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Register-resident FP32 path: 512 threads (16 warps); warp w keeps columns
// c = w + 16 s (s < 4) of an m x l matrix (m <= 512, l <= 64) in registers,
// lane holding rows 4 (lane + 32 k) + e (k < 4, e < 4).  A Householder step
// streams only the reflector through shared memory and takes one barrier;
// applying the reflectors backward (Q = H_0 ... H_{l-1} B) needs none.  The
// l x l problem uses one-sided Jacobi with one warp per pair and column norms
// kept incrementally (a' = a - t g, b' = b + t g; refreshed every sweep).
// Same arithmetic as the shared-memory routines, in a different order.
// ---------------------------------------------------------------------------
constexpr int kRegThreads = 512;
constexpr int kRegRK = 4;                    // float4 chunks per lane per column
constexpr int kRegCPW = 4;                   // columns per warp
constexpr int kRegRows = 4 * 32 * kRegRK;    // 512
constexpr int kRegCols = 16 * kRegCPW;       // 64
// Long-mode variant: eight float4 chunks per lane (1024 rows) with two
// column slots per warp (l <= 32): the same 64 register floats per thread.
constexpr int kRegRK2 = 8;
constexpr int kRegRows2 = 4 * 32 * kRegRK2;  // 1024
constexpr int kRegCols2 = 32;

__host__ __device__ __forceinline__ int reg_ld(int64_t m) { return (int)((m + 3) / 4 * 4); }

template <int CPW, int RK = kRegRK>
struct RegCols {
  float y[CPW][4 * RK];
  int lane, warp;
  __device__ __forceinline__ RegCols() : lane(threadIdx.x & 31), warp(threadIdx.x >> 5) {}
  __device__ __forceinline__ int col(int s) const { return warp + 16 * s; }
  __device__ __forceinline__ int row(int k, int e) const { return 4 * (lane + 32 * k) + e; }
  __device__ __forceinline__ bool has(int k, int md) const { return 4 * (lane + 32 * k) < md; }

  __device__ __forceinline__ void load_col(int s, const float* c, int md) {
#pragma unroll
    for (int k = 0; k < RK; ++k) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (has(k, md)) v = *reinterpret_cast<const float4*>(c + 4 * (lane + 32 * k));
      y[s][4 * k] = v.x; y[s][4 * k + 1] = v.y; y[s][4 * k + 2] = v.z; y[s][4 * k + 3] = v.w;
    }
  }
  __device__ __forceinline__ void store_col(int s, float* c, int md) const {
#pragma unroll
    for (int k = 0; k < RK; ++k)
      if (has(k, md))
        *reinterpret_cast<float4*>(c + 4 * (lane + 32 * k)) =
            make_float4(y[s][4 * k], y[s][4 * k + 1], y[s][4 * k + 2], y[s][4 * k + 3]);
  }
  // y(:, c) <- (I - tj v v^T) y(:, c) for the owned columns lo < c < hi;
  // v = reflector j in shared memory, stored in full (0 above row j, 1 at j)
  __device__ __forceinline__ void apply(const float* v, int md, float tj, int lo, int hi) {
    bool act[CPW];
    bool any = false;
#pragma unroll
    for (int s = 0; s < CPW; ++s) {
      act[s] = col(s) > lo && col(s) < hi;
      any = any || act[s];
    }
    if (!any || tj == 0.f) return;
    float d[CPW];
#pragma unroll
    for (int s = 0; s < CPW; ++s) d[s] = 0.f;
#pragma unroll
    for (int k = 0; k < RK; ++k) {
      if (!has(k, md)) continue;
      const float4 v4 = *reinterpret_cast<const float4*>(v + 4 * (lane + 32 * k));
      const float ve[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int s = 0; s < CPW; ++s)
          if (act[s]) d[s] = fmaf(ve[e], y[s][4 * k + e], d[s]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int s = 0; s < CPW; ++s) d[s] += __shfl_xor_sync(0xffffffffu, d[s], o);
#pragma unroll
    for (int s = 0; s < CPW; ++s) d[s] *= -tj;
#pragma unroll
    for (int k = 0; k < RK; ++k) {
      if (!has(k, md)) continue;
      const float4 v4 = *reinterpret_cast<const float4*>(v + 4 * (lane + 32 * k));
      const float ve[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int s = 0; s < CPW; ++s)
          if (act[s]) y[s][4 * k + e] = fmaf(d[s], ve[e], y[s][4 * k + e]);
    }
  }
  // reflector of column c (held in y[s]) as make_reflector builds it: R(r, c)
  // (r <= c) goes to rs[r * rr + c * rc] (when rs is given), the column is
  // stored as the full reflector (0 above row c, 1 at c, v below), tau[c]
  __device__ __forceinline__ void build(int s, int c, float* cp, int md, float* tau, float* rs,
                                        int rr, int rc) {
    float s0 = 0.f, s1 = 0.f, mine = 0.f;
#pragma unroll
    for (int k = 0; k < RK; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row(k, e);
        const float t = r > c ? y[s][4 * k + e] : 0.f;
        if (e & 1) s1 = fmaf(t, t, s1); else s0 = fmaf(t, t, s0);
        if (r == c) mine = y[s][4 * k + e];
      }
    const float ssq = warp_sum(s0 + s1);
    const float alpha = __shfl_sync(0xffffffffu, mine, (c >> 2) & 31);
    // the fast reciprocal square root and division intrinsics (a few ulp;
    // the correctly rounded forms cost ~5x their latency on the step's
    // critical path) -- the reflector stays orthogonal to FP32 rounding
    const float xnorm = ssq > 0.f ? ssq * rsqrtf(ssq) : 0.f;
    float beta = alpha, tj = 0.f, scal = 1.f;
    if (xnorm > 0.f) {
      const float mx = fmaxf(fabsf(alpha), xnorm);
      const float rmx = __fdividef(1.f, mx);
      const float a1 = alpha * rmx, x1 = xnorm * rmx;
      const float h = a1 * a1 + x1 * x1;   // in [1, 2]
      beta = -copysignf(mx * (h * rsqrtf(h)), alpha);
      tj = __fdividef(beta - alpha, beta);
      scal = __fdividef(1.f, alpha - beta);
    }
#pragma unroll
    for (int k = 0; k < RK; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row(k, e);
        float& x = y[s][4 * k + e];
        if (rs != nullptr && r <= c) rs[r * rr + c * rc] = r == c ? beta : x;
        x = r > c ? x * scal : (r == c ? 1.f : 0.f);
      }
    store_col(s, cp, md);
    if (lane == 0) tau[c] = tj;
  }
  // Householder QR of A (md x l in shared memory, ld md, rows past m zero)
  // with the columns in registers.  A ends holding the full reflectors
  // (column j: 0 above row j, 1 at j, v_j below), tau the factors, and R
  // (upper triangle) goes to rs[r * rr + c * rc] when rs is given.
  __device__ void qr(float* A, int md, int l, float* tau, float* rs, int rr, int rc) {
#pragma unroll
    for (int s = 0; s < CPW; ++s)
      if (col(s) < l) load_col(s, A + (int64_t)md * col(s), md);
    if (warp == 0) build(0, 0, A, md, tau, rs, rr, rc);
    __syncthreads();
    for (int j = 0; j < l; ++j) {
      const float tj = tau[j];
      const float* v = A + (int64_t)md * j;
      // the owner of column j+1 updates and factors it first (look-ahead)
#pragma unroll
      for (int s = 0; s < CPW; ++s)
        if (col(s) == j + 1 && j + 1 < l) {
          apply(v, md, tj, j, j + 2);
          build(s, j + 1, A + (int64_t)md * (j + 1), md, tau, rs, rr, rc);
        }
      apply(v, md, tj, j + 1, l);
      __syncthreads();
    }
  }
  // y(:, c) <- H_0 H_1 ... H_{l-1} y(:, c) for the owned columns c < nb
  // (full reflectors and tau of qr() in shared memory, read only)
  // (columns lo < c < nb only when lo >= 0)
  __device__ void apply_back(const float* A, int md, int l, const float* tau, int nb,
                             int lo = -1) {
    for (int j = l - 1; j >= 0; --j) apply(A + (int64_t)md * j, md, tau[j], lo, nb);
  }
  // y(:, c) = B(r, c) for r < l (B(r, c) = src[r + ld c'] with c' = perm[c]
  // when perm is given), 0 below
  __device__ __forceinline__ void init_top(const float* src, int ld, const int* perm, int l,
                                           int nb) {
#pragma unroll
    for (int s = 0; s < CPW; ++s) {
      const int c = col(s);
      const int cs = c < nb ? (perm ? perm[c] : c) : 0;
#pragma unroll
      for (int k = 0; k < RK; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = row(k, e);
          y[s][4 * k + e] = (c < nb && r < l) ? src[r + (int64_t)ld * cs] : 0.f;
        }
    }
  }
  // column c's entry of largest magnitude (lowest row on ties, rows < m):
  // its value, broadcast to the warp
  __device__ __forceinline__ float col_extreme(int s, int m, int* brow) const {
    float best = -1.f, bval = 0.f;
    int bi = 0;
#pragma unroll
    for (int k = 0; k < RK; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row(k, e);
        const float av = fabsf(y[s][4 * k + e]);
        if (r < m && av > best) { best = av; bi = r; bval = y[s][4 * k + e]; }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const float ov = __shfl_xor_sync(0xffffffffu, bval, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bval = ov; }
    }
    if (brow) *brow = bi;
    return bval;
  }
  // out[r + ldo c] = sgn y(r, c) for r < m (c < nb)
  template <typename O>
  __device__ __forceinline__ void store_out(int s, O* out, int64_t ldo, int m, float sgn) const {
#pragma unroll
    for (int k = 0; k < RK; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row(k, e);
        if (r < m) out[r + ldo * col(s)] = (O)(sgn * y[s][4 * k + e]);
      }
  }
};

// One-sided Jacobi on the l columns of J (l x l, l <= 128), accumulating the
// rotations in Vp; G lanes per column pair of a round-robin round (G = 16:
// two pairs per warp, l <= 64; G = 32: l <= 128), each lane holding 4
// entries of the pair's columns; column norms in nrm (l) kept incrementally;
// all threads of the block take part.
template <int G>
__device__ void jacobi_pairs_g(float* J, float* Vp, int l, float* nrm) {
  constexpr int PPW = 32 / G;   // pairs per warp and pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int hw = lane / G, sub = lane % G;
  const int m2 = l + (l & 1), npairs = m2 / 2;
  __shared__ int jflag[2];
  if (threadIdx.x == 0) jflag[0] = jflag[1] = 0;
  const float tol = jacobi_tol<float>(l);
  const float tol2 = tol * tol;
  for (int sweep = 0; sweep < 24; ++sweep) {
    for (int c = warp; c < l; c += nw) {
      const float* x = J + l * c;
      float a = 0.f;
      for (int i = lane; i < l; i += 32) a = fmaf(x[i], x[i], a);
      a = warp_sum(a);
      if (lane == 0) nrm[c] = a;
    }
    __syncthreads();
    const int fb = sweep & 1;
    int rotated = 0;
    for (int rd = 0; rd < m2 - 1; ++rd) {
      // uniform per warp: both halves iterate together (the shuffles need
      // every lane)
      for (int pr0 = PPW * warp; pr0 < npairs; pr0 += PPW * nw) {
        const int pr = pr0 + hw;
        int p = 0, q = 0;
        if (pr < npairs) {
          if (pr == 0) {
            p = rd;
            q = m2 - 1;
          } else {
            p = rd + pr;
            if (p >= m2 - 1) p -= m2 - 1;
            q = rd - pr;
            if (q < 0) q += m2 - 1;
          }
        }
        const bool act = pr < npairs && p < l && q < l;
        float* xp = J + l * p;
        float* xq = J + l * q;
        float u[4], w[4], g = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = sub + G * k;
          u[k] = (act && i < l) ? xp[i] : 0.f;
          w[k] = (act && i < l) ? xq[i] : 0.f;
          g = fmaf(u[k], w[k], g);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        const float a = act ? nrm[p] : 0.f, b = act ? nrm[q] : 0.f;
        if (act && g != 0.f && g * g > tol2 * a * b) {
          // rotation parameters with the fast intrinsics: any angle close to
          // the Jacobi angle is an exact plane rotation (cs, sn from t)
          const float zeta = __fdividef(b - a, g + g);
          float t;
          if (fabsf(zeta) > 1e15f) {
            t = __fdividef(0.5f, zeta);
          } else {
            const float h = 1.f + zeta * zeta;
            t = copysignf(__fdividef(1.f, fabsf(zeta) + h * rsqrtf(h)), zeta);
          }
          const float cs = rsqrtf(1.f + t * t);
          const float sn = cs * t;
          float* vp = Vp + l * p;
          float* vq = Vp + l * q;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = sub + G * k;
            if (i < l) {
              xp[i] = cs * u[k] - sn * w[k];
              xq[i] = sn * u[k] + cs * w[k];
              const float a1 = vp[i], b1 = vq[i];
              vp[i] = cs * a1 - sn * b1;
              vq[i] = sn * a1 + cs * b1;
            }
          }
          if (sub == 0) {
            nrm[p] = a - t * g;
            nrm[q] = b + t * g;
          }
          rotated = 1;
        }
      }
      // the other sweep's flag is free once every thread has passed this
      // sweep's first round
      if (rd == 0 && threadIdx.x == 0) jflag[fb ^ 1] = 0;
      __syncthreads();
    }
    if (rotated) jflag[fb] = 1;
    __syncthreads();
    if (!jflag[fb]) break;
  }
}

__device__ __forceinline__ void jacobi_pairs(float* J, float* Vp, int l, float* nrm) {
  if (l <= 64) jacobi_pairs_g<16>(J, Vp, l, nrm);
  else jacobi_pairs_g<32>(J, Vp, l, nrm);
}

// smem: A (md*l) | J (l*l) | Vp (l*l) | sg (l) | ts (l) | nrm (l), FP32
__host__ __device__ __forceinline__ size_t reg_one_smem(int64_t n, int l) {
  return ((size_t)reg_ld(n) * l + 2 * (size_t)l * l + 3 * (size_t)l) * sizeof(float);
}

// [Q, Sigma] = svd(Y) for n <= 128 RK, l <= 16 CPW (FP32 working precision), or
// with basis_only an orthonormal basis of span(Y); as svd_one_body.
template <int CPW, int RK = kRegRK>
__device__ __forceinline__ void svd_reg_body(const double* __restrict__ Y, int n, int l,
                                             double* __restrict__ Q, double* __restrict__ sigma,
                                             int shift_rule, int update_shift, int basis_only,
                                             double* __restrict__ alpha,
                                             double* __restrict__ alpha_hist,
                                             double* __restrict__ sigl_hist,
                                             int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int md = reg_ld(n);
  float* A = reinterpret_cast<float*>(smem_raw);
  float* J = A + (int64_t)md * l;
  float* Vp = J + l * l;
  float* sg = Vp + l * l;
  float* ts = sg + l;
  float* nrm = ts + l;
  __shared__ int perm[TK_MAX_L];
  __shared__ double wmax[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // scale Y to max |entry| = 1 (sums of squares cannot under/overflow)
  float mx = 0.f;
  for (int64_t e = tid; e < (int64_t)md * l; e += blockDim.x) {
    const int i = (int)(e % md), c = (int)(e / md);
    const float v = i < n ? (float)Y[i + (int64_t)n * c] : 0.f;
    A[e] = v;
    mx = fmaxf(mx, fabsf(v));
  }
  mx = warp_max(mx);
  if (lane == 0) wmax[warp] = (double)mx;
  __syncthreads();
  double gmax = 0.0;
  for (int w = 0; w < nw; ++w) gmax = fmax(gmax, wmax[w]);
  const double scale = (gmax > 0.0 && isfinite(gmax)) ? 1.0 / gmax : 1.0;
  const float sc = (float)scale;
  for (int64_t e = tid; e < (int64_t)md * l; e += blockDim.x) A[e] *= sc;
  __syncthreads();
  if (!basis_only)
    for (int e = tid; e < l * l; e += blockDim.x) J[e] = 0.f;
  __syncthreads();
  RegCols<CPW, RK> R;
  R.qr(A, md, l, ts, basis_only ? nullptr : J, l, 1);   // J = R^T
  if (basis_only) {
    // only span(Y) is needed: Q = Q_h
    for (int e = tid; e < l * l; e += blockDim.x) Vp[e] = (e % l == e / l) ? 1.f : 0.f;
    __syncthreads();
    R.init_top(Vp, l, nullptr, l, l);
    R.apply_back(A, md, l, ts, l);
#pragma unroll
    for (int s = 0; s < CPW; ++s)
      if (R.col(s) < l) R.store_out(s, Q, n, n, 1.f);
    return;
  }
  for (int e = tid; e < l * l; e += blockDim.x) Vp[e] = (e % l == e / l) ? 1.f : 0.f;
  __syncthreads();
  jacobi_pairs(J, Vp, l, nrm);
  sigma_perm(J, l, sg, perm, Vp);
  // Q = H_0 ... H_{l-1} [U_R; 0], U_R = Vp in perm order; sign convention
  // (entry of largest magnitude positive, lowest row on ties)
  R.init_top(Vp, l, perm, l, l);
  R.apply_back(A, md, l, ts, l);
#pragma unroll
  for (int s = 0; s < CPW; ++s)
    if (R.col(s) < l) {
      const float bv = R.col_extreme(s, n, nullptr);
      R.store_out(s, Q, n, n, bv < 0.f ? -1.f : 1.f);
    }
  if (tid < l) {
    const double sv = (double)sg[perm[tid]] / scale;
    sigma[tid] = sv;
    if (!isfinite(sv)) atomicExch(status, (int)TK_EBREAKDOWN);
  }
  if (tid == 0 && update_shift)
    shift_update((double)sg[perm[l - 1]] / scale, shift_rule, alpha, alpha_hist, sigl_hist);
}

template <int CPW, int RK = kRegRK>
__global__ void __launch_bounds__(kRegThreads)
k_svd_reg(const double* __restrict__ Y, int n, int l, double* __restrict__ Q,
          double* __restrict__ sigma, int shift_rule, int update_shift, int basis_only,
          double* __restrict__ alpha, double* __restrict__ alpha_hist,
          double* __restrict__ sigl_hist, int* __restrict__ status) {
  svd_reg_body<CPW, RK>(Y, n, l, Q, sigma, shift_rule, update_shift, basis_only, alpha,
                        alpha_hist, sigl_hist, status);
}

// TSQR leaf (MB <= 512 rows, a multiple of 32): reflectors to V (ld MB), tau,
// R into the stack Rst (Pb l x l, ld Pb l)
template <int CPW>
__device__ __forceinline__ void leaf_qr_reg_body(const double* __restrict__ Y, int64_t n, int l,
                                                 int MB, int Pb, float* __restrict__ V,
                                                 float* __restrict__ tau,
                                                 float* __restrict__ Rst, int b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* A = reinterpret_cast<float*>(smem_raw);
  float* ts = A + (int64_t)MB * l;
  const int64_t r0 = (int64_t)b * MB;
  const int64_t rows = min((int64_t)MB, n - r0);
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) {
    const int64_t i = e % MB, c = e / MB;
    A[e] = i < rows ? (float)Y[(r0 + i) + n * c] : 0.f;
  }
  __syncthreads();
  const int ldr = Pb * l;
  float* Rb = Rst + (int64_t)b * l;
  // the strictly lower part of this leaf's R block; qr() writes the rest
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    if (i > c) Rb[i + (int64_t)ldr * c] = 0.f;
  }
  RegCols<CPW> R;
  R.qr(A, MB, l, ts, Rb, 1, ldr);
  float* Vb = V + (int64_t)b * MB * l;
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) Vb[e] = A[e];
  for (int j = threadIdx.x; j < l; j += blockDim.x) tau[(int64_t)b * l + j] = ts[j];
}

template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_leaf_qr_reg(const double* __restrict__ Y, int64_t n, int l, int MB, int Pb,
              float* __restrict__ V, float* __restrict__ tau, float* __restrict__ Rst) {
  leaf_qr_reg_body<CPW>(Y, n, l, MB, Pb, V, tau, Rst, blockIdx.x);
}

// TSQR root (m = Pb l <= 512): QR of the stacked R's, svd of the root R, and
// Mout = Q_root U_R (m x l, ld m); sigma and the shift update.  With
// basis_only, Mout = Q_root: an orthonormal basis of the same span (no svd).
// smem: S (md*l) | J (l*l) | Vp (l*l) | sg (l) | ts (l) | nrm (l)
template <int CPW>
__device__ __forceinline__ void root_reg_body(const float* __restrict__ Rst, int Pb, int l,
                                              float* __restrict__ Mout,
                                              double* __restrict__ sigma, int shift_rule,
                                              int update_shift, int basis_only,
                                              double* __restrict__ alpha,
                                              double* __restrict__ alpha_hist,
                                              double* __restrict__ sigl_hist,
                                              int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = Pb * l, md = reg_ld(m);
  float* S = reinterpret_cast<float*>(smem_raw);
  float* J = S + (int64_t)md * l;
  float* Vp = J + l * l;
  float* sg = Vp + l * l;
  float* ts = sg + l;
  float* nrm = ts + l;
  __shared__ int perm[TK_MAX_L];
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)md * l; e += blockDim.x) {
    const int i = (int)(e % md), c = (int)(e / md);
    S[e] = i < m ? Rst[i + (int64_t)m * c] : 0.f;
  }
  for (int e = tid; e < l * l; e += blockDim.x) J[e] = 0.f;
  __syncthreads();
  RegCols<CPW> R;
  R.qr(S, md, l, ts, basis_only ? nullptr : J, l, 1);   // J = R^T
  for (int e = tid; e < l * l; e += blockDim.x) Vp[e] = (e % l == e / l) ? 1.f : 0.f;
  __syncthreads();
  if (basis_only) {
    R.init_top(Vp, l, nullptr, l, l);
    R.apply_back(S, md, l, ts, l);
#pragma unroll
    for (int s = 0; s < CPW; ++s)
      if (R.col(s) < l) R.store_out(s, Mout, m, m, 1.f);
    return;
  }
  jacobi_pairs(J, Vp, l, nrm);
  sigma_perm(J, l, sg, perm, Vp);
  R.init_top(Vp, l, perm, l, l);
  R.apply_back(S, md, l, ts, l);
#pragma unroll
  for (int s = 0; s < CPW; ++s)
    if (R.col(s) < l) R.store_out(s, Mout, m, m, 1.f);
  if (tid < l) {
    const double sv = (double)sg[perm[tid]];
    sigma[tid] = sv;
    if (!isfinite(sv)) atomicExch(status, (int)TK_EBREAKDOWN);
  }
  if (tid == 0 && update_shift)
    shift_update((double)sg[perm[l - 1]], shift_rule, alpha, alpha_hist, sigl_hist);
}

template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_root_reg(const float* __restrict__ Rst, int Pb, int l, float* __restrict__ Mout,
           double* __restrict__ sigma, int shift_rule, int update_shift, int basis_only,
           double* __restrict__ alpha, double* __restrict__ alpha_hist,
           double* __restrict__ sigl_hist, int* __restrict__ status) {
  root_reg_body<CPW>(Rst, Pb, l, Mout, sigma, shift_rule, update_shift, basis_only, alpha,
                     alpha_hist, sigl_hist, status);
}

// TSQR leaf Q: rows r0.. of Q = Q_leaf [M_b; 0] (M_b = rows b l.. of Mout),
// written in FP64, with each column's entry of largest magnitude (and its
// global row) for the sign pass.  The columns are independent: CTA
// (b, blockIdx.y) takes columns 16 y .. 16 y + 15, one per warp, so a leaf's
// columns spread over CPW CTAs.  smem: B (MB*l reflectors) | tau (l)
template <int CPW>
__device__ __forceinline__ void leaf_q_reg_body(const float* __restrict__ V,
                                                const float* __restrict__ tau,
                                                const float* __restrict__ Mout, int64_t n, int l,
                                                int MB, int Pb, double* __restrict__ Q,
                                                double* __restrict__ colmax,
                                                int* __restrict__ colidx, int b, int by) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* B = reinterpret_cast<float*>(smem_raw);
  float* ts = B + (int64_t)MB * l;
  const int m = Pb * l;
  const int64_t r0 = (int64_t)b * MB;
  const int rows = (int)min((int64_t)MB, n - r0);
  const float* Vb = V + (int64_t)b * MB * l;
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) B[e] = Vb[e];
  for (int j = threadIdx.x; j < l; j += blockDim.x) ts[j] = tau[(int64_t)b * l + j];
  __syncthreads();
  const int c_lo = 16 * by, c_hi = min(l, c_lo + 16);
  RegCols<CPW> R;
  R.init_top(Mout + (int64_t)b * l, m, nullptr, l, l);
  R.apply_back(B, MB, l, ts, c_hi, c_lo - 1);
#pragma unroll
  for (int s = 0; s < CPW; ++s)
    if (R.col(s) >= c_lo && R.col(s) < c_hi) {
      int bi = 0;
      const float bv = R.col_extreme(s, rows, &bi);
      R.store_out(s, Q + r0, n, rows, 1.f);
      if (R.lane == 0) {
        colmax[(int64_t)b * l + R.col(s)] = fabs((double)bv);
        colidx[(int64_t)b * l + R.col(s)] = (int)(r0 + bi);
      }
    }
}

template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_leaf_q_reg(const float* __restrict__ V, const float* __restrict__ tau,
             const float* __restrict__ Mout, int64_t n, int l, int MB, int Pb,
             double* __restrict__ Q, double* __restrict__ colmax, int* __restrict__ colidx) {
  leaf_q_reg_body<CPW>(V, tau, Mout, n, l, MB, Pb, Q, colmax, colidx, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
static const size_t kSmemBudget = kSvdSmemBudget;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t one_smem(int64_t n, int l, size_t es) {
  const size_t base = ((size_t)n * l + 2 * (size_t)l * l + 2 * (size_t)l) * es;
  return svd_fused_fits(n, l, es) ? base + (size_t)n * l * es : base;
}
static size_t root_smem(int Pb, int l, size_t es) {
  return ((size_t)Pb * l * l + 2 * (size_t)l * l + 2 * (size_t)l) * es;
}
static size_t leafq_smem(int MB, int l, size_t es) {
  return ((size_t)MB * l + (size_t)l * l + (size_t)l) * es;
}

// Pb == 1 selects the single-CTA path (MB = n).  FP32 problems with n <= 512
// and l <= 64, or n <= 1024 and l <= 32, take the register-resident
// single-CTA kernel; above the
// single-CTA shared-memory budget, FP32 TSQR takes the register-resident
// kernels when the leaves (<= 512 rows) and the root (Pb l <= 512 rows) fit.
// (The work-list svd follows the same single-CTA choice, so batched and
// single calls run the same kernels.)
bool svd_reg_fits(int64_t n, int l, bool fp64) {
  if (fp64 || l < 1 || n < l || reg_one_smem(n, l) > kSmemBudget) return false;
  return (n <= kRegRows && l <= kRegCols) || (n <= kRegRows2 && l <= kRegCols2);
}

SmallPlan small_plan(int64_t n, int l, bool fp64) {
  SmallPlan p{l, 0, 0, 0, 0};
  const size_t es = fp64 ? 8 : 4;
  if (l <= 0 || l > TK_MAX_L || n < l) return p;
  if (svd_reg_fits(n, l, fp64)) {
    p.MB = (int)n;
    p.Pb = 1;
    p.reg = 1;
    p.scratch_bytes = 256;
    return p;
  }
  if (one_smem(n, l, es) <= kSmemBudget) {
    p.MB = (int)n;
    p.Pb = 1;
    p.scratch_bytes = 256;
    return p;
  }
  if (!fp64 && l <= kRegCols) {
    for (int Pb = 2; Pb * l <= kRegRows; ++Pb) {
      int MB = (int)((n + Pb - 1) / Pb);
      MB = std::max(MB, l);
      MB = (MB + 31) / 32 * 32;
      if (MB > kRegRows) continue;
      const int Pbe = (int)((n + MB - 1) / MB);
      if (Pbe * l <= kRegRows && reg_one_smem((int64_t)Pbe * l, l) <= kSmemBudget) {
        p.MB = MB;
        p.Pb = Pbe;
        p.reg = 1;
      }
      break;
    }
  }
  if (p.Pb <= 0) {
    for (int Pb = 2; Pb <= 64; ++Pb) {
      int MB = (int)((n + Pb - 1) / Pb);
      MB = std::max(MB, l);
      MB = (MB + 31) / 32 * 32;
      const int Pbe = (int)((n + MB - 1) / MB);
      if (leafq_smem(MB, l, es) <= kSmemBudget && root_smem(Pbe, l, es) <= kSmemBudget) {
        p.MB = MB;
        p.Pb = Pbe;
        break;
      }
    }
  }
  if (p.Pb <= 0) return p;
  const size_t Pb = p.Pb, MBs = p.MB, L = l;
  p.scratch_bytes = align256(Pb * MBs * L * es) + align256(Pb * L * es) +
                    2 * align256(Pb * L * L * es) + align256(Pb * L * 8) + align256(Pb * L * 4);
  return p;
}

// TSQR scratch of Pb leaves of MB rows (es: bytes per solver entry): leaf
// reflectors, tau, stacked R's, root result, per-leaf column maxima.
struct TsqrScratch {
  void* V;
  void* tau;
  void* Rst;
  void* Mout;
  double* colmax;
  int* colidx;
};
static TsqrScratch tsqr_carve(void* scratch, int Pb, int MB, int l, size_t es) {
  TsqrScratch t;
  unsigned char* w = (unsigned char*)scratch;
  t.V = w;                    w += align256((size_t)Pb * MB * l * es);
  t.tau = w;                  w += align256((size_t)Pb * l * es);
  t.Rst = w;                  w += align256((size_t)Pb * l * l * es);
  t.Mout = w;                 w += align256((size_t)Pb * l * l * es);
  t.colmax = (double*)w;      w += align256((size_t)Pb * l * 8);
  t.colidx = (int*)w;
  return t;
}

// Register-resident kernels with CPW columns per warp (16 warps hold l <= 16 CPW
// columns; CPW = 2 for l <= 32 keeps no idle column slots).
template <int CPW>
static cudaError_t reg_go(const SmallPlan& pl, const double* Y, int64_t n, double* Q,
                          double* sigma, void* scratch, int shift_rule, bool update_shift,
                          bool basis_only, double* alpha, double* alpha_hist, double* sigl_hist,
                          int* status, cudaStream_t st) {
  const int l = pl.l, MB = pl.MB, Pb = pl.Pb;
  if (Pb == 1) {
    count_kernels(1);
    if (n > kRegRows) {
      if constexpr (CPW == 2) {
        k_svd_reg<2, kRegRK2><<<1, kRegThreads, reg_one_smem(n, l), st>>>(
            Y, (int)n, l, Q, sigma, shift_rule, update_shift ? 1 : 0, basis_only ? 1 : 0, alpha,
            alpha_hist, sigl_hist, status);
        return cudaGetLastError();
      }
      return cudaErrorInvalidValue;
    }
    k_svd_reg<CPW><<<1, kRegThreads, reg_one_smem(n, l), st>>>(
        Y, (int)n, l, Q, sigma, shift_rule, update_shift ? 1 : 0, basis_only ? 1 : 0, alpha,
        alpha_hist, sigl_hist, status);
    return cudaGetLastError();
  }
  const TsqrScratch t = tsqr_carve(scratch, Pb, MB, l, sizeof(float));
  float* V = (float*)t.V;
  float* tau = (float*)t.tau;
  float* Rst = (float*)t.Rst;
  float* Mout = (float*)t.Mout;
  double* colmax = t.colmax;
  int* colidx = t.colidx;
  const size_t leaf_smem = ((size_t)MB * l + l) * sizeof(float);
  count_kernels(4);
  k_leaf_qr_reg<CPW><<<Pb, kRegThreads, leaf_smem, st>>>(Y, n, l, MB, Pb, V, tau, Rst);
  k_root_reg<CPW><<<1, kRegThreads, reg_one_smem((int64_t)Pb * l, l), st>>>(
      Rst, Pb, l, Mout, sigma, shift_rule, update_shift ? 1 : 0, basis_only ? 1 : 0, alpha,
      alpha_hist, sigl_hist, status);
  k_leaf_q_reg<CPW><<<dim3(Pb, (l + 15) / 16), kRegThreads, leaf_smem, st>>>(
      V, tau, Mout, n, l, MB, Pb, Q, colmax, colidx);
  k_sign<<<l, 256, 0, st>>>(Q, n, l, Pb, colmax, colidx);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t small_go(const SmallPlan& pl, const double* Y, int64_t n, double* Q,
                            double* sigma, void* scratch, int shift_rule, bool update_shift,
                            bool basis_only, double* alpha, double* alpha_hist,
                            double* sigl_hist, int* status, cudaStream_t st) {
  const int l = pl.l, MB = pl.MB, Pb = pl.Pb;
  const size_t es = sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    const int mx = (int)kSmemBudget + 4096;
    cudaFuncSetAttribute(k_svd_one<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_qr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_root<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_q<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_svd_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_svd_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_svd_reg<2, kRegRK2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_qr_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_qr_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_root_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_root_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_q_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_leaf_q_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr_set = true;
  }
  if (pl.reg && sizeof(T) == 4) {
    if (l <= 32)
      return reg_go<2>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, basis_only, alpha,
                       alpha_hist, sigl_hist, status, st);
    return reg_go<4>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, basis_only, alpha,
                     alpha_hist, sigl_hist, status, st);
  }
  if (Pb == 1) {
    const int threads = (int64_t)n * l >= 4096 ? 1024 : 256;
    count_kernels(1);
    k_svd_one<T><<<1, threads, one_smem(n, l, es), st>>>(Y, (int)n, l, Q, sigma, shift_rule,
                                                          update_shift ? 1 : 0,
                                                          basis_only ? 1 : 0, alpha,
                                                          alpha_hist, sigl_hist, status);
    return cudaGetLastError();
  }
  const TsqrScratch t = tsqr_carve(scratch, Pb, MB, l, es);
  T* V = (T*)t.V;
  T* tau = (T*)t.tau;
  T* Rst = (T*)t.Rst;
  T* Mout = (T*)t.Mout;
  double* colmax = t.colmax;
  int* colidx = t.colidx;
  count_kernels(4);
  k_leaf_qr<T><<<Pb, 512, ((size_t)MB * l + l) * es, st>>>(Y, n, l, MB, Pb, V, tau, Rst);
  k_root<T><<<1, 1024, root_smem(Pb, l, es), st>>>(Rst, Pb, l, Mout, sigma, shift_rule,
                                                   update_shift ? 1 : 0, alpha, alpha_hist,
                                                   sigl_hist, status);
  k_leaf_q<T><<<Pb, 512, leafq_smem(MB, l, es), st>>>(V, tau, Mout, n, l, MB, Pb, Q, colmax,
                                                      colidx);
  k_sign<<<l, 256, 0, st>>>(Q, n, l, Pb, colmax, colidx);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Work-list launches (one CTA per svd job; polish as in launch_polish).
// ---------------------------------------------------------------------------
// up to 1024 threads (svd_threads): the bound keeps the FP64 body within the
// 64 registers a thread such a launch allows
template <typename T>
__global__ void __launch_bounds__(1024)
k_svd_batch(const SvdJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
            uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const SvdJob J = jobs[batch_job(start, njobs, b)];
    svd_one_body<T>(J.Y, J.n, J.l, J.Q, J.sigma, J.shift_rule, J.update_shift, J.basis_only,
                    J.alpha, J.ahist, J.shist, J.status);
    __syncthreads();
  }
}

template <int CPW, int RK = kRegRK>
__global__ void __launch_bounds__(kRegThreads)
k_svd_batch_reg(const SvdJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
                uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const SvdJob J = jobs[batch_job(start, njobs, b)];
    svd_reg_body<CPW, RK>(J.Y, J.n, J.l, J.Q, J.sigma, J.shift_rule, J.update_shift,
                          J.basis_only, J.alpha, J.ahist, J.shist, J.status);
    __syncthreads();
  }
}

// The TSQR chain over a work list: each job's blocks as the single call's grid
// (leaf Q, register-resident: block b + Pb y of the job is leaf b, columns
// 16 y ..).  T = the solver's type.
template <typename T>
__global__ void __launch_bounds__(512) k_tsqr_leaf_batch(const TsqrJob* __restrict__ jobs,
                                  const uint32_t* __restrict__ start, int njobs,
                                  uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const TsqrJob J = jobs[j];
    leaf_qr_body<T>(J.Y, J.n, J.l, J.MB, J.Pb, (T*)J.V, (T*)J.tau, (T*)J.Rst,
                    (int)(b - __ldg(start + j)));
    __syncthreads();
  }
}
template <typename T>
__global__ void __launch_bounds__(1024) k_tsqr_root_batch(const TsqrJob* __restrict__ jobs,
                                  const uint32_t* __restrict__ start, int njobs,
                                  uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const TsqrJob J = jobs[batch_job(start, njobs, b)];
    root_body<T>((const T*)J.Rst, J.Pb, J.l, (T*)J.Mout, J.sigma, J.shift_rule, J.update_shift,
                 J.alpha, J.ahist, J.shist, J.status);
    __syncthreads();
  }
}
template <typename T>
__global__ void __launch_bounds__(512) k_tsqr_leafq_batch(const TsqrJob* __restrict__ jobs,
                                   const uint32_t* __restrict__ start, int njobs,
                                   uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const TsqrJob J = jobs[j];
    leaf_q_body<T>((const T*)J.V, (const T*)J.tau, (const T*)J.Mout, J.n, J.l, J.MB, J.Pb, J.Q,
                   J.colmax, J.colidx, (int)(b - __ldg(start + j)));
    __syncthreads();
  }
}
template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_tsqr_leaf_batch_reg(const TsqrJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                      int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const TsqrJob J = jobs[j];
    leaf_qr_reg_body<CPW>(J.Y, J.n, J.l, J.MB, J.Pb, (float*)J.V, (float*)J.tau, (float*)J.Rst,
                          (int)(b - __ldg(start + j)));
    __syncthreads();
  }
}
template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_tsqr_root_batch_reg(const TsqrJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                      int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const TsqrJob J = jobs[batch_job(start, njobs, b)];
    root_reg_body<CPW>((const float*)J.Rst, J.Pb, J.l, (float*)J.Mout, J.sigma, J.shift_rule,
                       J.update_shift, J.basis_only, J.alpha, J.ahist, J.shist, J.status);
    __syncthreads();
  }
}
template <int CPW>
__global__ void __launch_bounds__(kRegThreads)
k_tsqr_leafq_batch_reg(const TsqrJob* __restrict__ jobs, const uint32_t* __restrict__ start,
                       int njobs, uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const TsqrJob J = jobs[j];
    const int lb = (int)(b - __ldg(start + j));
    leaf_q_reg_body<CPW>((const float*)J.V, (const float*)J.tau, (const float*)J.Mout, J.n, J.l,
                         J.MB, J.Pb, J.Q, J.colmax, J.colidx, lb % J.Pb, lb / J.Pb);
    __syncthreads();
  }
}
__global__ void __launch_bounds__(256) k_tsqr_sign_batch(const TsqrJob* __restrict__ jobs,
                                  const uint32_t* __restrict__ start, int njobs,
                                  uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const TsqrJob J = jobs[j];
    sign_body(J.Q, J.n, J.l, J.Pb, J.colmax, J.colidx, (int)(b - __ldg(start + j)));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
k_gram_batch(const GramJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
             uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const GramJob J = jobs[j];
    gram_part_body(J.U, J.n, J.r, J.part, b - __ldg(start + j));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
k_polish_batch(const PolishJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
               uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const PolishJob J = jobs[j];
    polish_body(J.U, J.n, J.r, J.nblk, J.part, J.status, b - __ldg(start + j));
    __syncthreads();
  }
}

// 0: not register-resident; 2 / 4: column slots per warp (512 rows); 3: two
// slots, 1024 rows.
int svd_variant(int64_t n, int l, bool fp64) {
  if (!svd_reg_fits(n, l, fp64)) return 0;
  if (n > kRegRows) return 3;
  return l <= 32 ? 2 : 4;
}
int svd_threads(int64_t n, int l, bool fp64) {
  if (svd_reg_fits(n, l, fp64)) return kRegThreads;
  return (int64_t)n * l >= 4096 ? 1024 : 256;
}
size_t svd_smem(int64_t n, int l, bool fp64) {
  return svd_reg_fits(n, l, fp64) ? reg_one_smem(n, l) : one_smem(n, l, fp64 ? 8 : 4);
}
int tsqr_job(const SmallPlan& pl, bool fp64, const double* Y, int64_t n, double* Q,
             double* sigma, void* scratch, int shift_rule, bool update_shift, bool basis_only,
             double* alpha, double* ahist, double* shist, int* status, TsqrJob* job,
             TsqrStage stages[4]) {
  const int l = pl.l, MB = pl.MB, Pb = pl.Pb;
  // the single call's choice (small_go): register-resident for FP32 plans
  // marked reg, with 2 columns per warp up to l = 32
  const int flag = (pl.reg && !fp64) ? (l <= 32 ? 2 : 4) : 0;
  const size_t es = flag ? sizeof(float) : (fp64 ? sizeof(double) : sizeof(float));
  const TsqrScratch t = tsqr_carve(scratch, Pb, MB, l, es);
  TsqrJob& J = *job;
  std::memset(&J, 0, sizeof(J));
  J.Y = Y;
  J.Q = Q;
  J.sigma = sigma;
  J.alpha = alpha;
  J.ahist = ahist;
  J.shist = shist;
  J.status = status;
  J.V = t.V;
  J.tau = t.tau;
  J.Rst = t.Rst;
  J.Mout = t.Mout;
  J.colmax = t.colmax;
  J.colidx = t.colidx;
  J.n = n;
  J.l = l;
  J.MB = MB;
  J.Pb = Pb;
  J.shift_rule = shift_rule;
  J.update_shift = update_shift ? 1 : 0;
  J.basis_only = basis_only ? 1 : 0;
  const size_t leaf = ((size_t)MB * l + l) * es;
  stages[0] = TsqrStage{BK_TSQR_LEAF, (uint32_t)Pb, leaf};
  stages[1] = TsqrStage{BK_TSQR_ROOT, 1u,
                        flag ? reg_one_smem((int64_t)Pb * l, l) : root_smem(Pb, l, es)};
  stages[2] = TsqrStage{BK_TSQR_LEAFQ, (uint32_t)(flag ? Pb * ((l + 15) / 16) : Pb),
                        flag ? leaf : leafq_smem(MB, l, es)};
  stages[3] = TsqrStage{BK_TSQR_SIGN, (uint32_t)l, 0};
  return flag;
}

int polish_blocks(int64_t n) { return (int)((n + kPolishRows - 1) / kPolishRows); }
size_t gram_smem(int r) { return (size_t)kPolishRows * r * sizeof(double); }
size_t polish_smem(int r) {
  return (((size_t)r * r * sizeof(float) + 15) & ~(size_t)15) + (size_t)kPolishRows * r * sizeof(double);
}

// Raises the dynamic shared-memory limit of the work-list kernels (once per
// process; call before capturing launches into a graph).
void batch_kernels_init() {
  static bool attr = false;
  if (attr) return;
  c32_batch_init();
  const int mx = (int)kSmemBudget + 4096;
  cudaFuncSetAttribute(k_svd_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_svd_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_svd_batch_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_svd_batch_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_svd_batch_reg<2, kRegRK2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_gram_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_polish_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_leaf_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_leaf_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_tsqr_root_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_root_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_tsqr_leafq_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_tsqr_leafq_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_tsqr_leaf_batch_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_leaf_batch_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_root_batch_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_root_batch_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_tsqr_leafq_batch_reg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  cudaFuncSetAttribute(k_tsqr_leafq_batch_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       mx);
  attr = true;
}

cudaError_t launch_batch_small(const BatchLaunch& b, cudaStream_t st) {
  batch_kernels_init();
  switch (b.kind) {
    case BK_SVD:
      if (b.xt == X_F64) return run_batch(k_svd_batch<double>, b, b.tile, st);
      // jobs of one launch share a thread count: the register-resident ones
      // run 512 threads, no other svd does
      if (b.tile == kRegThreads) {
        if (b.flag == 2) return run_batch(k_svd_batch_reg<2>, b, kRegThreads, st);
        if (b.flag == 3) return run_batch(k_svd_batch_reg<2, kRegRK2>, b, kRegThreads, st);
        return run_batch(k_svd_batch_reg<4>, b, kRegThreads, st);
      }
      return run_batch(k_svd_batch<float>, b, b.tile, st);
    case BK_GRAM:
      return run_batch(k_gram_batch, b, 256, st);
    case BK_POLISH:
      return run_batch(k_polish_batch, b, 256, st);
    // the TSQR chain with the single call's thread counts (register-resident:
    // 512 throughout; shared-memory: 512, root 1024, 512; sign 256)
    case BK_TSQR_LEAF:
      if (b.flag == 2) return run_batch(k_tsqr_leaf_batch_reg<2>, b, kRegThreads, st);
      if (b.flag == 4) return run_batch(k_tsqr_leaf_batch_reg<4>, b, kRegThreads, st);
      if (b.xt == X_F64) return run_batch(k_tsqr_leaf_batch<double>, b, 512, st);
      return run_batch(k_tsqr_leaf_batch<float>, b, 512, st);
    case BK_TSQR_ROOT:
      if (b.flag == 2) return run_batch(k_tsqr_root_batch_reg<2>, b, kRegThreads, st);
      if (b.flag == 4) return run_batch(k_tsqr_root_batch_reg<4>, b, kRegThreads, st);
      if (b.xt == X_F64) return run_batch(k_tsqr_root_batch<double>, b, 1024, st);
      return run_batch(k_tsqr_root_batch<float>, b, 1024, st);
    case BK_TSQR_LEAFQ:
      if (b.flag == 2) return run_batch(k_tsqr_leafq_batch_reg<2>, b, kRegThreads, st);
      if (b.flag == 4) return run_batch(k_tsqr_leafq_batch_reg<4>, b, kRegThreads, st);
      if (b.xt == X_F64) return run_batch(k_tsqr_leafq_batch<double>, b, 512, st);
      return run_batch(k_tsqr_leafq_batch<float>, b, 512, st);
    case BK_TSQR_SIGN:
      return run_batch(k_tsqr_sign_batch, b, 256, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz rotation of W = X^T Q before the precision form's FP32 step.
//
// After the bfloat16 steps the weak columns of Q carry components along the
// leading left singular directions of X at the copy's rounding level, so the
// columns of Y = X X^T Q are dominated by sigma_1^2 times those components and
// FP32 sums of Y = X W bury the weak directions under their rounding.  With
// Z the eigenvectors of G = W^T W = Q^T X X^T Q (the Ritz vectors of X X^T in
// span(Q)), Q Z has those cross components removed, and Y Z = X (W Z) spans
// the same subspace as Y with the same singular values, so the step computes
// X (W Z) instead.  G is summed in FP32 over 64-row tiles flushed to FP64
// every 16 tiles, partial G's of up to kRitzBlocks row ranges are summed in a
// fixed order, and the l x l eigenproblem is solved by one-sided Jacobi in
// FP32 on G scaled to a unit largest diagonal entry.
// ---------------------------------------------------------------------------
constexpr int kRitzRows = 64;      // rows of W per shared-memory tile
constexpr int kRitzBlocks = 304;   // row ranges (blocks) of the Gram pass
constexpr int kRitzFlush = 16;     // tiles summed in FP32 between FP64 flushes

__device__ __forceinline__ int64_t ritz_off(int64_t j, int64_t P, int l) {
  return P == 1 ? j * l : (j % P) + P * (int64_t)l * (j / P);
}

// Partial G over rows [b R, min(cols, (b+1) R)) of W (b = blockIdx.x), block
// (ba, bb) of 64 x 64 entries (blockIdx.y = ba + nbk bb, nbk = ceil(l / 64));
// thread (ty, tx) of a 16 x 16 grid owns G(64 ba + 4 ty + i, 64 bb + 4 tx + j),
// i, j < 4.  The tile holds all l columns at row stride S = 64 nbk.
__global__ void __launch_bounds__(256) k_ritz_gram(const float* __restrict__ W, int64_t cols,
                                                   int64_t P, int l, int64_t R,
                                                   double* __restrict__ part) {
  extern __shared__ __align__(16) float sgw[];     // kRitzRows x S
  __shared__ int64_t offw[kRitzRows];
  const int nbk = (l + 63) / 64, S = 64 * nbk;
  const int ba = (int)blockIdx.y % nbk, bb = (int)blockIdx.y / nbk;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ca = 64 * ba + 4 * ty, cb = 64 * bb + 4 * tx;
  for (int e = tid; e < kRitzRows * S; e += 256) sgw[e] = 0.f;
  float acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f, accd[i][j] = 0.0;
  const int64_t jb = (int64_t)blockIdx.x * R;
  const int64_t je = min(cols, jb + R);
  // mode-major W with l a multiple of 4: a tile is 64 l contiguous floats,
  // staged as float4 and the next tile prefetched into registers
  const bool vec = P == 1 && (l & 3) == 0 && l <= kRegCols;
  constexpr int NV = kRitzRows * kRegCols / 4 / 256;   // float4 per thread (l <= 64)
  float4 pre[NV];
  auto vload = [&](int64_t t0) {
    const int64_t nel = (min(je, t0 + kRitzRows) - t0) * l;
    const float4* src = reinterpret_cast<const float4*>(W + t0 * l);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e4 = tid + q * 256;
      pre[q] = 4 * (int64_t)e4 < nel ? __ldg(src + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (vec && jb < je) vload(jb);
  int tiles = 0;
  for (int64_t j0 = jb; j0 < je; j0 += kRitzRows) {
    __syncthreads();
    if (vec) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int e4 = tid + q * 256;
        if (4 * e4 < kRitzRows * l) {
          const float v[4] = {pre[q].x, pre[q].y, pre[q].z, pre[q].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int e = 4 * e4 + k, r = e / l;
            sgw[r * S + (e - r * l)] = v[k];
          }
        }
      }
      if (j0 + kRitzRows < je) vload(j0 + kRitzRows);
    } else {
      if (tid < kRitzRows) {
        const int64_t j = j0 + tid;
        offw[tid] = j < je ? ritz_off(j, P, l) : -1;
      }
      __syncthreads();
      for (int e = tid; e < kRitzRows * l; e += 256) {
        int r, c;
        if (P == 1) { r = e / l; c = e - r * l; } else { r = e % kRitzRows; c = e / kRitzRows; }
        const int64_t o = offw[r];
        sgw[r * S + c] = o >= 0 ? __ldg(W + o + P * c) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kRitzRows; ++r) {
      const float4 av = *reinterpret_cast<const float4*>(sgw + r * S + ca);
      const float4 bv = *reinterpret_cast<const float4*>(sgw + r * S + cb);
      const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (++tiles == kRitzFlush) {
      tiles = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accd[i][j] += (double)acc[i][j], acc[i][j] = 0.f;
    }
  }
  double* out = part + (int64_t)blockIdx.x * l * l;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = ca + i, b = cb + j;
      if (a < l && b < l) out[a + (int64_t)l * b] = accd[i][j] + (double)acc[i][j];
    }
}

__global__ void __launch_bounds__(256) k_ritz_sum(const double* __restrict__ part, int nb,
                                                  int ll, double* __restrict__ G) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= ll) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * ll + e];
  G[e] = s;
}

// Z (l x l, column c = eigenvector of the c-th largest eigenvalue of G).
// smem: J (l*l) | Vp (l*l) | sg (l) | nrm (l), FP32.
__global__ void __launch_bounds__(512) k_ritz_eig(const double* __restrict__ G, int l,
                                                  float* __restrict__ Z, int* __restrict__ status) {
  extern __shared__ __align__(16) float sre[];
  float* J = sre;
  float* Vp = J + l * l;
  float* sg = Vp + l * l;
  float* nrm = sg + l;
  __shared__ int perm[TK_MAX_L];
  __shared__ double dmax;
  const int tid = threadIdx.x;
  if (tid < 32) {
    double m = 0.0;
    for (int i = tid; i < l; i += 32) m = fmax(m, G[i + (int64_t)l * i]);
    m = warp_max(m);
    if (tid == 0) dmax = m;
  }
  __syncthreads();
  const double dm = dmax;
  const bool ok = dm > 0.0 && isfinite(dm);
  if (!ok && tid == 0 && !(dm == 0.0)) atomicExch(status, (int)TK_EBREAKDOWN);
  const double sc = ok ? 1.0 / dm : 1.0;
  for (int e = tid; e < l * l; e += blockDim.x) {
    J[e] = (float)(G[e] * sc);
    Vp[e] = (e % l == e / l) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_pairs(J, Vp, l, nrm);
  __syncthreads();
  sigma_perm(J, l, sg, perm, Vp);
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    Z[e] = Vp[i + l * perm[c]];
  }
}

// W <- W Z in place, 64-row tiles; warp w of 8 owns output columns
// [CW w, CW w + CW), lane the rows lane and lane + 32.
// smem: Zs (l x 8 CW, row k = Z(k, :), zero beyond l) | T (kRitzRows x (l | 1)).
template <int CW>
__global__ void __launch_bounds__(256) k_ritz_apply(float* __restrict__ W, int64_t cols,
                                                    int64_t P, int l,
                                                    const float* __restrict__ Z) {
  constexpr int ZS = 8 * CW;
  extern __shared__ __align__(16) float sra[];
  float* Zs = sra;
  float* T = Zs + l * ZS;
  const int TS = l | 1;
  __shared__ int64_t offw[kRitzRows];
  const int tid = threadIdx.x, lane = tid & 31, cg = tid >> 5;
  for (int e = tid; e < l * ZS; e += 256) {
    const int k = e / ZS, c = e - k * ZS;
    Zs[e] = c < l ? Z[k + (int64_t)l * c] : 0.f;
  }
  const int64_t ntile = (cols + kRitzRows - 1) / kRitzRows;
  // mode-major W with l a multiple of 4: a tile is 64 l contiguous floats,
  // moved as float4, and the next tile is fetched while this one is rotated
  const bool vec = P == 1 && (l & 3) == 0 && l <= kRegCols;
  constexpr int NV = kRitzRows * kRegCols / 4 / 256;   // float4 per thread (l <= 64)
  float4 pre[NV];
  auto vload = [&](int64_t t0) {
    const int64_t nel = (min(cols, t0 + kRitzRows) - t0) * l;
    const float4* src = reinterpret_cast<const float4*>(W + t0 * l);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e4 = tid + q * 256;
      pre[q] = 4 * (int64_t)e4 < nel ? src[e4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (vec && (int64_t)blockIdx.x < ntile) vload((int64_t)blockIdx.x * kRitzRows);
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t j0 = tile * kRitzRows;
    __syncthreads();
    if (vec) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int e4 = tid + q * 256;
        if (4 * e4 < kRitzRows * l) {
          const float v[4] = {pre[q].x, pre[q].y, pre[q].z, pre[q].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int e = 4 * e4 + k, r = e / l;
            T[r * TS + (e - r * l)] = v[k];
          }
        }
      }
      if (tile + gridDim.x < ntile) vload((tile + gridDim.x) * kRitzRows);
    } else {
      if (tid < kRitzRows) {
        const int64_t j = j0 + tid;
        offw[tid] = j < cols ? ritz_off(j, P, l) : -1;
      }
      __syncthreads();
      for (int e = tid; e < kRitzRows * l; e += 256) {
        int r, c;
        if (P == 1) { r = e / l; c = e - r * l; } else { r = e % kRitzRows; c = e / kRitzRows; }
        const int64_t o = offw[r];
        T[r * TS + c] = o >= 0 ? W[o + P * c] : 0.f;
      }
    }
    __syncthreads();
    float a0[CW], a1[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) a0[c] = 0.f, a1[c] = 0.f;
#pragma unroll 2
    for (int k = 0; k < l; ++k) {
      const float x0 = T[lane * TS + k], x1 = T[(lane + 32) * TS + k];
      const float4* z4 = reinterpret_cast<const float4*>(Zs + k * ZS + cg * CW);
#pragma unroll
      for (int q = 0; q < CW / 4; ++q) {
        const float4 z = z4[q];
        a0[4 * q] = fmaf(x0, z.x, a0[4 * q]);
        a0[4 * q + 1] = fmaf(x0, z.y, a0[4 * q + 1]);
        a0[4 * q + 2] = fmaf(x0, z.z, a0[4 * q + 2]);
        a0[4 * q + 3] = fmaf(x0, z.w, a0[4 * q + 3]);
        a1[4 * q] = fmaf(x1, z.x, a1[4 * q]);
        a1[4 * q + 1] = fmaf(x1, z.y, a1[4 * q + 1]);
        a1[4 * q + 2] = fmaf(x1, z.z, a1[4 * q + 2]);
        a1[4 * q + 3] = fmaf(x1, z.w, a1[4 * q + 3]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int col = cg * CW + c;
      if (col < l) {
        T[lane * TS + col] = a0[c];
        T[(lane + 32) * TS + col] = a1[c];
      }
    }
    __syncthreads();
    if (vec) {
      const int64_t nel = (min(cols, j0 + kRitzRows) - j0) * l;
      float4* dst = reinterpret_cast<float4*>(W + j0 * l);
      for (int e4 = tid; 4 * (int64_t)e4 < nel; e4 += 256) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = 4 * e4 + k, r = e / l;
          v[k] = T[r * TS + (e - r * l)];
        }
        dst[e4] = make_float4(v[0], v[1], v[2], v[3]);
      }
    } else {
      for (int e = tid; e < kRitzRows * l; e += 256) {
        int r, c;
        if (P == 1) { r = e / l; c = e - r * l; } else { r = e % kRitzRows; c = e / kRitzRows; }
        const int64_t o = offw[r];
        if (o >= 0) W[o + P * c] = T[r * TS + c];
      }
    }
  }
}

static size_t ritz_part_bytes(int l) { return align256((size_t)kRitzBlocks * l * l * sizeof(double)); }
static size_t ritz_g_bytes(int l) { return align256((size_t)l * l * sizeof(double)); }

size_t ritz_scratch(int l) {
  return ritz_part_bytes(l) + ritz_g_bytes(l) + align256((size_t)l * l * sizeof(float));
}

cudaError_t launch_ritz_rotate(float* W, int64_t cols, int64_t P, int l, void* scratch,
                               int* status, cudaStream_t st) {
  if (l < 1 || l > TK_MAX_L || cols < 1 || P < 1) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    const int eig_max = (2 * TK_MAX_L * TK_MAX_L + 2 * TK_MAX_L) * (int)sizeof(float);
    const int app_max = (TK_MAX_L * 128 + kRitzRows * (TK_MAX_L | 1)) * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_ritz_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         eig_max);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ritz_apply<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               app_max);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  unsigned char* sb = (unsigned char*)scratch;
  double* part = (double*)sb;
  double* G = (double*)(sb + ritz_part_bytes(l));
  float* Z = (float*)(sb + ritz_part_bytes(l) + ritz_g_bytes(l));
  int64_t R = (cols + kRitzBlocks - 1) / kRitzBlocks;
  R = (R + kRitzRows - 1) / kRitzRows * kRitzRows;
  const int nb = (int)((cols + R - 1) / R);
  const int nbk = (l + 63) / 64;
  k_ritz_gram<<<dim3(nb, nbk * nbk), 256, kRitzRows * 64 * nbk * sizeof(float), st>>>(W, cols, P,
                                                                                      l, R, part);
  count_kernels(1);
  k_ritz_sum<<<(l * l + 255) / 256, 256, 0, st>>>(part, nb, l * l, G);
  count_kernels(1);
  k_ritz_eig<<<1, 512, (2 * l * l + 2 * l) * sizeof(float), st>>>(G, l, Z, status);
  count_kernels(1);
  const int64_t ntile = (cols + kRitzRows - 1) / kRitzRows;
  const int grid = (int)std::min<int64_t>(ntile, 152 * 8);
  if (l <= 64)
    k_ritz_apply<8><<<grid, 256, (l * 64 + kRitzRows * (l | 1)) * sizeof(float), st>>>(
        W, cols, P, l, Z);
  else
    k_ritz_apply<16><<<grid, 256, (l * 128 + kRitzRows * (l | 1)) * sizeof(float), st>>>(
        W, cols, P, l, Z);
  count_kernels(1);
  return cudaGetLastError();
}

cudaError_t launch_small_svd(bool fp64, const SmallPlan& pl, const double* Y, int64_t n,
                             double* Q, double* sigma, void* scratch, int shift_rule,
                             bool update_shift, double* alpha, double* alpha_hist,
                             double* sigl_hist, int* status, cudaStream_t st,
                             bool basis_only) {
  if (pl.Pb <= 0) return cudaErrorInvalidValue;
  if (fp64)
    return small_go<double>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, basis_only,
                            alpha, alpha_hist, sigl_hist, status, st);
  return small_go<float>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, basis_only,
                         alpha, alpha_hist, sigl_hist, status, st);
}

}  // namespace tk
