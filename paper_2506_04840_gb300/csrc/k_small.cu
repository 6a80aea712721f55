// [Q, Sigma, ~] = svd(Y, 'econ') for a tall n x l matrix Y (Algorithms 2
// and 3 call it after the sketch and after every shifted power step), plus
// the adaptive shift update of Algorithms 2/3.
//
//  k_leaf_qr : Householder QR of row blocks of MB rows (one CTA each).
//  k_root    : Householder QR of the stacked l x l triangles, one-sided
//              (Hestenes) Jacobi on R^T, whose accumulated rotations are the
//              left singular vectors of R; descending sort; multiplication
//              of the root Q into them; the shift update.
//  k_leaf_q  : Q rows of each block = block reflectors applied to the
//              block's share of the root result; per-column largest |entry|.
//  k_sign    : sign convention (entry of largest |value| positive, lowest
//              row on ties).
//
// The working precision T is FP64 for FP64 tensors and FP32 for FP32/BF16
// tensors, matching the precision in which Y itself was formed.
#include <algorithm>
#include <cmath>

#include "tk_common.cuh"
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
      if (amax > (T)0)
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T t = x[i] / amax;
          ssq += t * t;
        }
      ssq = warp_sum(ssq);
      const T xnorm = amax * sqrt(ssq);
      const T alpha = x[j];
      T beta = alpha, tj = (T)0;
      if (xnorm > (T)0) {
        const T mx = max((T)fabs(alpha), xnorm);
        const T a1 = alpha / mx, x1 = xnorm / mx;
        beta = -copysign(mx * sqrt(a1 * a1 + x1 * x1), alpha);
        tj = (beta - alpha) / beta;
        const T scal = (T)1 / (alpha - beta);
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

// B (m x l, ld m, shared) <- H_0 H_1 ... H_{l-1} B for reflectors stored in
// V (ld m, global or shared) with factors tau.
template <typename T>
__device__ void apply_q(const T* V, const T* tau, T* B, int m, int l) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = l - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj != (T)0) {
      const T* v = V + (int64_t)m * j;
      for (int c = warp; c < l; c += nw) {
        T* y = B + (int64_t)m * c;
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

template <typename T>
__global__ void k_leaf_qr(const double* __restrict__ Y, int64_t n, int l, int MB, int Pb,
                          T* __restrict__ V, T* __restrict__ tau, T* __restrict__ Rst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* ts = A + (int64_t)MB * l;
  const int b = blockIdx.x;
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

template <typename T> __device__ __forceinline__ T jacobi_tol(int l);
template <> __device__ __forceinline__ float jacobi_tol<float>(int l) {
  return fmaxf(1e-6f, 8.0f * (float)l * 5.9604645e-8f);
}
template <> __device__ __forceinline__ double jacobi_tol<double>(int l) {
  return 8.0 * (double)l * 1.1102230246251565e-16;
}

template <typename T>
__global__ void k_root(const T* __restrict__ Rst, int Pb, int l, T* __restrict__ Vr,
                       T* __restrict__ taur, T* __restrict__ Mout, double* __restrict__ sigma,
                       int shift_rule, int update_shift, double* __restrict__ alpha,
                       double* __restrict__ alpha_hist, double* __restrict__ sigl_hist,
                       int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = Pb * l;
  T* S = reinterpret_cast<T*>(smem_raw);          // m x l
  T* J = S + (int64_t)m * l;                      // l x l, columns of R^T
  T* Vp = J + (int64_t)l * l;                     // l x l rotations
  T* sg = Vp + (int64_t)l * l;                    // l
  T* ts = sg + l;                                 // l
  __shared__ int perm[TK_MAX_L];
  __shared__ int flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int64_t e = tid; e < (int64_t)m * l; e += blockDim.x) S[e] = Rst[e];
  __syncthreads();
  householder_qr(S, m, l, ts);
  for (int64_t e = tid; e < (int64_t)m * l; e += blockDim.x) Vr[e] = S[e];
  for (int j = tid; j < l; j += blockDim.x) taur[j] = ts[j];
  // J = R^T: J(i, c) = R(c, i); Vp = I
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e % l, c = e / l;
    J[e] = (c <= i) ? S[c + (int64_t)m * i] : (T)0;
    Vp[e] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();

  // One-sided Jacobi on the columns of J, round-robin pairing.
  const int m2 = l + (l & 1);
  const T tol = jacobi_tol<T>(l);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) flag = 0;
    __syncthreads();
    for (int rd = 0; rd < m2 - 1; ++rd) {
      for (int pr = warp; pr < m2 / 2; pr += nw) {
        int p, q;
        if (pr == 0) { p = rd; q = m2 - 1; }
        else { p = (rd + pr) % (m2 - 1); q = (rd - pr + (m2 - 1)) % (m2 - 1); }
        if (p >= l || q >= l) continue;
        T* xp = J + (int64_t)l * p;
        T* xq = J + (int64_t)l * q;
        T a = 0, bb = 0, g = 0;
        for (int i = lane; i < l; i += 32) {
          a += xp[i] * xp[i];
          bb += xq[i] * xq[i];
          g += xp[i] * xq[i];
        }
        a = warp_sum(a);
        bb = warp_sum(bb);
        g = warp_sum(g);
        if (g != (T)0 && fabs(g) > tol * sqrt(a) * sqrt(bb)) {
          const T zeta = (bb - a) / (g + g);
          T t;
          if (fabs(zeta) > (T)1e15) t = (T)0.5 / zeta;
          else t = copysign((T)1 / (fabs(zeta) + sqrt((T)1 + zeta * zeta)), zeta);
          const T cs = (T)1 / sqrt((T)1 + t * t);
          const T sn = cs * t;
          for (int i = lane; i < l; i += 32) {
            const T u = xp[i], w = xq[i];
            xp[i] = cs * u - sn * w;
            xq[i] = sn * u + cs * w;
          }
          T* vp = Vp + (int64_t)l * p;
          T* vq = Vp + (int64_t)l * q;
          for (int i = lane; i < l; i += 32) {
            const T u = vp[i], w = vq[i];
            vp[i] = cs * u - sn * w;
            vq[i] = sn * u + cs * w;
          }
          if (lane == 0) flag = 1;
        }
      }
      __syncthreads();
    }
    const int f = flag;
    __syncthreads();
    if (!f) break;
  }
  // singular values = column norms of J
  for (int c = warp; c < l; c += nw) {
    const T* x = J + (int64_t)l * c;
    T s = 0;
    for (int i = lane; i < l; i += 32) s += x[i] * x[i];
    s = warp_sum(s);
    if (lane == 0) sg[c] = sqrt(s);
  }
  __syncthreads();
  for (int i = tid; i < l; i += blockDim.x) {
    const T si = sg[i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      const T sj = sg[j];
      if (sj > si || (sj == si && j < i)) ++rank;
    }
    perm[rank] = i;
  }
  __syncthreads();
  // B = [U_R ; 0] with U_R columns sorted by descending sigma
  for (int64_t e = tid; e < (int64_t)m * l; e += blockDim.x) {
    const int i = (int)(e % m), c = (int)(e / m);
    S[e] = i < l ? Vp[i + (int64_t)l * perm[c]] : (T)0;
  }
  if (tid < l) {
    const double sv = (double)sg[perm[tid]];
    sigma[tid] = sv;
    if (!isfinite(sv)) atomicExch(status, (int)TK_EBREAKDOWN);
  }
  __syncthreads();
  apply_q(Vr, ts, S, m, l);
  for (int64_t e = tid; e < (int64_t)m * l; e += blockDim.x) Mout[e] = S[e];
  if (tid == 0 && update_shift) {
    const double sl = (double)sg[perm[l - 1]];
    const double a0 = alpha[0];
    double an;
    if (shift_rule == (int)TK_SHIFT_NONE) an = 0.0;
    else an = (sl > a0) ? 0.5 * (sl + a0) : a0;
    alpha[0] = an;
    if (alpha_hist) alpha_hist[0] = an;
    if (sigl_hist) sigl_hist[0] = sl;
  }
}

template <typename T>
__global__ void k_leaf_q(const T* __restrict__ V, const T* __restrict__ tau,
                         const T* __restrict__ Mout, int64_t n, int l, int MB, int Pb,
                         double* __restrict__ Q, double* __restrict__ colmax,
                         int* __restrict__ colidx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* B = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.x;
  const int m = Pb * l;
  const int64_t r0 = (int64_t)b * MB;
  const int64_t rows = min((int64_t)MB, n - r0);
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) {
    const int i = (int)(e % MB), c = (int)(e / MB);
    B[e] = i < l ? Mout[((int64_t)b * l + i) + (int64_t)m * c] : (T)0;
  }
  __syncthreads();
  apply_q(V + (int64_t)b * MB * l, tau + (int64_t)b * l, B, MB, l);
  for (int64_t e = threadIdx.x; e < (int64_t)MB * l; e += blockDim.x) {
    const int64_t i = e % MB, c = e / MB;
    if (i < rows) Q[(r0 + i) + n * c] = (double)B[e];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < l; c += nw) {
    double best = -1.0;
    int bi = 0;                      // a valid row even if every entry is NaN
    for (int i = lane; i < rows; i += 32) {
      const double v = fabs((double)B[i + (int64_t)MB * c]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      // (lanes that saw only NaN keep best = -1 and lose every comparison)
    }
    if (lane == 0) {
      colmax[(int64_t)b * l + c] = best;
      colidx[(int64_t)b * l + c] = (int)(r0 + bi);
    }
  }
}

__global__ void k_sign(double* __restrict__ Q, int64_t n, int l, int Pb,
                       const double* __restrict__ colmax, const int* __restrict__ colidx) {
  __shared__ double sgn;
  const int c = blockIdx.x;
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

// ---------------------------------------------------------------------------
// FP64 re-orthonormalisation of a factor computed in FP32 arithmetic:
// U <- U R^{-1} with R^T R = U^T U (one CholeskyQR step).  U is already
// orthonormal to FP32 rounding, so the Gram matrix is within ~1e-5 of the
// identity and the Cholesky factorisation is perfectly conditioned.
// ---------------------------------------------------------------------------
constexpr int kPolishRows = 64;

__global__ void k_gram_part(const double* __restrict__ U, int64_t n, int r,
                            double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ub = reinterpret_cast<double*>(smem_raw);     // kPolishRows x r
  const int b = blockIdx.x;
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

__global__ void k_polish(double* __restrict__ U, int64_t n, int r, int nblk,
                         const double* __restrict__ part, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* R = reinterpret_cast<double*>(smem_raw);      // r x r
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < r * r; e += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * r * r + e];
    R[e] = s;
  }
  __syncthreads();
  // Cholesky, upper factor in place: R(i, j) for i <= j, R^T R = G.
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      double d = R[j + r * j];
      for (int k = 0; k < j; ++k) d -= R[k + r * j] * R[k + r * j];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      R[j + r * j] = sqrt(d);
    }
    __syncthreads();
    const double djj = R[j + r * j];
    for (int c = j + 1 + tid; c < r; c += blockDim.x) {
      double s = R[j + r * c];
      for (int k = 0; k < j; ++k) s -= R[k + r * j] * R[k + r * c];
      R[j + r * c] = s / djj;
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0 && blockIdx.x == 0) atomicExch(status, (int)TK_EBREAKDOWN);
    return;
  }
  // rows of this block: u <- u R^{-1} (forward substitution on R^T)
  const int64_t r0 = (int64_t)blockIdx.x * kPolishRows;
  const int rows = (int)min((int64_t)kPolishRows, n - r0);
  for (int i = tid; i < rows; i += blockDim.x) {
    double* u = U + r0 + i;
    for (int c = 0; c < r; ++c) {
      double s = u[n * c];
      for (int k = 0; k < c; ++k) s -= u[n * k] * R[k + r * c];
      u[n * c] = s / R[c + r * c];
    }
  }
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
  k_polish<<<nblk, 128, (size_t)r * r * sizeof(double), st>>>(U, n, r, nblk,
                                                               (const double*)scratch, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
static const size_t kSmemBudget = 200 * 1024;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t root_smem(int Pb, int l, size_t es) {
  return ((size_t)Pb * l * l + 2 * (size_t)l * l + 2 * (size_t)l) * es;
}

SmallPlan small_plan(int64_t n, int l, bool fp64) {
  SmallPlan p{l, 0, 0, 0};
  const size_t es = fp64 ? 8 : 4;
  if (l <= 0 || l > TK_MAX_L || n < l) return p;
  int MB = (int)std::max<int64_t>(l, std::min<int64_t>(n, 128));
  MB = (MB + 31) / 32 * 32;
  for (;;) {
    const int Pb = (int)((n + MB - 1) / MB);
    const size_t leaf = ((size_t)MB * l + l) * es;
    if (leaf > kSmemBudget) return p;
    if (root_smem(Pb, l, es) <= kSmemBudget) {
      p.MB = MB;
      p.Pb = Pb;
      break;
    }
    if (Pb == 1) return p;
    MB *= 2;
  }
  const size_t Pb = p.Pb, MBs = p.MB, L = l;
  p.scratch_bytes = align256(Pb * MBs * L * es) + align256(Pb * L * es) +
                    3 * align256(Pb * L * L * es) + align256(L * es) + align256(Pb * L * 8) +
                    align256(Pb * L * 4);
  return p;
}

template <typename T>
static cudaError_t small_go(const SmallPlan& pl, const double* Y, int64_t n, double* Q,
                            double* sigma, void* scratch, int shift_rule, bool update_shift,
                            double* alpha, double* alpha_hist, double* sigl_hist, int* status,
                            cudaStream_t st) {
  const int l = pl.l, MB = pl.MB, Pb = pl.Pb;
  const size_t es = sizeof(T);
  unsigned char* w = (unsigned char*)scratch;
  T* V = (T*)w;            w += align256((size_t)Pb * MB * l * es);
  T* tau = (T*)w;          w += align256((size_t)Pb * l * es);
  T* Rst = (T*)w;          w += align256((size_t)Pb * l * l * es);
  T* Vr = (T*)w;           w += align256((size_t)Pb * l * l * es);
  T* Mout = (T*)w;         w += align256((size_t)Pb * l * l * es);
  T* taur = (T*)w;         w += align256((size_t)l * es);
  double* colmax = (double*)w; w += align256((size_t)Pb * l * 8);
  int* colidx = (int*)w;

  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_leaf_qr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget + 4096);
    cudaFuncSetAttribute(k_root<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget + 4096);
    cudaFuncSetAttribute(k_leaf_q<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget + 4096);
    attr_set = true;
  }
  const size_t leaf_smem = ((size_t)MB * l + l) * es;
  count_kernels(4);
  k_leaf_qr<T><<<Pb, 256, leaf_smem, st>>>(Y, n, l, MB, Pb, V, tau, Rst);
  k_root<T><<<1, 512, root_smem(Pb, l, es), st>>>(Rst, Pb, l, Vr, taur, Mout, sigma, shift_rule,
                                                  update_shift ? 1 : 0, alpha, alpha_hist,
                                                  sigl_hist, status);
  k_leaf_q<T><<<Pb, 256, (size_t)MB * l * es, st>>>(V, tau, Mout, n, l, MB, Pb, Q, colmax,
                                                    colidx);
  k_sign<<<l, 256, 0, st>>>(Q, n, l, Pb, colmax, colidx);
  return cudaGetLastError();
}

cudaError_t launch_small_svd(bool fp64, const SmallPlan& pl, const double* Y, int64_t n,
                             double* Q, double* sigma, void* scratch, int shift_rule,
                             bool update_shift, double* alpha, double* alpha_hist,
                             double* sigl_hist, int* status, cudaStream_t st) {
  if (pl.Pb <= 0) return cudaErrorInvalidValue;
  if (fp64)
    return small_go<double>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, alpha,
                            alpha_hist, sigl_hist, status, st);
  return small_go<float>(pl, Y, n, Q, sigma, scratch, shift_rule, update_shift, alpha,
                         alpha_hist, sigl_hist, status, st);
}

}  // namespace tk
