// Small elementwise kernels: Omega tiles for inspection, the bfloat16
// shadow of the precision form, factor/core copies with type conversion.
#include <algorithm>

#include "tk_common.cuh"
#include "tk_batch.h"
#include "tk_internal.h"

namespace tk {

// out (rows x l, column-major) = Omega_k rows [row0, row0+rows).
__global__ void k_omega(int k, int64_t row0, int64_t rows, int l, uint64_t seed, uint32_t tag,
                        float* __restrict__ out) {
  const int groups = (l + 3) / 4;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * groups) return;
  const int64_t r = idx % rows;
  const int g = (int)(idx / rows);
  float w[4];
  omega4((uint64_t)(row0 + r), g, k, tag, seed, w);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (4 * g + q < l) out[r + rows * (int64_t)(4 * g + q)] = w[q];
}

cudaError_t launch_omega(int k, int64_t row0, int64_t rows, int l, uint64_t seed, uint32_t tag,
                         float* out, cudaStream_t st) {
  const int64_t tot = rows * ((l + 3) / 4);
  if (tot <= 0) return cudaSuccess;
  count_kernels(1);
  k_omega<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k, row0, rows, l, seed, tag, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Structured test matrices (Section 5.5): dense uniform and Khatri-Rao
// products, written out into the sketch's W buffer.
// ---------------------------------------------------------------------------

// u = (2 (w >> 8) + 1 - 2^24) 2^-24: an odd multiple of 2^-24 in (-1, 1); the
// integer is below 2^24 in magnitude, so both conversions are exact.
__device__ __forceinline__ float uniform_word(uint32_t w) {
  const int32_t num = (int32_t)(2u * (w >> 8) + 1u) - (1 << 24);
  return __int2float_rn(num) * 0x1p-24f;
}

__device__ __forceinline__ void uniform4(uint64_t j, int g, int k, uint32_t tag, uint64_t seed,
                                         float out[4]) {
  const uint4 ctr = make_uint4((uint32_t)j, (uint32_t)(j >> 32), (uint32_t)g,
                               ((uint32_t)k & 0xFFu) | (tag << 8));
  const uint4 w = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
  out[0] = uniform_word(w.x);
  out[1] = uniform_word(w.y);
  out[2] = uniform_word(w.z);
  out[3] = uniform_word(w.w);
}

// Khatri-Rao factors of mode k: factor f (mode geo.mode[f]) is written as
// geo.size[f] rows of lp floats (row i at kr + geo.off[f] + i lp).
__global__ void k_kr_factors(OmegaGeom geo, int k, int lp, bool gauss, uint64_t seed,
                             uint32_t tag, float* __restrict__ kr) {
  const int64_t tot = geo.off[geo.nf] / 4;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int f = 0;
    while (f + 1 < geo.nf && 4 * idx >= geo.off[f + 1]) ++f;
    const int64_t e = 4 * idx - geo.off[f];
    const int64_t i = e / lp;
    const int g = (int)((e % lp) / 4);
    const uint4 ctr = make_uint4((uint32_t)i, 0x80000000u | (uint32_t)geo.mode[f], (uint32_t)g,
                                 ((uint32_t)k & 0xFFu) | (tag << 8));
    const uint4 w = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
    float v[4];
    if (gauss) {
      box_muller(w.x, w.y, v[0], v[1]);
      box_muller(w.z, w.w, v[2], v[3]);
    } else {
      v[0] = uniform_word(w.x);
      v[1] = uniform_word(w.y);
      v[2] = uniform_word(w.z);
      v[3] = uniform_word(w.w);
    }
    *reinterpret_cast<float4*>(kr + 4 * idx) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// out(j, c) = Omega_k(jk, c) for the layout's column j, jk = j / ka + kb (j % ka)
// its row of Omega_k; four columns per thread.  P >= 1: the W layout of the
// products, (j, c) at j % P + P (c + l (j / P)); P = 0: column-major
// (cols x l).  Threads run over the four-column groups first when P = 1 and
// over j first otherwise, so that neighbouring threads write neighbouring
// addresses.
template <typename T>
__global__ void k_omega_fill(int kind, int k, int64_t cols, int l, int64_t ka, int64_t kb,
                             OmegaGeom geo, int lp, const float* __restrict__ kr,
                             uint64_t seed, uint32_t tag, T* __restrict__ out, int64_t P) {
  const int groups = (l + 3) / 4;
  const int64_t tot = cols * groups;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = P == 1 ? idx / groups : idx % cols;
    const int g = (int)(P == 1 ? idx % groups : idx / cols);
    const uint64_t jk = (uint64_t)(j / ka + kb * (j % ka));
    // the Khatri-Rao product is taken in FP64, factor by factor in ascending
    // mode order, and rounded once to the output type (exact for two
    // factors)
    double v[4] = {1.0, 1.0, 1.0, 1.0};
    if (kind == TK_OMEGA_UNIFORM || kind == TK_OMEGA_GAUSS) {
      float u[4];
      if (kind == TK_OMEGA_UNIFORM)
        uniform4(jk, g, k, tag, seed, u);
      else
        omega4(jk, g, k, tag, seed, u);
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (double)u[e];
    } else {
      uint64_t rest = jk;
      for (int f = 0; f < geo.nf; ++f) {
        const uint64_t sz = (uint64_t)geo.size[f];
        const uint64_t i = rest % sz;
        rest /= sz;
        const float4 t = __ldg(reinterpret_cast<const float4*>(kr + geo.off[f] + i * lp) + g);
        if (f == 0) {
          v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
          v[0] = __dmul_rn(v[0], (double)t.x);
          v[1] = __dmul_rn(v[1], (double)t.y);
          v[2] = __dmul_rn(v[2], (double)t.z);
          v[3] = __dmul_rn(v[3], (double)t.w);
        }
      }
    }
    const int64_t base = P == 0 ? j : (j % P) + P * l * (j / P);
    const int64_t cs = P == 0 ? cols : P;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * g + e < l) out[base + (int64_t)(4 * g + e) * cs] = (T)v[e];
  }
}

OmegaGeom omega_geom(const int64_t* dims, int d, int k, int l) {
  OmegaGeom geo{};
  const int lp = (l + 3) / 4 * 4;
  geo.off[0] = 0;
  for (int m = 0; m < d; ++m) {
    if (m == k) continue;
    geo.mode[geo.nf] = m;
    geo.size[geo.nf] = dims[m];
    geo.off[geo.nf + 1] = geo.off[geo.nf] + dims[m] * lp;
    ++geo.nf;
  }
  return geo;
}

size_t omega_scratch(int kind, const int64_t* dims, int d, int k, int l) {
  if (kind != TK_OMEGA_KR_GAUSS && kind != TK_OMEGA_KR_UNIFORM) return 0;
  const OmegaGeom geo = omega_geom(dims, d, k, l);
  return (size_t)geo.off[geo.nf] * sizeof(float);
}

cudaError_t launch_omega_fill(int kind, const int64_t* dims, int d, int k, int l, uint64_t seed,
                              uint32_t tag, int64_t ka, int64_t kb, float* kr, void* out,
                              bool f64, int64_t P, cudaStream_t st) {
  const OmegaGeom geo = omega_geom(dims, d, k, l);
  int64_t cols = 1;
  for (int f = 0; f < geo.nf; ++f) cols *= geo.size[f];
  if (cols <= 0 || l <= 0) return cudaSuccess;
  if (ka <= 0) {
    ka = cols;
    kb = 1;
  }
  const int lp = (l + 3) / 4 * 4;
  const int blocks_cap = 8 * num_sms();
  if (kind == TK_OMEGA_KR_GAUSS || kind == TK_OMEGA_KR_UNIFORM) {
    if (kr == nullptr) return cudaErrorInvalidValue;
    const int64_t tot = geo.off[geo.nf] / 4;
    if (tot > 0) {
      count_kernels(1);
      k_kr_factors<<<(unsigned)std::min<int64_t>((tot + 255) / 256, blocks_cap), 256, 0, st>>>(
          geo, k, lp, kind == TK_OMEGA_KR_GAUSS, seed, tag, kr);
    }
  }
  const int64_t tot = cols * ((l + 3) / 4);
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 4 * blocks_cap);
  count_kernels(1);
  if (f64)
    k_omega_fill<double><<<blocks, 256, 0, st>>>(kind, k, cols, l, ka, kb, geo, lp, kr, seed, tag,
                                                 (double*)out, P);
  else
    k_omega_fill<float><<<blocks, 256, 0, st>>>(kind, k, cols, l, ka, kb, geo, lp, kr, seed, tag,
                                                (float*)out, P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Holistic variants (Algorithms A.2 / B.1): the small deterministic
// ST-HOSVD of the l_1 x ... x l_d tensor and U_k = Q_k V_k.
// ---------------------------------------------------------------------------

// M (n x n, column-major) = B_(k) B_(k)^T for the strided view (P, n, S) of an
// FP64 tensor (entry (i, j = p + P s) at p + P (i + n s)).  Block t takes the
// pair (i, i') of the lower triangle with t = i (i + 1) / 2 + i'; its threads
// sum over the P S columns in a fixed order.
__global__ void k_gram_unfold(const double* __restrict__ B, int64_t P, int64_t n, int64_t S,
                              double* __restrict__ M) {
  __shared__ double red[32];
  const int64_t t = blockIdx.x;
  int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  const int64_t ip = t - i * (i + 1) / 2;
  const int64_t cols = P * S;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
    const int64_t s = j / P, p = j - s * P;
    const double a = B[p + P * (i + n * s)];
    const double b = B[p + P * (ip + n * s)];
    acc = fma(a, b, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = acc;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    acc = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      M[i + n * ip] = acc;
      M[ip + n * i] = acc;
    }
  }
}

cudaError_t launch_gram_unfold(const double* B, View v, double* M, cudaStream_t st) {
  const int64_t pairs = v.n * (v.n + 1) / 2;
  if (pairs <= 0) return cudaSuccess;
  count_kernels(1);
  k_gram_unfold<<<(unsigned)pairs, 256, 0, st>>>(B, v.P, v.n, v.S, M);
  return cudaGetLastError();
}

// U (n x r, column-major, type T) = Q (n x l, FP64) V (l x r, FP64), each
// entry summed over c in ascending order in FP64.
template <typename T>
__global__ void k_qv(const double* __restrict__ Q, int64_t n, int l, const double* __restrict__ V,
                     int r, T* __restrict__ U) {
  const int64_t tot = n * r;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    double acc = 0.0;
    for (int c = 0; c < l; ++c) acc = fma(Q[i + n * c], V[c + (int64_t)l * j], acc);
    U[idx] = (T)acc;
  }
}

cudaError_t launch_qv(const double* Q, int64_t n, int l, const double* V, int r, void* U,
                      XType dt, cudaStream_t st) {
  const int64_t tot = n * r;
  if (tot <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 8 * num_sms());
  count_kernels(1);
  if (dt == X_F64)
    k_qv<double><<<blocks, 256, 0, st>>>(Q, n, l, V, r, (double*)U);
  else
    k_qv<float><<<blocks, 256, 0, st>>>(Q, n, l, V, r, (float*)U);
  return cudaGetLastError();
}

// Round to nearest even bfloat16, 8 values per thread per step (two 16-byte
// loads, one 16-byte store) with a scalar tail.
__global__ void k_to_bf16(const float* __restrict__ x, int64_t count, uint16_t* __restrict__ out) {
  const int64_t nvec = count / 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = ((((uintptr_t)x) & 15) == 0) && ((((uintptr_t)out) & 15) == 0);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (aligned) {
    for (; i < nvec; i += stride) {
      const float4 a = reinterpret_cast<const float4*>(x)[2 * i];
      const float4 b = reinterpret_cast<const float4*>(x)[2 * i + 1];
      __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(a.z, a.w);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(b.z, b.w);
      uint4 o;
      o.x = *reinterpret_cast<uint32_t*>(&h0);
      o.y = *reinterpret_cast<uint32_t*>(&h1);
      o.z = *reinterpret_cast<uint32_t*>(&h2);
      o.w = *reinterpret_cast<uint32_t*>(&h3);
      reinterpret_cast<uint4*>(out)[i] = o;
    }
    i = nvec * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  }
  for (; i < count; i += stride) {
    __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
    out[i] = *reinterpret_cast<uint16_t*>(&h);
  }
}

cudaError_t launch_to_bf16(const float* x, int64_t count, uint16_t* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count / 8 + 255) / 256;
  const int64_t cap = 8LL * num_sms();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  count_kernels(1);
  k_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(x, count, out);
  return cudaGetLastError();
}

template <typename TO>
__device__ __forceinline__ void copy_matrix_body(const double* __restrict__ src, int64_t lds,
                                                 TO* __restrict__ dst, int64_t ldd, int64_t rows,
                                                 int64_t cols, unsigned bx) {
  const int64_t idx = (int64_t)bx * 256 + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx % rows, c = idx / rows;
  dst[i + ldd * c] = (TO)src[i + lds * c];
}

template <typename TO>
__global__ void __launch_bounds__(256)
k_copy_matrix(const double* __restrict__ src, int64_t lds, TO* __restrict__ dst, int64_t ldd,
              int64_t rows, int64_t cols) {
  copy_matrix_body<TO>(src, lds, dst, ldd, rows, cols, blockIdx.x);
}

cudaError_t launch_copy_matrix(const double* src, int64_t ld_src, void* dst, int64_t ld_dst,
                               int64_t rows, int64_t cols, XType dt, cudaStream_t st) {
  const int64_t tot = rows * cols;
  if (tot <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  count_kernels(1);
  if (dt == X_F64)
    k_copy_matrix<double><<<blocks, 256, 0, st>>>(src, ld_src, (double*)dst, ld_dst, rows, cols);
  else
    k_copy_matrix<float><<<blocks, 256, 0, st>>>(src, ld_src, (float*)dst, ld_dst, rows, cols);
  return cudaGetLastError();
}

// ROUND: the FP64 destination receives the value rounded to FP32 first (an
// FP64 copy of a factor returned in FP32).
template <typename TO, bool ROUND>
__global__ void __launch_bounds__(256)
k_copy_batch(const CopyJob* __restrict__ jobs, const uint32_t* __restrict__ start, int njobs,
             uint32_t total) {
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int j = batch_job(start, njobs, b);
    const CopyJob J = jobs[j];
    const int64_t idx = (int64_t)(b - __ldg(start + j)) * 256 + threadIdx.x;
    if (ROUND) {
      if (idx < J.rows * J.cols) {
        const int64_t i = idx % J.rows, c = idx / J.rows;
        ((TO*)J.dst)[i + J.ldd * c] = (TO)(float)J.src[i + J.lds * c];
      }
    } else {
      copy_matrix_body<TO>(J.src, J.lds, (TO*)J.dst, J.ldd, J.rows, J.cols,
                           b - __ldg(start + j));
    }
  }
}

cudaError_t launch_batch_misc(const BatchLaunch& b, cudaStream_t st) {
  if (b.kind != BK_COPY) return cudaErrorInvalidValue;
  if (b.xt == X_F64)
    return b.flag ? run_batch(k_copy_batch<double, true>, b, 256, st)
                  : run_batch(k_copy_batch<double, false>, b, 256, st);
  return run_batch(k_copy_batch<float, false>, b, 256, st);
}

cudaError_t launch_batch(const BatchLaunch& b, cudaStream_t st) {
  switch (b.kind) {
    case BK_XB:
    case BK_REDUCE:
    case BK_XTB:
    case BK_ERRFIN:
      return launch_batch_contract(b, st);
    case BK_SVD:
    case BK_GRAM:
    case BK_POLISH:
    case BK_TSQR_LEAF:
    case BK_TSQR_ROOT:
    case BK_TSQR_LEAFQ:
    case BK_TSQR_SIGN:
      return launch_batch_small(b, st);
    case BK_XTB32:
    case BK_XB32:
    case BK_XTB32RED:
    case BK_ERR32:
      return launch_batch_c32(b, st);
    case BK_TC32SPLIT:
    case BK_TC32XTB:
    case BK_TC32SKETCH:
      return launch_batch_tc32(b, st);
    default:
      return launch_batch_misc(b, st);
  }
}

cudaError_t launch_copy_tensor(const void* src, void* dst, int64_t count, XType dt,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, (size_t)count * xsize(dt), cudaMemcpyDeviceToDevice, st);
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t count, int* status) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count && !isfinite(x[idx])) atomicExch(status, (int)TK_EBREAKDOWN);
}

cudaError_t launch_check_finite(const double* x, int64_t count, int* status, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  count_kernels(1);
  k_check_finite<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(x, count, status);
  return cudaGetLastError();
}

__global__ void k_f32_to_f64(const float* __restrict__ x, int64_t count, double* __restrict__ y) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) y[idx] = (double)x[idx];
}

cudaError_t launch_to_f64_from_f32(const float* x, int64_t count, double* y, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  count_kernels(1);
  k_f32_to_f64<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(x, count, y);
  return cudaGetLastError();
}

}  // namespace tk
