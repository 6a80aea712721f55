// Small elementwise kernels: Omega tiles for inspection, the bfloat16
// shadow of the precision form, factor/core copies with type conversion.
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
      return launch_batch_small(b, st);
    case BK_XTB32:
    case BK_XB32:
    case BK_XTB32RED:
    case BK_ERR32:
      return launch_batch_c32(b, st);
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
