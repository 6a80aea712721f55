// Common device code of the GB300 Tucker library: Philox4x32-10 Gaussian
// test-matrix entries (Omega_k of Algorithms 2 and 3, never stored) and
// small helpers.  sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "tucker.h"

#define TK_THREADS 256

namespace tk {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  One round maps
// (c0,c1,c2,c3) to (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0));
// the key advances by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Box-Muller with the library's own FP32 log and sin/cos.  Only correctly
// rounded single operations (__fadd_rn/__fmul_rn/__fdiv_rn/__fsqrt_rn) are
// used, so no contraction into FMA can change the bits; the sequence is
// fixed by the library's Omega definition and matches the CPU oracle bit
// for bit.
//   u1 = (2*(wa>>9)+1) 2^-24 = m 2^-24, m odd;  m = f 2^e with f moved into
//   [sqrt(1/2), sqrt(2)];  ln f = 2 atanh(s), s = (f-1)/(f+1), Taylor series
//   to s^11;  ln u1 = (e-24) ln2 (hi+lo split) + ln f.
//   angle = 2 pi (wb>>8) / 2^24 reduced exactly to an octant on the integer
//   bits; sin/cos of theta in [0, pi/4] by Taylor series to theta^9 and
//   theta^10; octant symmetries.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ln_u1(uint32_t wa) {
  const uint32_t m = 2u * (wa >> 9) + 1u;          // odd, < 2^24
  int e = 31 - __clz(m);                           // floor(log2 m)
  uint32_t fbits = 0x3F800000u | ((m << (23 - e)) & 0x7FFFFFu);
  if (fbits > 0x3FB504F3u) {                       // f > sqrt(2) (FP32)
    fbits -= 0x00800000u;                          // f / 2, exact
    e += 1;
  }
  const float f = __uint_as_float(fbits);
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float z = __fmul_rn(s, s);
  float t = __fmul_rn(0x1.745d18p-4f, z);          // 1/11
  t = __fadd_rn(t, 0x1.c71c72p-4f);                // 1/9
  t = __fmul_rn(t, z);
  t = __fadd_rn(t, 0x1.24924ap-3f);                // 1/7
  t = __fmul_rn(t, z);
  t = __fadd_rn(t, 0x1.99999ap-3f);                // 1/5
  t = __fmul_rn(t, z);
  t = __fadd_rn(t, 0x1.555556p-2f);                // 1/3
  t = __fmul_rn(t, z);
  t = __fadd_rn(t, 1.0f);
  const float lnf = __fmul_rn(__fadd_rn(s, s), t);
  const float E = (float)(e - 24);                 // exact small integer
  return __fadd_rn(__fmul_rn(E, 0x1.62e4p-1f), __fadd_rn(__fmul_rn(E, 0x1.7f7d1cp-20f), lnf));
}

__device__ __forceinline__ void cos_sin_2pi(uint32_t wb, float& cv, float& sv) {
  const int x = (int)(wb >> 8);
  const int oct = x >> 21;
  const int rem = x & 0x1FFFFF;
  const int rr = (oct & 1) ? (0x200000 - rem) : rem;
  const float th = __fmul_rn((float)rr, 0x1.921fb6p-22f);   // (pi/4) 2^-21
  const float z = __fmul_rn(th, th);
  float p = __fmul_rn(0x1.71de3ap-19f, z);                  // 1/9!
  p = __fadd_rn(p, -0x1.a01a02p-13f);                       // -1/7!
  p = __fmul_rn(p, z);
  p = __fadd_rn(p, 0x1.111112p-7f);                         // 1/5!
  p = __fmul_rn(p, z);
  p = __fadd_rn(p, -0x1.555556p-3f);                        // -1/3!
  const float st = __fadd_rn(th, __fmul_rn(__fmul_rn(th, z), p));
  float c = __fmul_rn(-0x1.27e4fcp-22f, z);                 // -1/10!
  c = __fadd_rn(c, 0x1.a01a02p-16f);                        // 1/8!
  c = __fmul_rn(c, z);
  c = __fadd_rn(c, -0x1.6c16c2p-10f);                       // -1/6!
  c = __fmul_rn(c, z);
  c = __fadd_rn(c, 0x1.555556p-5f);                         // 1/4!
  c = __fmul_rn(c, z);
  c = __fadd_rn(c, -0.5f);                                  // -1/2!
  const float ct = __fadd_rn(1.0f, __fmul_rn(z, c));
  switch (oct) {
    case 0: cv = ct;  sv = st;  break;
    case 1: cv = st;  sv = ct;  break;
    case 2: cv = -st; sv = ct;  break;
    case 3: cv = -ct; sv = st;  break;
    case 4: cv = -ct; sv = -st; break;
    case 5: cv = -st; sv = -ct; break;
    case 6: cv = st;  sv = -ct; break;
    default: cv = ct; sv = -st; break;
  }
}

__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& za, float& zb) {
  const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_u1(wa)));
  float cv, sv;
  cos_sin_2pi(wb, cv, sv);
  za = __fmul_rn(r, cv);
  zb = __fmul_rn(r, sv);
}

// Four consecutive entries Omega_k(j, 4g .. 4g+3).
__device__ __forceinline__ void omega4(uint64_t j, int g, int k, uint32_t tag, uint64_t seed,
                                       float out[4]) {
  const uint4 ctr = make_uint4((uint32_t)j, (uint32_t)(j >> 32), (uint32_t)g,
                               ((uint32_t)k & 0xFFu) | (tag << 8));
  const uint4 w = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
  box_muller(w.x, w.y, out[0], out[1]);
  box_muller(w.z, w.w, out[2], out[3]);
}

// ---------------------------------------------------------------------------
// Type helpers.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename TA, typename TX> __device__ __forceinline__ TA load_as(const TX* p) {
  return (TA)(*p);
}
template <> __device__ __forceinline__ float load_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// Accumulation type for an input element type.
template <typename TX> struct acc_of { typedef float type; };
template <> struct acc_of<double> { typedef double type; };

// Work-list launches: the job whose block range [start[j], start[j+1])
// holds block b (start ascending, start[0] == 0).
__device__ __forceinline__ int batch_job(const uint32_t* __restrict__ start, int njobs,
                                         uint32_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace tk
