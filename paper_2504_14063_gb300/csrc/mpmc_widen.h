// Exact FP32 -> FP64 widening from the bits, on the integer pipes.
//
// The mixed-precision update widens every FP32 face flux before the FP64
// divergence and RK combination (so that the flux differences telescope
// exactly and the scheme stays conservative to FP64 rounding).  The
// hardware conversion issues on the FP64 pipe, which the update's FP64
// arithmetic already keeps busy; rebuilding the IEEE-754 binary64 pattern
// from the binary32 one takes a few integer operations instead.
//
// binary32: sign | 8-bit exponent (bias 127) | 23-bit fraction
// binary64: sign | 11-bit exponent (bias 1023) | 52-bit fraction
// normal:     exponent + 896, fraction shifted left by 29
// zero:       sign only
// subnormal:  normalised first (the leading one moved to bit 23)
// inf / NaN:  exponent all ones, fraction shifted (a NaN stays a NaN)
//
// Host-compilable so that a host test can compare it with the C cast over
// every binary32 bit pattern.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define MPMC_HD __host__ __device__ __forceinline__
#else
#define MPMC_HD inline
#endif

namespace mpmc {

MPMC_HD uint64_t widen_bits(uint32_t u) {
  const uint32_t s = u & 0x80000000u;
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi, lo;
  if (a >= 0x00800000u && a < 0x7f800000u) {          // normal
    hi = s | ((a >> 3) + (896u << 20));
    lo = a << 29;
  } else if (a == 0u) {                               // signed zero
    hi = s;
    lo = 0u;
  } else if (a >= 0x7f800000u) {                      // infinity, NaN
    hi = s | 0x7ff00000u | ((a & 0x007fffffu) >> 3);
    lo = a << 29;
  } else {                                            // subnormal: a = m 2^-149
#ifdef __CUDA_ARCH__
    const uint32_t sh = (uint32_t)__clz((int)a) - 8u;   // leading one to bit 23
#else
    const uint32_t sh = (uint32_t)__builtin_clz(a) - 8u;
#endif
    const uint32_t m = (a << sh) & 0x007fffffu;
    hi = s | ((897u - sh) << 20) | (m >> 3);
    lo = m << 29;
  }
  return ((uint64_t)hi << 32) | lo;
}

MPMC_HD double widen(float x) {
#ifdef __CUDA_ARCH__
  const uint64_t b = widen_bits(__float_as_uint(x));
  return __longlong_as_double((long long)b);
#else
  uint32_t u;
  std::memcpy(&u, &x, sizeof u);
  const uint64_t b = widen_bits(u);
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

}  // namespace mpmc
