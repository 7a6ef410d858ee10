// FP64 -> FP32 rounding to nearest, ties to even, from the bits on the
// integer pipes.
//
// The mixed-precision primitive pass rounds a dozen FP64 values per cell to
// FP32 for its cache.  The hardware conversion issues on the FP64 pipe, which
// the pass's FP64 inversion already keeps busy.  For inputs in the normal
// FP32 range (and zeros) the binary32 pattern is built from the binary64 one:
//   exponent - 1023 + 127, the 52-bit fraction cut to 23 bits and rounded to
//   nearest with ties to even (a carry into the exponent is the correct next
//   binade, or infinity above the largest finite value);
// subnormal results, infinities and NaN take the hardware conversion, which
// computes the same rounding.
//
// Host-compilable so that a host test can compare it with the C cast (and
// the zero / sign tests below with the C comparisons).
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define MPMC_HD2 __host__ __device__ __forceinline__
#else
#define MPMC_HD2 inline
#endif

namespace mpmc {

// the binary32 pattern of x rounded to nearest even, or 0x7fc00001 (a NaN
// pattern the rounding never produces) when x needs the general conversion
MPMC_HD2 uint32_t narrow_bits(uint64_t b) {
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0x000fffffffffffffull;
  if (e == 0 && m == 0) return sign;                     // signed zero
  const int E = e - 1023 + 127;
  if (E < 1 || E > 254) return 0x7fc00001u;              // subnormal, overflow, inf, NaN
  uint32_t out = sign | ((uint32_t)E << 23) | (uint32_t)(m >> 29);
  const uint64_t rem = m & 0x1fffffffull, half = 0x10000000ull;
  if (rem > half || (rem == half && (out & 1u))) out += 1u;  // carry may reach inf: correct
  return out;
}

MPMC_HD2 float narrow(double x) {
#ifdef __CUDA_ARCH__
  const uint32_t r = narrow_bits((uint64_t)__double_as_longlong(x));
  return r == 0x7fc00001u ? (float)x : __uint_as_float(r);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  const uint32_t r = narrow_bits(b);
  if (r == 0x7fc00001u) return (float)x;
  float f;
  std::memcpy(&f, &r, sizeof f);
  return f;
#endif
}

MPMC_HD2 uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

// y != 0, y > 0 and y < 0 from the bits, on the integer pipes (an FP64 comparison
// issues on the FP64 pipe, which binds the FP64 kernels); the same results
// as the comparisons for every input: +-0 is zero, NaN is nonzero and not
// positive, +inf is positive
MPMC_HD2 bool nonzero(double y) { return (bits_of(y) << 1) != 0ull; }
MPMC_HD2 bool positive(double y) {
  const int64_t b = (int64_t)bits_of(y);
  return b > 0 && b <= (int64_t)0x7ff0000000000000ull;
}
// y < 0: the sign bit set on a nonzero magnitude that is not NaN
MPMC_HD2 bool negative(double y) {
  const uint64_t b = bits_of(y), m = b & 0x7fffffffffffffffull;
  return (b >> 63) != 0 && m != 0 && m <= 0x7ff0000000000000ull;
}

}  // namespace mpmc
