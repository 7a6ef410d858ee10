"""Host check of the bit-level FP64 -> FP32 rounding the mixed-precision
primitive pass uses (csrc/mpmc_narrow.h): compiled with the host compiler
and compared bit for bit with the C conversion (round to nearest, ties to
even) on random doubles over the whole exponent range, exact ties of both
parities, and the boundaries (the largest finite FP32 and the carry into
infinity, the smallest normal, zeros, infinities, NaN).  The same header's
integer-pipe zero and sign tests (nonzero, positive, negative) are compared with the C
comparisons on random bit patterns of every class (normal, subnormal, zero,
infinity, NaN) and the special values."""
import os
import shutil
import subprocess

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2504_14063_gb300", "csrc")

SRC = r"""
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <limits>
#include "mpmc_narrow.h"
static unsigned long long bad = 0, n = 0;
static void check(double x) {
  ++n;
  const float a = mpmc::narrow(x), b = (float)x;
  if (std::isnan(b)) {
    if (!std::isnan(a)) ++bad;
    return;
  }
  uint32_t ua, ub;
  std::memcpy(&ua, &a, 4);
  std::memcpy(&ub, &b, 4);
  if (ua != ub) {
    if (bad < 5) std::printf("mismatch %.17g\n", x);
    ++bad;
  }
}
static double from_bits(uint64_t u) { double d; std::memcpy(&d, &u, 8); return d; }
int main() {
  uint64_t s = 88172645463325252ull;
  auto rnd = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
  for (int i = 0; i < 20000000; ++i) {
    // exponents spread over FP32's range and beyond it on both sides
    const uint64_t e = 1023 - 160 + (rnd() % 310);
    const uint64_t m = rnd() & 0x000fffffffffffffull;
    const uint64_t sg = (rnd() & 1) << 63;
    check(from_bits(sg | (e << 52) | m));
    // an exact tie: the 29 dropped bits are 1000...0
    const uint64_t mt = (m & ~0x1fffffffull) | 0x10000000ull;
    check(from_bits(sg | (e << 52) | mt));
  }
  const double edge[] = {0.0, -0.0, (double)FLT_MAX, -(double)FLT_MAX, (double)FLT_MIN, (double)FLT_MIN * 0.5,
                         std::nextafter((double)FLT_MAX, 1e300), 3.4028235677973366e38, 3.402823567797337e38,
                         std::ldexp(1.0, 128), std::ldexp(1.0, -126), std::ldexp(1.0, -127), std::ldexp(1.0, -149),
                         std::ldexp(1.0, -150), 1e-300, 1e300, std::numeric_limits<double>::infinity(),
                         -std::numeric_limits<double>::infinity(), std::numeric_limits<double>::quiet_NaN(),
                         1.0, 1.0 + std::ldexp(1.0, -24), 1.0 + std::ldexp(1.0, -24) + std::ldexp(1.0, -52),
                         1.0 + 3 * std::ldexp(1.0, -24), 0.1, 300.0, 101325.0, 6e8};
  for (double x : edge) check(x);
  // the integer-pipe zero and sign tests against the comparisons: random
  // bit patterns of every class, and the special values
  for (int i = 0; i < 4000000; ++i) {
    const uint64_t u = rnd();
    const double xs[] = {from_bits(u), from_bits(u & 0x800fffffffffffffull), from_bits(u | 0x7ff0000000000000ull)};
    for (double x : xs) {
      ++n;
      if (mpmc::nonzero(x) != (x != 0.0) || mpmc::positive(x) != (x > 0.0) || mpmc::negative(x) != (x < 0.0)) ++bad;
    }
  }
  for (double x : edge) {
    ++n;
    if (mpmc::nonzero(x) != (x != 0.0) || mpmc::positive(x) != (x > 0.0) || mpmc::negative(x) != (x < 0.0)) ++bad;
    if (mpmc::nonzero(-x) != (-x != 0.0) || mpmc::positive(-x) != (-x > 0.0) || mpmc::negative(-x) != (-x < 0.0))
      ++bad;
  }
  std::printf("%llu %llu\n", bad, n);
  return bad != 0;
}
"""


def test_narrow_equals_the_c_conversion(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "narrow.cpp"
    exe = tmp_path / "narrow"
    src.write_text(SRC)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    bad, n = (int(v) for v in out.stdout.split()[-2:])
    assert n > 40000000
    assert out.returncode == 0 and bad == 0, out.stdout
