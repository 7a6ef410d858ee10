"""Host check of the bit-level FP32 -> FP64 widening the mixed-precision
update uses (csrc/mpmc_widen.h): compiled with the host compiler and
compared with the C conversion over every binary32 bit pattern (bit for
bit; NaNs: still NaN with the same sign)."""
import os
import shutil
import subprocess

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2504_14063_gb300", "csrc")

SRC = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include "mpmc_widen.h"
int main() {
  unsigned long long bad = 0, nan = 0;
  for (unsigned long long i = 0; i <= 0xffffffffull; ++i) {
    const unsigned u = (unsigned)i;
    float x;
    std::memcpy(&x, &u, 4);
    const double w = mpmc::widen(x);
    if (x != x) {
      ++nan;
      if (!(w != w) || std::signbit(w) != std::signbit(x)) ++bad;
      continue;
    }
    const double r = (double)x;
    if (std::memcmp(&w, &r, 8) != 0) {
      if (bad < 5) std::printf("mismatch %08x\n", u);
      ++bad;
    }
  }
  std::printf("%llu %llu\n", bad, nan);
  return bad != 0;
}
"""


def test_widen_equals_the_c_conversion_on_every_float(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "widen.cpp"
    exe = tmp_path / "widen"
    src.write_text(SRC)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    bad, nan = (int(v) for v in out.stdout.split()[-2:])
    assert nan == 2 * (2 ** 23 - 1)      # every NaN pattern was seen
    assert out.returncode == 0 and bad == 0, out.stdout
