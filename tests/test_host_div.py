"""Host side of the multiply-shift division used by the tensor-core GEMM's
output index maps and by the sketch's layout map: the constants that
div_magic (csrc/tcgemm.h) computes must reproduce unsigned division exactly
for every index below 2^31 (the kernels compute q = (umulhi(i, mul) + i) >> shr,
Granlund and Montgomery, 1994).  A small C++ program built against the real
header checks divisors 1..4096, the powers of two and their neighbours, the
radix of an unbounded last digit (2^31 - 1, and 0 standing for it) and random
divisors, each on edge indices and random indices."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_15234_gb300", "csrc")

PROGRAM = r"""
#include <cstdint>
#include <cstdio>
#include "tcgemm.h"

static uint32_t quot(uint32_t i, uint32_t mul, uint32_t shr) {
  const uint64_t t = ((uint64_t)i * mul) >> 32;
  return (uint32_t)((t + i) >> shr);
}

int main() {
  uint64_t s = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(s >> 33);                      // below 2^31
  };
  long checked = 0, bad = 0;
  auto check_div = [&](uint64_t d) {
    uint32_t mul, shr;
    peps::div_magic(d, &mul, &shr);
    const uint64_t dd = d == 0 ? 0x7fffffffull : d;
    uint32_t idx[10] = {0u, 1u, (uint32_t)(dd - 1), 0x7fffffffu, 0x7ffffffeu, 0, 0, 0, 0, 0};
    int ni = 5;
    if (dd < 0x7fffffffull) { idx[ni++] = (uint32_t)dd; idx[ni++] = (uint32_t)(dd + 1); }
    for (int r = 0; r < 64; ++r) {
      const uint32_t i = r < ni ? idx[r] : rnd();
      if (i >= 0x80000000u) continue;
      ++checked;
      if (quot(i, mul, shr) != (uint32_t)(i / dd)) {
        if (bad < 5) std::printf("d=%llu i=%u got %u want %u\n", (unsigned long long)d, i, quot(i, mul, shr),
                                 (uint32_t)(i / dd));
        ++bad;
      }
    }
  };
  for (uint64_t d = 0; d <= 4096; ++d) check_div(d);
  for (int b = 1; b < 31; ++b)
    for (int e = -1; e <= 1; ++e) check_div((1ull << b) + e);
  check_div(0x7fffffffull);
  for (int r = 0; r < 20000; ++r) check_div(1 + rnd() % 0x7fffffffu);
  std::printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
"""


def _cuda_include():
    from paper_2006_15234_gb300 import build
    try:
        nvcc = build.nvcc_path()
    except RuntimeError:
        return None
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda.h")) else None


def test_div_magic_matches_integer_division():
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "div.cpp")
        exe = os.path.join(tmp, "div")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", inc, src, "-o", exe], check=True,
                       capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
        assert "bad 0" in r.stdout
