"""The multiply-shift division the kernels use for run coordinates and vector indices
(Granlund-Montgomery division by an invariant integer), checked against integer division.
The magic numbers come from the library's own host code (sf_plan.h, compiled here with g++);
the quotient is formed as the kernels form it: (n * m) >> s on 64 bits."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PLAN_H = os.path.join(ROOT, "paper_2102_13018_gb300", "csrc", "sf_plan.h")

CHECK = r'''
#include <cstdio>
#include <cstdint>
#include "sf_plan.h"
using namespace sfgb;
static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t next31() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return uint32_t(state >> 33); }
static int check(uint32_t d, uint32_t n) {
  const DivMagic dm = div_magic(d);
  const uint32_t q = uint32_t((uint64_t(n) * dm.m) >> dm.s);
  if (q != n / d) { std::printf("d=%u n=%u got %u want %u\n", d, n, q, n / d); return 1; }
  return 0;
}
int main() {
  int bad = 0;
  std::vector<uint32_t> ds;
  for (uint32_t d = 1; d <= 4096; ++d) ds.push_back(d);
  for (int l = 12; l <= 31; ++l)
    for (int64_t e = -3; e <= 3; ++e) {
      const int64_t d = (int64_t(1) << l) + e;
      if (d >= 1 && d < (int64_t(1) << 31)) ds.push_back(uint32_t(d));
    }
  for (uint32_t d : ds) {
    const uint32_t top = 0x7FFFFFFFu;
    for (uint32_t n = 0; n < 4096; ++n) bad += check(d, n);
    for (uint32_t n = top - 4096; n < top; ++n) bad += check(d, n);
    bad += check(d, top);
    for (uint64_t q = 1; q * d <= top && q < 64; ++q) {   // around multiples of d
      bad += check(d, uint32_t(q * d - 1));
      bad += check(d, uint32_t(q * d));
    }
    for (int r = 0; r < 2000; ++r) bad += check(d, next31());
    if (bad) break;
  }
  for (uint32_t d = 1; d <= 300 && !bad; ++d)      // exhaustive below 2^20 for small divisors
    for (uint32_t n = 0; n < (1u << 20); ++n) bad += check(d, n);
  std::printf("%s\n", bad ? "FAIL" : "OK");
  return bad != 0;
}
'''


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_div_magic_matches_integer_division(tmp_path):
    src = tmp_path / "div_check.cpp"
    src.write_text(CHECK.replace("#include <cstdint>", "#include <cstdint>\n#include <vector>"))
    exe = tmp_path / "div_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(PLAN_H), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout[-2000:]
