"""Multiply-high division by invariant divisors (the index decoding of the
element-wise, reduction, flat-contraction and packing kernels) against exact
integer division: the header's host path is the same arithmetic as the
device path (__umulhi is the high half of the 64-bit product)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1701_02011_gb300", "csrc")

PROGRAM = r"""
#include "kernels.cuh"
#include <cstdio>
#include <cstdint>
using namespace dsrg;
static uint64_t state = 88172645463325252ull;
static uint32_t next32() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return (uint32_t)state; }
int main() {
  long long bad = 0, checked = 0;
  auto check = [&](uint32_t d, uint32_t n) {
    FastDiv f = make_fastdiv(d);
    ++checked;
    if (fast_div(n, f) != n / d) { if (bad < 5) printf("d=%u n=%u\n", d, n); ++bad; }
  };
  for (uint32_t d = 1; d <= 4096; ++d) {
    const uint32_t edge[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d - 1u, 0x7fffffffu, 0x80000000u, 0xffffffffu};
    for (uint32_t n : edge) check(d, n);
    for (int i = 0; i < 64; ++i) check(d, next32());
  }
  for (int k = 1; k < 32; ++k) {
    const uint32_t ds[] = {(1u << k) - 1u, 1u << k, (1u << k) + 1u};
    for (uint32_t d : ds)
      for (int i = 0; i < 256; ++i) check(d, next32());
  }
  for (int i = 0; i < 200000; ++i) {
    uint32_t d = next32() >> (next32() & 31);
    if (d == 0) d = 1;
    check(d, next32());
  }
  printf("checked %lld bad %lld\n", checked, bad);
  return bad != 0;
}
"""


def test_fast_division_matches_exact_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    src = tmp_path / "fastdiv.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
