"""The integer-pipe FP32 <-> FP64 conversions of the mixed-precision PCG
kernels (csrc/fpconv.cuh), compiled as plain C++ on the host and checked
against the compiler's IEEE conversions: every FP32 bit pattern for the
widening conversion, and random plus boundary FP64 patterns for the rounding
one (equal to IEEE round-to-nearest-even except on exact ties, which go away
from zero, and below the FP32 normal range, which flushes to zero)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2504_12908_b300", "csrc", "fpconv.cuh")

SRC = r"""
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <random>
#include "fpconv.cuh"
using namespace ipc;

static int check_d2f(double x, long long* n_bad) {
  float got = d2f_bits(x), want = (float)x;
  if (std::isnan(x)) { if (!std::isnan(got)) ++*n_bad; return 0; }
  uint64_t b = fpc_bits64(x);
  double ax = std::fabs(x);
  if (ax < (double)FLT_MIN) {  // flushed: signed zero, or FLT_MIN when rounding carries
    bool ok = (got == 0.0f || std::fabs(got) == FLT_MIN) && std::signbit(got) == std::signbit(x);
    if (!ok) ++*n_bad;
    return 0;
  }
  if ((b & ((1ull << 29) - 1)) == (1ull << 28)) {  // exact tie: away from zero
    float lo = (float)std::nextafter(x, 0.0);
    float away = std::nextafter(lo, x > 0 ? INFINITY : -INFINITY);
    if (fpc_bits32(got) != fpc_bits32(away)) ++*n_bad;
    return 1;
  }
  if (fpc_bits32(got) != fpc_bits32(want)) ++*n_bad;
  return 0;
}

int main() {
  // widening: every FP32 pattern
  long long bad_f2d = 0;
  for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
    float f = fpc_float((uint32_t)u);
    double got = f2d_bits(f);
    uint32_t ex = ((uint32_t)u >> 23) & 0xff;
    if (std::isnan(f)) { if (!std::isnan(got)) ++bad_f2d; continue; }
    if (ex == 0) {  // subnormal or zero -> signed zero
      if (!(got == 0.0 && std::signbit(got) == std::signbit(f))) ++bad_f2d;
      continue;
    }
    if (fpc_bits64(got) != fpc_bits64((double)f)) ++bad_f2d;
  }
  // narrowing: random patterns, values near FP32 boundaries, ties, specials
  long long bad_d2f = 0, ties = 0, n = 0;
  std::mt19937_64 rng(12345);
  for (int i = 0; i < 20000000; ++i) {
    uint64_t b = rng();
    double x;
    std::memcpy(&x, &b, 8);
    ties += check_d2f(x, &bad_d2f); ++n;
    // the same value scaled into the FP32 range
    int e;
    double fr = std::frexp(x, &e);
    if (std::isfinite(x) && x != 0.0) { ties += check_d2f(std::ldexp(fr, (int)(rng() % 300) - 150), &bad_d2f); ++n; }
  }
  for (uint32_t k = 0; k < 2000000; ++k) {  // exact ties and their neighbours at random FP32 values
    uint32_t u = (uint32_t)rng();
    double base = (double)fpc_float(u);
    if (!std::isfinite(base)) continue;
    uint64_t b = fpc_bits64(base) | (1ull << 28);
    for (int dlt = -1; dlt <= 1; ++dlt) {
      double x;
      uint64_t bb = b + dlt;
      std::memcpy(&x, &bb, 8);
      ties += check_d2f(x, &bad_d2f); ++n;
    }
  }
  const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, (double)FLT_MAX, -(double)FLT_MAX,
                       (double)FLT_MAX * (1 + 1e-9), 1e300, -1e300, (double)FLT_MIN, 1e-300, 1.0, -1.0};
  for (double x : sp) { ties += check_d2f(x, &bad_d2f); ++n; }
  std::printf("%lld %lld %lld %lld\n", bad_f2d, bad_d2f, ties, n);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_pipe_conversions_match_ieee(tmp_path):
    src = tmp_path / "fpconv_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fpconv_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=600).stdout.split()
    bad_f2d, bad_d2f, ties, n = (int(v) for v in out)
    assert bad_f2d == 0
    assert bad_d2f == 0
    assert ties > 1000 and n > 20000000
