"""Host-side checks of the 64-bit fixed-point conversions used by the FP64 PCG's
integer stencil (fx_from_double / fx_to_double / fx_exponent in
csrc/mqs_internal.cuh): compiled for the host with nvcc and compared, bit for
bit, with exact scaled arithmetic in 80-bit long double (a power-of-two scaling
and a 63-bit integer are exact there; the final rounding is the one under test).
No GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "mqs_internal.cuh"
using namespace mqs;

static long long exact_fx(double v, int sh) {            // round half away from zero
  const long double x = ldexpl((long double)v, sh);
  return (long long)llroundl(x);
}
static double exact_to_double(long long t, int sh) {     // nearest, ties to even
  return (double)ldexpl((long double)t, sh);
}
static bool same(double a, double b) { return std::memcmp(&a, &b, sizeof a) == 0; }

int main() {
  std::mt19937_64 rng(1611);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  long bad = 0, n = 0;
  // to fixed: |v| < 2^(E-1), sh = 58 - E, E over a wide range
  for (int E = -300; E <= 300; E += 7)
    for (int q = 0; q < 2000; ++q) {
      double v = std::ldexp(u(rng), E - 1) * std::ldexp(1.0, -(int)(rng() % 60));
      if (q % 97 == 0) v = std::ldexp(q % 2 ? 1.0 : -1.0, E - 2);          // powers of two
      if (q % 101 == 0) v = std::nextafter(std::ldexp(1.0, E - 1), 0.0);   // just below the bound
      if (q == 5) v = 0.0;
      if (q == 6) v = 4.9e-324;                                            // subnormal
      const int sh = 58 - E;
      const long long got = fx_from_double(v, sh), want = (v == 4.9e-324) ? 0 : exact_fx(v, sh);
      ++n;
      if (got != want) { if (bad++ < 5) printf("to_fx E=%d v=%a got %lld want %lld\n", E, v, got, want); }
      if (got >= (1LL << 58) || got <= -(1LL << 58)) { ++bad; printf("range %lld\n", got); }
    }
  // to double: integers up to 2^62 in magnitude, scales over a wide range, ties included
  for (int q = 0; q < 400000; ++q) {
    const int bits = 1 + (int)(rng() % 62);
    long long t = (long long)(rng() >> (64 - bits));
    if (q % 3 == 0) t = -t;
    if (q % 11 == 0) t = (t | 1) << (q % 9);                              // exact ties at the 53-bit cut
    if (q % 13 == 0) t = ((1LL << 53) + 1) << (q % 9);
    const int sh = -400 + (int)(rng() % 450);
    const double got = fx_to_double(t, sh), want = exact_to_double(t, sh);
    ++n;
    if (!same(got, want)) { if (bad++ < 5) printf("to_double t=%lld sh=%d got %a want %a\n", t, sh, got, want); }
  }
  // the scale: every component of a vector of squared norm ss lies below 2^(E-1)
  for (int q = 0; q < 200000; ++q) {
    const double ss = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), -1000 + (int)(rng() % 2000));
    const int E = fx_exponent(ss);
    ++n;
    if (!(std::sqrt(ss) * (1.0 + 1e-9) < std::ldexp(1.0, E - 1)) || !(std::sqrt(ss) >= std::ldexp(1.0, E - 4))) {
      if (bad++ < 5) printf("exponent ss=%a E=%d\n", ss, E);
    }
  }
  printf("checked %ld bad %ld\n", n, bad);
  return bad != 0;
}
"""


def test_fixed_point_conversions_are_exactly_rounded(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "fx_check.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "fx_check"
    inc = os.path.join(ROOT, "paper_1611_06721_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-I", inc, str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout[-2000:]
    assert "bad 0" in res.stdout
