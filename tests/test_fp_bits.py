"""The integer-pipe operations of csrc/fp_bits.h on the host: the double ->
float conversion against the
host's IEEE conversion (round to nearest, ties to even, with subnormals),
on random bit patterns of every class and on the rounding boundaries:
exact ties in the normal and subnormal ranges, one unit either side of
them, the overflow threshold and the subnormal underflow threshold."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2110_08683_gb300", "csrc")

DRIVER = r"""
#include <math.h>
#include <stdio.h>
#include "fp_bits.h"

static uint64_t st = 0x9e3779b97f4a7c15ull;
static uint64_t next(void) {  /* splitmix64 */
  uint64_t z = (st += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static long bad = 0, n = 0;
static void check(uint64_t b) {
  double x;
  memcpy(&x, &b, 8);
  volatile double vx = x;
  const float want = (float)vx, got = fpb_double_to_float_rn(x);
  uint32_t wb, gb;
  memcpy(&wb, &want, 4);
  memcpy(&gb, &got, 4);
  ++n;
  if (isnan(want) ? !isnan(got) : wb != gb) {
    if (bad < 10) printf("mismatch %016llx: want %08x got %08x\n", (unsigned long long)b, wb, gb);
    ++bad;
  }
}
int main(void) {
  for (int k = 0; k < 2000000; ++k) check(next());
  /* exponents of the float range and just beyond, low fraction bits at and
     around the rounding point (29 dropped bits normal, more when subnormal) */
  for (int e = 1023 - 160; e <= 1023 + 130; ++e)
    for (int k = 0; k < 2000; ++k) {
      const uint64_t s = (next() & 1) ? 0x8000000000000000ull : 0;
      const uint64_t hi = next() & 0x000fffffe0000000ull;
      const int drop = e - 1023 + 127 > 0 ? 29 : 29 + (1 - (e - 1023 + 127));
      const uint64_t half = drop < 53 ? 1ull << (drop - 1) : 0;
      const uint64_t frac[6] = {0, half, half - 1, half + 1, (half << 1) - 1, next() & 0xfffff};
      for (int f = 0; f < 6; ++f) {
        const uint64_t m = drop < 53 ? ((hi & ~((1ull << drop) - 1)) | (frac[f] & ((1ull << drop) - 1)))
                                     : (hi | (frac[f] & 0x1fffffffull));
        check(s | ((uint64_t)e << 52) | (m & 0x000fffffffffffffull));
      }
    }
  /* zeros, infinities, NaNs, double subnormals, FLT_MAX neighbourhood */
  const uint64_t sp[] = {0, 0x8000000000000000ull, 0x7ff0000000000000ull, 0xfff0000000000000ull,
                         0x7ff8000000000000ull, 0x7ff0000000000001ull, 0xfff4000000000000ull,
                         1, 0x000fffffffffffffull, 0x47efffffe0000000ull, 0x47efffffefffffffull,
                         0x47effffff0000000ull, 0x47effffff0000001ull, 0x36a0000000000000ull,
                         0x3690000000000000ull, 0x3690000000000001ull, 0x368fffffffffffffull};
  for (unsigned k = 0; k < sizeof sp / sizeof sp[0]; ++k) check(sp[k]);
  printf("checked %ld mismatches %ld\n", n, bad);
  return bad != 0;
}
"""


def test_double_to_float_rn_matches_the_host_conversion(tmp_path):
    src = tmp_path / "fpb.c"
    src.write_text(DRIVER)
    exe = tmp_path / "fpb"
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-I", CSRC, str(src),
                        "-o", str(exe), "-lm"], capture_output=True, text=True)
    if r.returncode:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "mismatches 0" in r.stdout


COMPARE_DRIVER = r"""
#include <math.h>
#include <stdio.h>
#include "fp_bits.h"

static uint64_t st = 0x243f6a8885a308d3ull;
static uint64_t next(void) {  /* splitmix64 */
  uint64_t z = (st += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double of(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
static long bad = 0, n = 0;
static void check(double a, double b) {
  volatile double va = a, vb = b;
  const int nan = isnan(va) || isnan(vb);
  ++n;
  int ok = fpb_lt_ieee(a, b) == (va < vb) && fpb_le_ieee(a, b) == (va <= vb);
  if (!nan) ok = ok && fpb_lt_num(a, b) == (va < vb);
  if (!isnan(va)) ok = ok && fpb_ge0_num(a) == (va >= 0.0) && fpb_gt0_num(a) == (va > 0.0);
  ok = ok && fpb_is_nan(a) == (isnan(va) != 0);
  if (!ok) {
    if (bad < 10) printf("mismatch %a %a\n", a, b);
    ++bad;
  }
}
int main(void) {
  const double sp[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, -NAN,
                       of(1), of(0x8000000000000001ull), of(0x000fffffffffffffull),
                       of(0x0010000000000000ull), of(0x7fefffffffffffffull),
                       of(0xffefffffffffffffull), of(0x7ff0000000000001ull),
                       of(0xfff8000000000001ull), 2.5, -2.5, 1e-300, -1e-300};
  const int ns = sizeof sp / sizeof sp[0];
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) check(sp[i], sp[j]);
  for (int k = 0; k < 3000000; ++k) {
    const uint64_t x = next();
    check(of(x), of(next()));
    /* neighbours: equal, one ulp apart, the other sign, the same magnitude */
    check(of(x), of(x));
    check(of(x), of(x + 1));
    check(of(x + 1), of(x));
    check(of(x), of(x ^ 0x8000000000000000ull));
    /* values of ordinary size, where a mistake in the ordering shows */
    const double a = ldexp((double)(next() >> 11), -26) - 65536.0;
    const double b = (next() & 1) ? -a : ldexp((double)(next() >> 11), -26) - 65536.0;
    check(a, b);
  }
  printf("checked %ld mismatches %ld\n", n, bad);
  return bad != 0;
}
"""


def test_integer_comparisons_match_ieee(tmp_path):
    """The integer-pipe comparisons of fp_bits.h that the FP64 Riemann
    solvers and detection use give the IEEE answer on every class of
    double: signed zeros, subnormals, infinities, NaNs, neighbours one ulp
    apart and values of ordinary size."""
    src = tmp_path / "cmp.c"
    src.write_text(COMPARE_DRIVER)
    exe = tmp_path / "cmp"
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-I", CSRC, str(src),
                        "-o", str(exe), "-lm"], capture_output=True, text=True)
    if r.returncode:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "mismatches 0" in r.stdout
