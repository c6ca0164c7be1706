"""Host build of the double <-> double-float conversions (csrc/ddconv.cuh) against exact rational
arithmetic: the split of a double into hi + lo, the exact widening of a float, and the join of a
pair into a double as the kernels form it (both parts widened, one FP64 addition).

The transforms of the FP64 form compute in double-float and read or write FP64 spectra through
these routines, so their error bounds are what the FP64 form's accuracy rests on there."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2302_08694_gb300", "csrc", "ddconv.cuh")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "ddconv.cuh"
using namespace fsib::ddconv;
int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (op[0] == 's') {
      unsigned long long b = 0;
      if (std::scanf("%llx", &b) != 1) return 1;
      double x; std::memcpy(&x, &b, 8);
      float hi = 0, lo = 0;
      const bool ok = split_double(x, hi, lo);
      std::printf("%d %08x %08x\n", ok ? 1 : 0, f2u(hi), f2u(lo));
    } else {
      unsigned h = 0, l = 0;
      if (std::scanf("%x %x", &h, &l) != 2) return 1;
      const double o = widen_float(u2f(h)) + widen_float(u2f(l));
      std::printf("1 %016llx\n", (unsigned long long)d2u(o));
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ddconv")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.dirname(HDR), str(src), "-o",
                    str(exe)], check=True)

    def run(lines):
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return r.stdout.split("\n")[: len(lines)]
    return run


def f32(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def f64(bits):
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def random_double(rng, emin, emax):
    e = rng.randint(emin, emax) + 1023
    m = rng.getrandbits(52)
    s = rng.getrandbits(1)
    return (s << 63) | (e << 52) | m


def test_split_is_exact_up_to_the_low_part_rounding(harness):
    rng = random.Random(7)
    xs = [random_double(rng, -74, 127) for _ in range(4000)]
    # boundaries of the covered range and special mantissas
    xs += [dbits(v) for v in (1.0, -1.0, 2.0 ** -74, -(2.0 ** -74), 2.0 ** 127, 1.5, 3.0, 0.1, -0.3, 1e-20, 1e30,
                              (2.0 - 2.0 ** -52) * 2.0 ** 127, 1.0 + 2.0 ** -52, 1.0 + 2.0 ** -23, 1.0 - 2.0 ** -53)]
    out = harness([f"s {b:016x}" for b in xs])
    for b, line in zip(xs, out):
        ok, h, l = line.split()
        assert ok == "1", hex(b)
        x = Fraction(f64(b))
        hi, lo = Fraction(f32(int(h, 16))), Fraction(f32(int(l, 16)))
        ulp_hi = Fraction(2) ** ((int(h, 16) >> 23) & 0xFF) / 2 ** 150
        # hi: x cut towards zero to 24 bits; lo: the rest rounded to 24 bits, so |lo| <= ulp(hi) and
        # both share x's sign
        assert abs(hi) <= abs(x) < abs(hi) + ulp_hi
        assert (hi > 0) == (x > 0)
        assert lo == 0 or (lo > 0) == (x > 0)
        assert abs(lo) <= ulp_hi
        assert abs(x - (hi + lo)) <= abs(x) * Fraction(1, 2 ** 48)


def test_split_of_small_and_out_of_range_values(harness):
    # |x| < 2^-126 (zeros and denormals included): hi = lo = signed zero
    tiny = [0, 1 << 63, 1, (1 << 63) | 12345, dbits(2.0 ** -127), dbits(-1e-300)]
    out = harness([f"s {b:016x}" for b in tiny])
    for b, line in zip(tiny, out):
        ok, h, l = line.split()
        sign = (b >> 32) & 0x80000000
        assert ok == "1" and int(h, 16) == sign and int(l, 16) == sign
    # 2^-126 <= |x| < 2^-74: hi = x cut to 24 bits, lo = signed zero (error below 2^-97)
    rng = random.Random(5)
    small = [random_double(rng, -126, -75) for _ in range(500)] + [dbits(2.0 ** -126), dbits(-(2.0 ** -75))]
    out = harness([f"s {b:016x}" for b in small])
    for b, line in zip(small, out):
        ok, h, l = line.split()
        x, hi = Fraction(f64(b)), Fraction(f32(int(h, 16)))
        assert ok == "1" and int(l, 16) == (b >> 32) & 0x80000000
        assert abs(hi) <= abs(x) and abs(x - hi) <= abs(x) * Fraction(1, 2 ** 23)
        assert abs(x - hi) < Fraction(1, 2 ** 97)
    # |x| >= 2^128, infinities, NaN: declined (the caller converts them in FP64)
    outside = [dbits(v) for v in (2.0 ** 128, -1e300, float("inf"), float("-inf"), float("nan"))]
    out = harness([f"s {b:016x}" for b in outside])
    assert all(line.split()[0] == "0" for line in out)


def test_widen_is_exact(harness):
    rng = random.Random(11)
    floats = [(rng.getrandbits(1) << 31) | (rng.randint(1, 254) << 23) | rng.getrandbits(23) for _ in range(3000)]
    floats += [0x3F800000, 0xBF800000, 0x00800000, 0x7F7FFFFF, 0xFF7FFFFF]
    out = harness([f"j {h:08x} 00000000" for h in floats])  # hi + (+0)
    for h, line in zip(floats, out):
        assert int(line.split()[1], 16) == dbits(f32(h)), hex(h)
    # zero and denormals widen to a signed zero; infinities and NaN keep their value
    zs = (0x00000000, 0x80000000, 0x00000001, 0x807FFFFF)
    out = harness([f"j {h:08x} {h & 0x80000000:08x}" for h in zs])  # lo: a zero of the same sign
    assert [int(line.split()[1], 16) for line in out] == [0, 1 << 63, 0, 1 << 63]
    out = harness([f"j {h:08x} 00000000" for h in (0x7F800000, 0xFF800000)])
    assert [f64(int(line.split()[1], 16)) for line in out] == [float("inf"), float("-inf")]


def test_round_trip(harness):
    """split, then the kernels' join: within the pair's 2^-48 of x plus the final rounding"""
    rng = random.Random(3)
    xs = [random_double(rng, -70, 120) for _ in range(2000)]
    out = harness([f"s {b:016x}" for b in xs])
    pairs = [(int(line.split()[1], 16), int(line.split()[2], 16)) for line in out]
    back = harness([f"j {h:08x} {l:08x}" for h, l in pairs])
    for b, line in zip(xs, back):
        ok, o = line.split()
        x = Fraction(f64(b))
        assert abs(Fraction(f64(int(o, 16))) - x) <= abs(x) * Fraction(1, 2 ** 47)
