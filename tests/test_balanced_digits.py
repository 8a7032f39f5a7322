"""The digit representation of the basis digit cache (csrc/ozbalanced.cuh),
compiled for the host and checked against exact rational arithmetic: for an
element x and a reference exponent E, the seven signed digits are integers
(|D_0| <= 256, the others in [-128, 127] before the sign), exact in bf16,
and sum (with weights 2^(8 (6 - i)) 2^(E - 1078)) to x truncated to 56 bits
below 2^(E - 1078 + 56), including subnormals, zeros, both signs and
carries into the top digit; non-finite entries give zero digits."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2507_07788_gb300", "csrc")

HARNESS = r'''
#include <stdio.h>
#include <math.h>
#include "ozbalanced.cuh"
int main() {
  unsigned long long b; int E;
  while (scanf("%llx %d", &b, &E) == 2) {
    const unsigned long long W = cqr::cwords(b, E);
    const float s = (b >> 63) ? -1.0f : 1.0f;
    for (int i = 0; i < 7; ++i) printf("%.1f ", (double)cqr::cdigit(W, i, s));
    printf("\n");
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("bal")
    src = d / "h.cu"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)])
    return str(exe)


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def cases():
    rng = random.Random(7)
    out = []
    for _ in range(3000):
        x = rng.uniform(-1, 1) * 10.0 ** rng.uniform(-300, 300)
        ef = max((bits(x) >> 52) & 0x7FF, 1)
        out.append((bits(x), ef + rng.choice([0, 0, 1, 3, 8, 20, 55, 56, 70])))
    # carries into the top digit: significands near all ones at the reference
    for k in range(200):
        m = (1 << 53) - 1 - rng.randrange(1 << 12)
        x = math.ldexp(m, -52) * rng.choice([1, -1])
        out.append((bits(x), (bits(x) >> 52) & 0x7FF))
    for x in (0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1.7976931348623157e308, 1.0, -1.0):
        out.append((bits(x), max((bits(x) >> 52) & 0x7FF, 1)))
    for b in (0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000):  # Inf, -Inf, NaN
        out.append((b, 0x7FF))
    return out


def test_balanced_digits_reconstruct(harness):
    cs = cases()
    inp = "".join(f"{b:x} {E}\n" for b, E in cs)
    res = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True)
    lines = res.stdout.strip().split("\n")
    assert len(lines) == len(cs)
    for (b, E), line in zip(cs, lines):
        D = [float(v) for v in line.split()]
        assert all(d == int(d) for d in D)
        D = [int(d) for d in D]
        ef = (b >> 52) & 0x7FF
        if ef == 0x7FF:
            assert D == [0] * 7
            continue
        sign = -1 if b >> 63 else 1
        mags = [sign * d for d in D]
        assert 0 <= mags[0] <= 256 and all(-128 <= v <= 127 for v in mags[1:]), (hex(b), E, D)
        x = struct.unpack("<d", struct.pack("<Q", b))[0]
        unit = Fraction(2) ** (E - 1078)
        trunc = Fraction(math.floor(Fraction(abs(x)) / unit)) * unit
        got = sum(Fraction(d) * 2 ** (8 * (6 - i)) for i, d in enumerate(D)) * unit
        assert got == sign * trunc, (hex(b), E, D)
        assert abs(Fraction(abs(x)) - trunc) < unit  # the dropped part lies below one unit
