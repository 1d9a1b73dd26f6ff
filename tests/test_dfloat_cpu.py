"""Double-float arithmetic of the FP64-accuracy residual operator
(csrc/dfloat.cuh), host path, against exact rational arithmetic.

A small C++ program built from the header with g++ (no contraction of
multiplies into additions, as on the device, where the round-to-nearest
intrinsics forbid it) prints, for seeded random operands spanning many
binades and signs, the double-float results of: the sum, the difference,
the two-term dot product, the complex product and the complex sum.  Each
result must be normalised (|lo| <= ulp(hi)/2) and within the error bounds
of the algorithms: the sloppy sum O(2^-47 (|x| + |y|)), the dot product
O(2^-47 (|x1 y1| + |x2 y2|)).  The device forms (packed FP32x2 sums, scalar
dot products) run the same operations per part; the GPU operator tests
compare the whole double-float operator with the FP64 one and the oracle.
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "paper_2508_16471_gb300/csrc/dfloat.cuh"
using namespace vie;
static uint64_t st = 0x9e3779b97f4a7c15ull;
static double rnd() {  // xorshift64*: sign, mantissa and a binade in [-20, 20]
    st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
    const uint64_t v = st * 2685821657736338717ull;
    const double m = (double)(v >> 11) / 9007199254740992.0;
    const int e = (int)((v >> 3) % 41) - 20;
    return ((v & 1) ? -1.0 : 1.0) * std::ldexp(0.5 + 0.5 * m, e);
}
static void put(dfl a) { std::printf(" %a %a", (double)a.hi, (double)a.lo); }
int main() {
    for (int t = 0; t < 4000; ++t) {
        const dfl x(rnd()), y(rnd()), z(rnd()), w(rnd());
        // near-cancelling pair for the sum: y close to -x
        const dfl yc(-(double)x.hi * (1.0 + std::ldexp(rnd(), -30)));
        std::printf("S");  put(x); put(y); put(x + y); std::printf("\n");
        std::printf("S");  put(x); put(yc); put(x + yc); std::printf("\n");
        std::printf("D");  put(x); put(y); put(x - y); std::printf("\n");
        std::printf("P");  put(x); put(y); put(z); put(w); put(dot2(x, y, z, w)); std::printf("\n");
        const cdf a{x, y}, b{z, w};
        const cdf p = a * b, s = a + b;
        std::printf("C");  put(x); put(y); put(z); put(w); put(p.x); put(p.y); std::printf("\n");
        std::printf("A");  put(x); put(y); put(z); put(w); put(s.x); put(s.y); std::printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ and the CUDA headers are needed to build the host test program")
    d = tmp_path_factory.mktemp("dfloat")
    src, exe = d / "t.cpp", d / "t"
    src.write_text(PROGRAM)
    cmd = [gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", ROOT, "-I", os.path.join(ROOT, "include"),
           "-I", CUDA_INC, str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return [ln.split() for ln in out.splitlines()]


def _vals(tok):
    """hex floats -> double-float values as exact fractions (hi + lo) and the pairs"""
    f = [float.fromhex(t) for t in tok]
    pairs = [(f[2 * i], f[2 * i + 1]) for i in range(len(f) // 2)]
    return [Fraction(h) + Fraction(l) for h, l in pairs], pairs


def _ulp32(v):
    """unit in the last place of a (normal) FP32 value"""
    return math.ldexp(1.0, math.frexp(v)[1] - 24)


def _normalised(h, l):
    return (h == 0.0 and l == 0.0) or abs(l) <= 0.5 * _ulp32(h)


U = Fraction(1, 2 ** 47)


def test_sum_and_difference(lines):
    n = 0
    for tok in lines:
        if tok[0] not in "SD":
            continue
        (x, y, s), pairs = _vals(tok[1:])
        exact = x + y if tok[0] == "S" else x - y
        assert _normalised(*pairs[2]), tok
        assert abs(s - exact) <= 4 * U * (abs(x) + abs(y)), tok
        n += 1
    assert n == 12000


def test_two_term_dot_product(lines):
    n = 0
    for tok in lines:
        if tok[0] != "P":
            continue
        (x1, y1, x2, y2, p), pairs = _vals(tok[1:])
        exact = x1 * y1 + x2 * y2
        assert _normalised(*pairs[4]), tok
        assert abs(p - exact) <= 8 * U * (abs(x1 * y1) + abs(x2 * y2)), tok
        n += 1
    assert n == 4000


def test_complex_product_and_sum(lines):
    n = 0
    for tok in lines:
        if tok[0] not in "CA":
            continue
        (ar, ai, br, bi, re, im), pairs = _vals(tok[1:])
        if tok[0] == "C":
            er, ei = ar * br - ai * bi, ar * bi + ai * br
            sr, si = abs(ar * br) + abs(ai * bi), abs(ar * bi) + abs(ai * br)
            assert abs(re - er) <= 8 * U * sr and abs(im - ei) <= 8 * U * si, tok
        else:
            assert abs(re - (ar + br)) <= 4 * U * (abs(ar) + abs(br)), tok
            assert abs(im - (ai + bi)) <= 4 * U * (abs(ai) + abs(bi)), tok
        assert _normalised(*pairs[4]) and _normalised(*pairs[5]), tok
        n += 1
    assert n == 8000


def test_planted_error_is_caught(lines):
    """The bounds are tight enough to see a dropped low part: replacing a
    product's low part by zero violates the dot-product bound somewhere."""
    bad = 0
    for tok in lines:
        if tok[0] != "P":
            continue
        (x1, y1, x2, y2, p), pairs = _vals(tok[1:])
        exact = x1 * y1 + x2 * y2
        if abs(Fraction(pairs[4][0]) - exact) > 8 * U * (abs(x1 * y1) + abs(x2 * y2)):
            bad += 1
    assert bad > 100
