"""The FP64 walk's exponential variate -ln(1 - u), (sin, cos)(2 pi u),
reciprocal and square root, compiled for the host.

cls_intmath.h is integer arithmetic only, so the host build computes exactly
what the device computes; it is checked here against 50-digit decimal
references (Python's `decimal`) on draws that cover every table entry, both
logarithm paths and their boundary (u = 2^-9), the tabulated angles and the
points halfway between them, and the ends of [0, 1)."""
from __future__ import annotations

import math
import os
import random
import shutil
import subprocess
from decimal import Decimal, getcontext

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1708_00765_gb300", "csrc")

PROGRAM = r"""
#define CLS_TABLE_SPACE
#include "cls_intmath.h"
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
    if (argc > 1 && argv[1][0] == 's') {  // sqrt(X 2^-scale) for "X_hi X_lo scale" lines
        unsigned long long hi, lo;
        int sc;
        while (std::scanf("%llu %llu %d", &hi, &lo, &sc) == 3) std::printf("%a\n", cls::sqrt_int(cls::U128{lo, hi}, sc));
        return 0;
    }
    if (argc > 1) {  // reciprocals of the doubles read as hex floats
        char buf[64];
        while (std::scanf("%63s", buf) == 1) std::printf("%a\n", cls::recip_int(std::strtod(buf, nullptr)));
        return 0;
    }
    cls::IntLogTables tab{cls::cls_log_n_init, cls::cls_log_t_init};
    unsigned long long k;
    while (std::scanf("%llu", &k) == 1) {
        double s, c;
        cls::sincos_2pi_int(k, cls::cls_sincos_q62_init, &s, &c);
        std::printf("%a %a %a\n", cls::exp_variate(k, tab), s, c);
    }
}
"""


@pytest.fixture(scope="module")
def intmath(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("intlog")
    src, exe = d / "t.cc", d / "t"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def recip(xs):
        out = subprocess.run([str(exe), "recip"], input="\n".join(x.hex() for x in xs), capture_output=True,
                             text=True, check=True).stdout.split()
        return [float.fromhex(v) for v in out]

    def run(ks):
        out = subprocess.run([str(exe)], input="\n".join(map(str, ks)), capture_output=True, text=True,
                             check=True).stdout.split("\n")
        return [tuple(float.fromhex(v) for v in line.split()) for line in out[:len(ks)]]

    def sqrt(cases):
        inp = "\n".join(f"{x >> 64} {x & (2**64 - 1)} {sc}" for x, sc in cases)
        out = subprocess.run([str(exe), "sqrt"], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return [float.fromhex(v) for v in out]

    run.recip = recip
    run.sqrt = sqrt
    return run


def draws():
    rnd = random.Random(3)
    ks = [0, 1, 2, 3, 2**44 - 1, 2**44, 2**44 + 1, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 2, 2**53 - 1]
    for p in (52, 44, 30, 12, 3):  # 1 - u = n 2^-53 at every table boundary, for several exponents
        for i in range(256):
            n = (2**52 + i * 2**44) >> (52 - p)
            for dn in (-1, 0, 1):
                if 1 <= n + dn <= 2**53 - 2**44:
                    ks.append(2**53 - (n + dn))
    ks += [rnd.getrandbits(53) for _ in range(4000)]
    ks += [rnd.getrandbits(rnd.randint(1, 44)) for _ in range(2000)]          # u < 2^-9
    ks += [2**53 - 1 - rnd.getrandbits(rnd.randint(1, 52)) for _ in range(2000)]  # u near 1
    return ks


def test_exp_variate_within_one_ulp(intmath):
    getcontext().prec = 50
    ks = draws()
    got = [g[0] for g in intmath(ks)]
    two53 = Decimal(2) ** 53
    worst = 0.0
    for k, v in zip(ks, got):
        if k == 0:
            assert v == 0.0
            continue
        ref = -((two53 - k) / two53).ln()
        err = abs(Decimal(v) - ref) / Decimal(math.ulp(float(ref)))
        worst = max(worst, float(err))
    assert worst <= 1.0, worst


def dec_pi():
    # Machin's formula
    def atan_inv(n):
        x = Decimal(1) / n
        term, total, j = x, x, 1
        while abs(term) > Decimal(10) ** -55:
            term *= -x * x
            j += 2
            total += term / j
        return total
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def dec_sin_cos(a):
    s, c, term, j = Decimal(0), Decimal(0), Decimal(1), 0
    while abs(term) > Decimal(10) ** -55 or j < 4:
        if j % 4 == 0:
            c += term
        elif j % 4 == 1:
            s += term
        elif j % 4 == 2:
            c -= term
        else:
            s -= term
        j += 1
        term = term * a / j
    return s, c


def test_sincos_within_2m53(intmath):
    getcontext().prec = 50
    rnd = random.Random(4)
    ks = [0, 1, 2**53 - 1] + [j * 2**45 + d for j in range(257) for d in (-2**44, -1, 0, 1, 2**44 - 1)
                              if 0 <= j * 2**45 + d < 2**53]
    ks += [rnd.getrandbits(53) for _ in range(3000)]
    got = intmath(ks)
    two_pi, two53 = 2 * dec_pi(), Decimal(2) ** 53
    worst = 0.0
    for k, (_, s, c) in zip(ks, got):
        a = two_pi * k / two53
        if a > dec_pi():
            a -= two_pi  # |a| <= pi keeps the series short
        rs, rc = dec_sin_cos(a)
        worst = max(worst, float(abs(Decimal(s) - rs)), float(abs(Decimal(c) - rc)))
    assert worst <= 2.0**-53, worst


def test_reciprocal_within_one_ulp(intmath):
    """recip_int against exact rational reciprocals.  The host seeds the
    Newton-Raphson steps with the correctly rounded FP32 reciprocal, the device
    with the approximate one; the two Newton steps (32-bit, then Q62) leave either within an ulp."""
    from fractions import Fraction
    rnd = random.Random(6)
    xs = [1.0, -1.0, 0.5, 1.5, math.nextafter(2.0, 0.0), math.nextafter(1.0, 2.0), -0.3, 1e-20, 2.0**-1000, 0.0]
    xs += [rnd.uniform(-1.0, 1.0) for _ in range(5000)]
    xs += [rnd.uniform(1.0, 2.0) * 2.0**rnd.randint(-80, 5) for _ in range(3000)]
    got = intmath.recip(xs)
    worst = 0.0
    for x, v in zip(xs, got):
        if x == 0.0:
            assert math.isinf(v)
            continue
        ref = 1 / Fraction(x)
        worst = max(worst, float(abs(Fraction(v) - ref) / Fraction(math.ulp(float(ref)))))
    assert worst <= 1.0, worst


def test_sqrt_within_one_ulp(intmath):
    """sqrt_int against integer square roots (math.isqrt), on the walk's three
    uses -- sqrt(u), sqrt(1 - u) and sqrt(4 u (1 - u)) for u = k 2^-53 -- and on
    arbitrary 128-bit arguments."""
    from fractions import Fraction
    rnd = random.Random(8)
    cases = [(0, 0), (1, 0), (2, 0), (4, 0), (2**126, 0), (2**127 - 1, 0), (3, 2), (2**104, 106)]
    for k in [1, 2, 2**52, 2**53 - 1] + [rnd.getrandbits(53) or 1 for _ in range(3000)]:
        cases += [(4 * k * (2**53 - k), 106), (2 * k, 54), (2 * (2**53 - k), 54)]
    cases += [(rnd.getrandbits(rnd.randint(1, 126)) | 1, 2 * rnd.randint(0, 60)) for _ in range(2000)]
    got = intmath.sqrt(cases)
    worst = 0.0
    for (x, sc), v in zip(cases, got):
        if x == 0:
            assert v == 0.0
            continue
        ref = Fraction(math.isqrt(x << 200), 2**100) / 2 ** (sc // 2)
        worst = max(worst, float(abs(Fraction(v) - ref) / Fraction(math.ulp(float(ref)))))
    assert worst <= 1.0, worst


def test_committed_tables_are_the_generators():
    """cls_math_tables.h is exactly what gen_math_tables.py computes in decimal arithmetic."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_math_tables", os.path.join(CSRC, "gen_math_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(CSRC, "cls_math_tables.h")) as f:
        assert f.read() == gen.render()
