"""Write cls_math_tables.h: the tables of the FP64 walk's logarithm and sine/cosine.

Run from this directory (`python gen_math_tables.py`); the output is committed.
Every value is computed here in exact or 60-digit decimal arithmetic (Python's
standard `decimal` module) and rounded once to the nearest double.

Logarithm (table-driven, after P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16, 1990):
for a double m in [1, 2) whose top 8 fraction bits are i, take
c_i = 1 + (i + 1/2)/256, F_i = the double nearest 1/c_i, and
r = m F_i - 1 (|r| <= 2^-9), so ln m = -ln F_i + ln(1 + r).  Entries with
m >= 3/2 fold one ln 2 into the table: T_i = -ln(2 F_i), and the caller adds
one to the binary exponent, so arguments just below 1 meet no cancellation
against a large multiple of ln 2.  T_i is split into a head rounded to a
multiple of 2^-47 and a tail (double); ln 2 likewise, so E ln2_hi + T_hi is
exact for |E| < 64.  Entry 256 (F = 1/2, T = 0, exponent + 1) serves the
arguments 1 - u with u < 2^-9, for which r = -u exactly.

Sine/cosine of 2 pi j / 256, j = 0..255, each rounded to the nearest double
(exact zeros and ones at the quadrant points).
"""
from __future__ import annotations

import os
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def dec(fr: Fraction) -> Decimal:
    return Decimal(fr.numerator) / Decimal(fr.denominator)


def to_double(x: Decimal) -> float:
    # Python's float() of a decimal string is correctly rounded
    return float(x)


def quantize(x: Decimal, bits: int) -> Fraction:
    """x rounded to the nearest multiple of 2^-bits, exactly."""
    scale = Decimal(2) ** bits
    n = int((x * scale).to_integral_value())
    return Fraction(n, 2 ** bits)


def ln(x: Decimal) -> Decimal:
    return x.ln()


def pi() -> Decimal:
    # Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(n: int) -> Decimal:
        x = Decimal(1) / n
        x2 = x * x
        term, total, k = x, x, 1
        while True:
            term *= -x2
            k += 2
            t = term / k
            if abs(t) < Decimal(10) ** -65:
                break
            total += t
        return total

    return 16 * atan_inv(5) - 4 * atan_inv(239)


def sin_cos(a: Decimal) -> tuple[Decimal, Decimal]:
    s, c = Decimal(0), Decimal(0)
    term, k = Decimal(1), 0  # a^k / k!
    while abs(term) > Decimal(10) ** -70 or k < 4:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
    return s, c


def hexd(v: float) -> str:
    return v.hex() if v != 0.0 else "0x0p+0"


def log_table() -> tuple[list[tuple[float, float, float]], float, float]:
    ln2 = ln(Decimal(2))
    ln2_hi = quantize(ln2, 47)
    ln2_lo = to_double(ln2 - dec(ln2_hi))
    rows = []
    for i in range(257):
        if i < 256:
            c = Fraction(1) + Fraction(2 * i + 1, 512)
            F = float(Fraction(1) / c)  # nearest double to 1/c
            fold = i >= 128
            T = -ln(dec(Fraction(F) * (2 if fold else 1)))
        else:
            F = 0.5
            T = Decimal(0)
        T_hi = quantize(T, 47)
        T_lo = to_double(T - dec(T_hi))
        rows.append((F, float(T_hi), T_lo))
        assert Fraction(float(T_hi)) == T_hi
    assert Fraction(float(ln2_hi)) == ln2_hi
    return rows, float(ln2_hi), ln2_lo


def sincos_table() -> list[tuple[float, float]]:
    twopi = 2 * pi()
    rows = []
    for j in range(256):
        if j % 64 == 0:
            q = j // 64
            rows.append(((0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0))[q])
            continue
        s, c = sin_cos(twopi * j / 256)
        rows.append((to_double(s), to_double(c)))
    return rows


def main() -> None:
    logs, ln2_hi, ln2_lo = log_table()
    sc = sincos_table()
    out = [
        "// Generated by gen_math_tables.py; do not edit.",
        "#pragma once",
        "",
        "namespace cls {",
        "",
        "// ln 2 = LN2_HI + LN2_LO, LN2_HI a multiple of 2^-47",
        f"#define CLS_LN2_HI {hexd(ln2_hi)}",
        f"#define CLS_LN2_LO {hexd(ln2_lo)}",
        "#define CLS_LOG_TABLE_N 257",
        "#define CLS_SINCOS_TABLE_N 256",
        "",
        "// {F_i, T_hi, T_lo}: r = m F_i - 1, ln m = T_hi + T_lo + ln(1 + r) (+ ln 2 for i >= 128)",
        "__device__ const double cls_log_table_init[CLS_LOG_TABLE_N][3] = {",
    ]
    for F, th, tl in logs:
        out.append(f"    {{{hexd(F)}, {hexd(th)}, {hexd(tl)}}},")
    out += ["};", "", "// {sin, cos} of 2 pi j / 256",
            "__device__ const double cls_sincos_table_init[CLS_SINCOS_TABLE_N][2] = {"]
    for s, c in sc:
        out.append(f"    {{{hexd(s)}, {hexd(c)}}},")
    out += ["};", "", "}  // namespace cls", ""]
    with open(os.path.join(HERE, "cls_math_tables.h"), "w") as fh:
        fh.write("\n".join(out))


if __name__ == "__main__":
    main()
