"""Write cls_math_tables.h: the tables of the FP64 walk's logarithm and sine/cosine.

Run from this directory (`python gen_math_tables.py`); the output is committed.
Every value is computed here in exact or 60-digit decimal arithmetic (Python's
standard `decimal` module) and rounded once to a fixed-point integer.

Logarithm (table-driven, after P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16, 1990),
for the walk's integer evaluation of -ln(1 - u): for m in [1, 2) whose top 8
fraction bits are i, N_i = round(2048 / c_i), c_i = 1 + (i + 1/2)/256, so that
r = m N_i / 2048 - 1 is an exact 64-bit product with |r| < 2^-8.6, and
ln m = T_i + ln(1 + r), T_i = -ln(N_i / 2048), tabulated as a 128-bit
fixed-point number with 120 fraction bits (as is ln 2).

Sine/cosine of 2 pi j / 256, j = 0..255, as 64-bit fixed-point numbers with 62
fraction bits, rounded (exact zeros and ones at the quadrant points).
"""
from __future__ import annotations

import os
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def dec(fr: Fraction) -> Decimal:
    return Decimal(fr.numerator) / Decimal(fr.denominator)


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


def log_table() -> tuple[list[tuple[int, int]], int]:
    """[(N_i, T_i 2^120 rounded)], ln 2 2^120 rounded."""
    scale = Decimal(2) ** 120
    ln2 = int((ln(Decimal(2)) * scale).to_integral_value())
    rows = []
    for i in range(256):
        c = Fraction(1) + Fraction(2 * i + 1, 512)
        N = round(Fraction(2048) / c)
        assert 1024 < N <= 2048
        T = -ln(dec(Fraction(N, 2048)))
        rows.append((N, int((T * scale).to_integral_value())))
    return rows, ln2


def sincos_table() -> list[tuple[int, int]]:
    """[(sin, cos) of 2 pi j / 256, times 2^62, rounded]."""
    twopi = 2 * pi()
    one = 1 << 62
    rows = []
    for j in range(256):
        if j % 64 == 0:
            rows.append(((0, one), (one, 0), (0, -one), (-one, 0))[j // 64])
            continue
        s, c = sin_cos(twopi * j / 256)
        scale = Decimal(one)
        rows.append((int((s * scale).to_integral_value()), int((c * scale).to_integral_value())))
    return rows


def two_pi_q60() -> int:
    return int((2 * pi() * Decimal(2) ** 60).to_integral_value())


def render() -> str:
    """The text of cls_math_tables.h."""
    logs, ln2 = log_table()
    sc = sincos_table()
    M64 = (1 << 64) - 1
    out = [
        "// Generated by gen_math_tables.py; do not edit.",
        "#pragma once",
        "",
        "#include <stdint.h>",
        "",
        "#ifndef CLS_TABLE_SPACE",
        "#define CLS_TABLE_SPACE __device__",
        "#endif",
        "",
        "namespace cls {",
        "",
        "// ln 2 2^120, rounded: high and low 64-bit words",
        f"#define CLS_LN2_Q120_HI 0x{ln2 >> 64:016x}ull",
        f"#define CLS_LN2_Q120_LO 0x{ln2 & M64:016x}ull",
        "// 2 pi 2^60, rounded",
        f"#define CLS_TWO_PI_Q60 0x{two_pi_q60():016x}ll",
        "#define CLS_LOG_TABLE_N 256",
        "#define CLS_SINCOS_TABLE_N 256",
        "",
        "// N_i = round(2048 / c_i), c_i = 1 + (i + 1/2)/256",
        "CLS_TABLE_SPACE const uint16_t cls_log_n_init[CLS_LOG_TABLE_N] = {",
    ]
    for j in range(0, 256, 16):
        out.append("    " + ", ".join(str(N) for N, _ in logs[j:j + 16]) + ",")
    out += ["};", "",
            "// T_i = -ln(N_i / 2048) 2^120, rounded: {low, high} 64-bit words",
            "CLS_TABLE_SPACE const uint64_t cls_log_t_init[CLS_LOG_TABLE_N][2] = {"]
    for _, T in logs:
        out.append(f"    {{0x{T & M64:016x}ull, 0x{T >> 64:016x}ull}},")
    out += ["};", "", "// {sin, cos} of 2 pi j / 256, times 2^62, rounded",
            "CLS_TABLE_SPACE const int64_t cls_sincos_q62_init[CLS_SINCOS_TABLE_N][2] = {"]
    for s_, c_ in sc:
        out.append(f"    {{{s_}ll, {c_}ll}},")
    out += ["};", "", "}  // namespace cls", ""]
    return "\n".join(out)


def main() -> None:
    with open(os.path.join(HERE, "cls_math_tables.h"), "w") as fh:
        fh.write(render())


if __name__ == "__main__":
    main()
