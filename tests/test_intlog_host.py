"""The FP64 walk's exponential variate -ln(1 - u), compiled for the host.

cls_intlog.h is integer arithmetic only, so the host build computes exactly
what the device computes; it is checked here against 50-digit decimal
logarithms (Python's `decimal`) on draws that cover every table entry, both
evaluation paths and their boundary (u = 2^-9), and the ends of [0, 1)."""
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
#include "cls_intlog.h"
#include <cstdio>
int main() {
    cls::IntLogTables tab{cls::cls_log_n_init, cls::cls_log_t_init};
    unsigned long long k;
    while (std::scanf("%llu", &k) == 1) std::printf("%a\n", cls::exp_variate(k, tab));
}
"""


@pytest.fixture(scope="module")
def exp_variate(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("intlog")
    src, exe = d / "t.cc", d / "t"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(ks):
        out = subprocess.run([str(exe)], input="\n".join(map(str, ks)), capture_output=True, text=True,
                             check=True).stdout.split()
        return [float.fromhex(v) for v in out]

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


def test_exp_variate_within_one_ulp(exp_variate):
    getcontext().prec = 50
    ks = draws()
    got = exp_variate(ks)
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
