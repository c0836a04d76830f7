"""Pins for the deterministic Levermore-Pomraning solver (oracle/lp_ado.py).

The solver is checked against things other than itself: textbook closed forms
(homogeneous rod two-stream, pure absorbers with exponential integrals,
matrix exponentials), the Lambda -> infinity and atomic-mix limits (paper
Sec. 2), and the CLS results the paper prints for suite I (Tables 3-5).
"""
import json
from fractions import Fraction
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import lp_ado

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cls_suite1.json")


def rod_homogeneous(sigma, c, L):
    """Rod (directions +-1) through one material, unit current on x = 0:
    a = Sigma (1 - c/2), b = c Sigma / 2, kappa = sqrt(a^2 - b^2);
    T = kappa / D, R = b sinh(kappa L) / D, D = kappa cosh(kappa L) + a sinh(kappa L)."""
    a = sigma * (1 - c / 2)
    b = c * sigma / 2
    kap = math.sqrt(a * a - b * b)
    if kap * L < 1e-12:
        D = 1 + a * L
        return b * L / D, 1 / D
    D = kap * math.cosh(kap * L) + a * math.sinh(kap * L)
    return b * math.sinh(kap * L) / D, kap / D


@pytest.mark.parametrize("sigma,c,L", [(0.5, 0.0, 10.0), (1.3, 0.5, 3.0), (2.0, 0.9, 4.0), (0.7, 0.99, 10.0)])
@pytest.mark.parametrize("lam", [(2.0, 0.5), (0.1, 7.0)])
def test_rod_identical_materials_is_homogeneous_two_stream(sigma, c, L, lam):
    out = lp_ado.solve([sigma, sigma], lam, [c, c], L, "rod", nbins=0)
    R, T = rod_homogeneous(sigma, c, L)
    assert out["R"] == pytest.approx(R, rel=1e-9, abs=1e-13)
    assert out["T"] == pytest.approx(T, rel=1e-9, abs=1e-13)
    if c < 1:
        # absorption rate balance: A = (1 - c) Sigma <phi>
        assert out["total_flux"] == pytest.approx((1 - R - T) / ((1 - c) * sigma), rel=1e-9)


@pytest.mark.parametrize("sig,lam,L", [((0.5, 5.0), (2.0, 0.5), 10.0), ((0.1, 10.0), (1.0, 0.1), 3.0),
                                       ((1.0, 0.2), (0.3, 3.0), 5.0)])
def test_rod_pure_absorber_matrix_exponential(sig, lam, L):
    """u' = A u with A = [[-(S0 + 1/L0), 1/L1], [1/L0, -(S1 + 1/L1)]], u(0) = p: T = 1^T e^{AL} p;
    bin integrals from the Van Loan block exponential."""
    nb = 20
    out = lp_ado.solve(sig, lam, [0.0, 0.0], L, "rod", nbins=nb)
    A = np.array([[-(sig[0] + 1 / lam[0]), 1 / lam[1]], [1 / lam[0], -(sig[1] + 1 / lam[1])]])
    p = np.array(lam) / sum(lam)
    assert out["T"] == pytest.approx(float(np.ones(2) @ scipy.linalg.expm(A * L) @ p), rel=1e-10)
    assert out["R"] == pytest.approx(0.0, abs=1e-14)
    big = np.zeros((4, 4))
    big[:2, :2] = A
    big[:2, 2:] = np.eye(2)
    edges = np.arange(nb + 1) * L / nb
    integ = [scipy.linalg.expm(big * x)[:2, 2:] @ p for x in edges]
    ref = np.array([np.sum(integ[k + 1] - integ[k]) for k in range(nb)]) / (L / nb)
    np.testing.assert_allclose(out["flux"], ref, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("sigma,L", [(0.3, 10.0), (1.0, 2.0)])
def test_box_single_material_pure_absorber_exponential_integrals(sigma, L):
    """Cosine-law incidence on a pure absorber: T = 2 E3(Sigma L);
    bin-averaged flux 2 (E3(S x_k) - E3(S x_k+1)) / (S dx)."""
    nb = 10
    out = lp_ado.solve([sigma, sigma], [1.0, 2.0], [0.0, 0.0], L, "box3d", nbins=nb, n_half=48)
    assert out["T"] == pytest.approx(2 * scipy.special.expn(3, sigma * L), rel=2e-6)
    edges = np.arange(nb + 1) * L / nb
    e3 = scipy.special.expn(3, sigma * edges)
    np.testing.assert_allclose(out["flux"], 2 * (e3[:-1] - e3[1:]) / (sigma * L / nb), rtol=2e-6)


def test_box_two_material_pure_absorber_exponential_integrals():
    """Survival along a path of length t is 1^T e^{At} p = sum_k w_k e^{l_k t}; averaging over
    the cosine law with t = L/mu gives T = sum_k w_k 2 E3(-l_k L)."""
    sig, lam, L = (0.1, 10.0), (1.0, 0.1), 10.0
    A = np.array([[-(sig[0] + 1 / lam[0]), 1 / lam[1]], [1 / lam[0], -(sig[1] + 1 / lam[1])]])
    p = np.array(lam) / sum(lam)
    ev, V = np.linalg.eig(A)
    ev, V = np.real_if_close(ev).astype(float), np.real_if_close(V).astype(float)
    wk = (np.ones(2) @ V) * np.linalg.solve(V, p)
    T = float(np.sum(wk * 2 * scipy.special.expn(3, -ev * L)))
    out = lp_ado.solve(sig, lam, [0, 0], L, "box3d", nbins=0, n_half=48)
    assert out["T"] == pytest.approx(T, rel=2e-6)


def test_long_chords_mix_single_material_answers():
    """Lambda_0, Lambda_1 >> L: no switching, the answer is the p-weighted mix of
    the two single-material rods (paper Sec. 2, p_i = Lambda_i / (Lambda_0 + Lambda_1))."""
    sig, c, L = (0.5, 3.0), (0.6, 0.2), 4.0
    lam = (3e9, 1e9)
    out = lp_ado.solve(sig, lam, c, L, "rod")
    p = np.array(lam) / sum(lam)
    R = sum(p[i] * rod_homogeneous(sig[i], c[i], L)[0] for i in range(2))
    T = sum(p[i] * rod_homogeneous(sig[i], c[i], L)[1] for i in range(2))
    assert out["R"] == pytest.approx(R, rel=1e-6)
    assert out["T"] == pytest.approx(T, rel=1e-6)


def test_atomic_mix_limit():
    """Lambda_i -> 0 at fixed ratio: homogenised <Sigma> = sum p_i Sigma_i and
    <Sigma_s> = sum p_i c_i Sigma_i (the atomic-mix limit named in paper Sec. 2)."""
    sig, c, L = (0.5, 5.0), (0.5, 0.9), 3.0
    prev = None
    for scale in (1e-3, 1e-4, 1e-5):
        lam = (2.0 * scale, 0.5 * scale)
        out = lp_ado.solve(sig, lam, c, L, "rod")
        p = np.array(lam) / sum(lam)
        s_mix = float(p @ np.array(sig))
        c_mix = float(p @ (np.array(c) * np.array(sig))) / s_mix
        R, T = rod_homogeneous(s_mix, c_mix, L)
        err = abs(out["T"] - T) + abs(out["R"] - R)
        assert err < 50 * scale
        if prev is not None:
            assert err < prev  # converges as Lambda -> 0
        prev = err


def _load_rows():
    with open(GOLDEN) as f:
        g = json.load(f)
    mats = g["materials"]
    rows = []
    for r in g["rows"]:
        case, sub = r["case"][0], r["case"][1]
        sig = [float(Fraction(s)) for s in mats[case]["sigma"]]
        lam = [float(Fraction(s)) for s in mats[case]["lambda"]]
        c = [float(s) for s in mats[sub]["c"]]
        rows.append((r, sig, lam, c))
    return rows


def _printed_unit(s):
    """Unit of the last printed digit of a decimal string."""
    return 10.0 ** -(len(s.split(".")[1]) if "." in s else 0)


@pytest.mark.parametrize("row", _load_rows(), ids=lambda r: f"{r[0]['case']}-d{r[0]['d']}")
def test_paper_suite1_cls_tables(row):
    """The LP solution equals the expectation of the paper's CLS estimates (Tables 3-5,
    suite I): |LP - CLS| <= 4 sqrt(sigma^2 + (half a printed unit)^2) for R, T and <phi>."""
    r, sig, lam, c = row
    kind = {1: "slab1d", 2: "extruded2d", 3: "box3d"}[r["d"]]
    out = lp_ado.solve(sig, lam, c, 10.0, kind, n_half=16 if r["d"] == 2 else 32)
    for key, ours in (("R", out["R"]), ("T", out["T"]), ("phi", out["total_flux"])):
        val, sd = r[key]
        tol = 4 * math.hypot(float(sd), 0.5 * _printed_unit(val)) + 1e-6 * abs(float(val))
        assert abs(ours - float(val)) <= tol, (key, ours, val, sd)


def test_quadrature_converged():
    a = lp_ado.solve([0.1, 10.0], [1.0, 0.1], [0.99, 0.99], 10.0, "box3d", nbins=50, n_half=16)
    b = lp_ado.solve([0.1, 10.0], [1.0, 0.1], [0.99, 0.99], 10.0, "box3d", nbins=50, n_half=48)
    for k in ("R", "T", "total_flux"):
        assert a[k] == pytest.approx(b[k], rel=1e-5)
    np.testing.assert_allclose(a["flux"], b["flux"], rtol=1e-4)
    assert b["A"] == pytest.approx(b["A_track"], rel=1e-9)


def _load_rows2():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_cls_suite2.json")) as f:
        g = json.load(f)
    with open(GOLDEN) as f:
        mats = json.load(f)["materials"]
    rows = []
    for r in g["rows"]:
        case, sub = r["case"][0], r["case"][1]
        sig = [float(Fraction(s)) for s in mats[case]["sigma"]]
        lam = [float(Fraction(s)) for s in mats[case]["lambda"]]
        c = [float(s) for s in mats[sub]["c"]]
        rows.append((r, sig, lam, c))
    return rows


@pytest.mark.parametrize("row", _load_rows2(), ids=lambda r: f"{r[0]['case']}-d{r[0]['d']}")
def test_paper_suite2_cls_tables(row):
    """The LP solution with the uniform isotropic volume source equals the paper's
    suite II CLS estimates (Tables 6-8): leakage L = (T + R)/2 and <phi>."""
    r, sig, lam, c = row
    kind = {1: "slab1d", 2: "extruded2d", 3: "box3d"}[r["d"]]
    out = lp_ado.solve(sig, lam, c, 10.0, kind, n_half=16 if r["d"] == 2 else 32, source="volume")
    for key, ours in (("L", out["Lk"]), ("phi", out["total_flux"])):
        val, sd = r[key]
        tol = 4 * math.hypot(float(sd), 0.5 * _printed_unit(val)) + 1e-6 * abs(float(val))
        assert abs(ours - float(val)) <= tol, (key, ours, val, sd)


def test_volume_source_balance_and_symmetry():
    """One source particle: A + R + T = 1 with A from the track-length estimator, and
    by symmetry of the uniform source the two faces leak equally (paper Sec. 2)."""
    out = lp_ado.solve([0.3, 2.0], [0.7, 0.4], [0.6, 0.8], 4.0, "box3d", nbins=20, source="volume")
    assert out["A_track"] + out["R"] + out["T"] == pytest.approx(1.0, rel=1e-9)
    assert out["R"] == pytest.approx(out["T"], rel=1e-9)
    np.testing.assert_allclose(out["flux"], out["flux"][::-1], rtol=1e-9)


def test_extruded_quadrature_converged():
    a = lp_ado.solve([0.1, 10.0], [1.0, 0.1], [0.9, 0.9], 10.0, "extruded2d", nbins=20, n_half=12)
    b = lp_ado.solve([0.1, 10.0], [1.0, 0.1], [0.9, 0.9], 10.0, "extruded2d", nbins=20, n_half=20)
    for k in ("R", "T", "total_flux"):
        assert a[k] == pytest.approx(b[k], rel=2e-5)
    assert b["A"] == pytest.approx(b["A_track"], rel=1e-8)


def test_extruded_reduces_to_box_without_switching():
    """Lambda -> infinity: no interfaces, so the projection of the chords no longer
    matters and the extruded geometry equals the box."""
    a = lp_ado.solve([0.3, 1.1], [1e9, 3e9], [0.7, 0.4], 5.0, "extruded2d", n_half=12)
    b = lp_ado.solve([0.3, 1.1], [1e9, 3e9], [0.7, 0.4], 5.0, "box3d", n_half=12)
    assert a["R"] == pytest.approx(b["R"], rel=1e-6) and a["T"] == pytest.approx(b["T"], rel=1e-6)
