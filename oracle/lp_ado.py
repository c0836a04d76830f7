"""Deterministic solution of the Levermore-Pomraning (LP) equations.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

CLS Algorithm A solves the LP model -- the ensemble-averaged transport
equation (paper Eq. ``boltzmann_ave``) closed with <phi_ab> = <phi_a> and
transition rate p_ij = p_i / Lambda_i (paper Eq. ``closure_lp_boltzmann``) --
exactly in expectation (paper Sec. 4).  This module solves those equations
without Monte Carlo, so it pins the oracle's expected R, T, <phi> and phi(x).

Geometry: the LP equations for the x-marginal of the flux,

    mu_n d psi_{i,n}/dx = -(Sigma_i + r_i(mu_n)) psi_{i,n} + r_j(mu_n) psi_{j,n}
                          + (c_i Sigma_i / 2) sum_m w_m psi_{i,m},

with interface rate per unit path length r_i(mu):
  * ``"box3d"``: 1/Lambda_i -- the 3D box, whose interface distance is drawn
    along the flight (paper Sec. 4.3, d_i = -Lambda ln(1 - xi)); specular
    lateral faces leave the x-marginal equal to an infinite slab;
  * ``"slab1d"``: |mu|/Lambda_i -- the paper's d = 1 slab, whose interface
    distance is projected on x (paper Sec. 4.1, d_i = -Lambda/|mu| ln(1 - xi));
  * ``"extruded2d"``: rho/Lambda_i with rho = sqrt(1 - mu_z^2) -- the paper's
    2D extruded geometry, whose interface distance is the in-plane chord
    projected on the flight (paper Sec. 4.2, d_i = -Lambda/sqrt(1-mu^2)
    ln(1 - xi), mu the cosine to the extrusion axis z); the rate then depends
    on the azimuth psi of the direction around x, mu_z = sqrt(1 - mu^2) sin psi;
  * ``"rod"``: mu = +-1 with weights 1, rate 1/Lambda_i.
Directions use a double Gauss-Legendre rule on [0,1] and [-1,0] (box3d, slab1d),
times a Gauss-Legendre rule in psi on [0, pi/2] for extruded2d (the solution
depends on psi only through sin^2 psi).

Suite I incidence: psi_i(0, mu > 0) = p_i f with f = 1 / sum_{mu_n > 0} w_n mu_n
(unit incident current, isotropic incident angular flux -- the cosine law of
paper Sec. 4.1/4.3); psi(L, mu < 0) = 0.

Suite II: a uniform isotropic volume source of one particle in total, born in
material i with probability p_i (paper Sec. 2, 4.1, 4.3): the source term
q_i = p_i / (L sum_m w_m) is added to every equation, no incident flux.  Its
particular solution is the constant psi_p = -C^-1 q of the collision /
transition matrix C; the modal part then satisfies psi_p + psi_h = 0 on the
incoming directions of both faces.

The solution is the analytical discrete-ordinates form psi(x) = sum_k a_k v_k
exp(lambda_k (x - x_k)) with x_k = L for growing modes and 0 for decaying
ones, so no exponential overflows; the 2N boundary conditions fix a_k.
Bin integrals of exp are done in closed form.
"""
from __future__ import annotations

import numpy as np


def directions(kind: str, n_half: int = 32, n_psi: int = 12):
    """(mu, w, rate): x direction cosines, weights (sum 2) and the factor that
    multiplies 1/Lambda in each direction's interface rate."""
    if kind == "rod":
        return np.array([1.0, -1.0]), np.array([1.0, 1.0]), np.array([1.0, 1.0])
    x, w = np.polynomial.legendre.leggauss(n_half)
    mu_h = 0.5 * (x + 1.0)
    w_h = 0.5 * w
    mu = np.concatenate([mu_h, -mu_h])
    wt = np.concatenate([w_h, w_h])
    if kind == "slab1d":
        return mu, wt, np.abs(mu)
    if kind == "box3d":
        return mu, wt, np.ones_like(mu)
    if kind == "extruded2d":
        xp, wp = np.polynomial.legendre.leggauss(n_psi)
        psi = 0.25 * np.pi * (xp + 1.0)
        wpsi = wp / 2.0  # normalised to sum 1 over [0, pi/2]
        MU, PSI = np.meshgrid(mu, psi, indexing="ij")
        W = np.outer(wt, wpsi)
        rho = np.sqrt(1.0 - (1.0 - MU ** 2) * np.sin(PSI) ** 2)
        return MU.ravel(), W.ravel(), rho.ravel()
    raise ValueError(kind)


def _integral_exp(lam, a, b, ref):
    """int_a^b exp(lam (x - ref)) dx, stable for lam -> 0."""
    h = b - a
    small = np.abs(lam) * h < 1e-8
    safe = np.where(lam == 0.0, 1.0, lam)
    # factor out the larger end so the remaining exponent is <= 0:
    #   lam > 0: exp(lam(b-ref)) * (1 - exp(-lam h)) / lam
    #   lam < 0: exp(lam(a-ref)) * (exp(lam h) - 1) / lam
    grow = lam > 0.0
    top = np.where(grow, lam * (b - ref), lam * (a - ref))
    with np.errstate(over="ignore", invalid="ignore"):
        body = np.where(grow, -np.expm1(-lam * h), np.expm1(lam * h)) / safe
        out = np.where(small, np.exp(lam * (0.5 * (a + b) - ref)) * h, np.exp(top) * body)
    return out


def solve(sigma, lam, c, L, kind: str, nbins: int = 0, n_half: int = 32, source: str = "incident") -> dict:
    """Solve the LP equations for suite I (source="incident") or suite II
    (source="volume") sources.

    Returns R, T, A, total_flux (= int phi dx), track (per material), and if
    nbins > 0 the bin-averaged flux on the uniform mesh e_k = k L / nbins.
    For the volume source R and T are the currents leaving x = 0 and x = L and
    Lk = (R + T) / 2 is the paper's leakage observable."""
    sigma = np.asarray(sigma, dtype=float)
    lam = np.asarray(lam, dtype=float)
    c = np.asarray(c, dtype=float)
    mu, w, rate = directions(kind, n_half)
    n = mu.size
    K = 2 * n
    p = lam / lam.sum()
    C = np.zeros((K, K))
    for i in range(2):
        j = 1 - i
        for a in range(n):
            row = i * n + a
            ri, rj = rate[a] / lam[i], rate[a] / lam[j]
            C[row, row] -= sigma[i] + ri
            C[row, j * n + a] += rj
            C[row, i * n:(i + 1) * n] += 0.5 * c[i] * sigma[i] * w
    mu2 = np.concatenate([mu, mu])
    w2 = np.concatenate([w, w])
    M = C / mu2[:, None]
    ev, V = np.linalg.eig(M)
    if np.max(np.abs(ev.imag)) > 1e-9 * max(1.0, np.max(np.abs(ev.real))):
        raise ValueError("complex LP eigenvalues")
    ev = ev.real
    V = V.real
    ref = np.where(ev > 0.0, L, 0.0)
    volume = source == "volume"
    if volume:
        q = np.repeat(p, n) / (L * np.sum(w))
        psi_p = -np.linalg.solve(C, q)  # constant particular solution
    else:
        psi_p = np.zeros(K)
    f = 1.0 / np.sum((w * mu)[mu > 0])
    A = np.zeros((K, K))
    b = np.zeros(K)
    for r in range(K):
        i = r // n
        if mu2[r] > 0:
            A[r] = V[r] * np.exp(ev * (0.0 - ref))
            b[r] = (0.0 if volume else p[i] * f) - psi_p[r]
        else:
            A[r] = V[r] * np.exp(ev * (L - ref))
            b[r] = -psi_p[r]
    coef = np.linalg.solve(A, b)
    psi0 = V @ (coef * np.exp(ev * (0.0 - ref))) + psi_p
    psiL = V @ (coef * np.exp(ev * (L - ref))) + psi_p
    R = float(np.sum((w2 * np.abs(mu2) * psi0)[mu2 < 0]))
    T = float(np.sum((w2 * mu2 * psiL)[mu2 > 0]))
    out = {"R": R, "T": T, "A": 1.0 - R - T, "Lk": 0.5 * (R + T)}
    full = _integral_exp(ev, 0.0, L, ref) * coef
    track = []
    for i in range(2):
        sl = slice(i * n, (i + 1) * n)
        track.append(float(w @ (V[sl] @ full)) + L * float(w @ psi_p[sl]))
    out["track"] = tuple(track)
    out["total_flux"] = track[0] + track[1]
    # absorption from the track-length estimator, sum_i Sigma_a,i * track_i
    out["A_track"] = float(sum(sigma[i] * (1.0 - c[i]) * track[i] for i in range(2)))
    if nbins > 0:
        edges = np.arange(nbins + 1) * L / nbins
        sw = w2 @ V  # angular integral of each mode
        flux = np.empty(nbins)
        for k in range(nbins):
            flux[k] = np.sum(sw * coef * _integral_exp(ev, edges[k], edges[k + 1], ref))
        out["flux"] = flux / (L / nbins) + float(w2 @ psi_p)
    return out
