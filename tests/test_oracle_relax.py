"""Pins of the oracle's energy minimiser (FIRE on E(x) = min_q E(x, q)):
the minima of small systems whose energy is a closed form of one distance,
a crystal already at a stationary point, frozen atoms, descent.

* Si-C dimer inside R: E(r) is the 2x2 KKT closed form; FIRE must stop at
  its minimiser r* (found here by a scalar minimisation of the closed form).
* Linear Si3 (all charges zero, ends beyond S of each other): E(d) =
  3 E0 + 2 f_R(d) - f_A(d) - b_mid f_A(d) with b_mid from Eq. 7 at
  zeta_l = ang_l(-1); symmetric forces keep the chain linear and
  symmetric, so FIRE must stop at the minimiser d* of that closed form.
* Ideal 3C-SiC: every force vanishes by symmetry, so no iteration is taken.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")
OPEN = np.array([False] * 3)


def _dimer_energy(r):
    pr, se, co = P1["pair"]["SiC"], P1["self"], P1["coulomb"]
    fA = pr["B"] * math.exp(-pr["lambda2"] * r)
    fR = pr["A"] * math.exp(-pr["lambda1"] * r)
    gam = math.sqrt(co["gamma"][0] * co["gamma"][1])
    xr = r / co["r_coul"]
    taper = 1 - 35 * xr ** 4 + 84 * xr ** 5 - 70 * xr ** 6 + 20 * xr ** 7
    K = co["k_e"] * taper / (r ** 3 + gam ** -3) ** (1 / 3)
    q = (se["chi"][1] - se["chi"][0]) / (2 * se["J"][0] + 2 * se["J"][1] + 8 * pr["kappa"] * fA - 2 * K)
    return (se["E0"][0] + se["E0"][1] + (se["chi"][0] - se["chi"][1]) * q + (se["J"][0] + se["J"][1]) * q * q
            + fR - (1 - pr["kappa"] * 4 * q * q) * fA - q * q * K)


def _si3_energy(d):
    pr, bo, tp = P1["pair"]["SiSi"], P1["bond"]["SiSi"], P1["triplet"]["SiSiSi"]
    fR = pr["A"] * math.exp(-pr["lambda1"] * d)
    fA = pr["B"] * math.exp(-pr["lambda2"] * d)
    p, sg = bo["p"], bo["sigma"]
    terms, norm = 0.0, 0.0
    for l in range(2):
        c2, d2 = tp["c"][l] ** 2, tp["d"][l] ** 2
        zeta = tp["gamma"][l] * (1 + c2 / d2 - c2 / (d2 + (tp["h"][l] + 1.0) ** 2))
        terms += (bo["g"][l] + zeta ** bo["n"][l]) ** (-p)
        norm += bo["g"][l] ** (-p)
    b_mid = (terms / norm) ** (1.0 / (2.0 * sg * p))
    return 3 * P1["self"]["E0"][0] + 2 * fR - fA - b_mid * fA


def test_dimer_reaches_closed_form_minimum():
    rs = minimize_scalar(_dimer_energy, bounds=(1.0, 2.19), method="bounded", options={"xatol": 1e-12})
    assert 1.1 < rs.x < 2.1
    x = np.array([[10.0, 10.0, 10.0], [12.0, 10.3, 9.8]])
    xf, it, E, ok = O.fire_minimize(x, np.array([0, 1]), np.full(3, 40.0), OPEN, P1, fmax=1e-7, max_iter=5000)
    assert ok and it > 0
    r = np.linalg.norm(xf[1] - xf[0])
    assert r == pytest.approx(rs.x, abs=1e-7)
    assert E[-1] == pytest.approx(_dimer_energy(rs.x), abs=1e-10)


def test_linear_si3_reaches_closed_form_minimum():
    rs = minimize_scalar(_si3_energy, bounds=(1.9, 2.44), method="bounded", options={"xatol": 1e-12})
    assert 1.9 < rs.x < 2.44 and 2 * rs.x > P1["pair"]["SiSi"]["S"]
    d0 = 2.3
    x = np.array([[10.0, 10.0, 10.0], [10.0 + d0, 10.0, 10.0], [10.0 + 2 * d0, 10.0, 10.0]])
    xf, it, E, ok = O.fire_minimize(x, np.zeros(3, int), np.full(3, 40.0), OPEN, P1, fmax=1e-7, max_iter=5000)
    assert ok
    d1, d2 = np.linalg.norm(xf[1] - xf[0]), np.linalg.norm(xf[2] - xf[1])
    assert d1 == pytest.approx(rs.x, abs=1e-7) and d2 == pytest.approx(rs.x, abs=1e-7)


def test_ideal_crystal_takes_no_iteration():
    s = st.sic_3c(2, 4.36, 0.0, seed=1)
    xf, it, E, ok = O.fire_minimize(s.x, s.types, s.box, s.pbc, P1, fmax=1e-6)
    assert ok and it == 0 and np.array_equal(xf, s.x)


def test_descent_and_frozen_atoms():
    s = st.stepped_slab_small(6, 3, 4)
    xf, it, E, ok = O.fire_minimize(s.x, s.types, s.box, s.pbc, P1, frozen=s.frozen, fmax=1e-9, n_iter=40)
    assert it == 40 and E[-1] < E[0]
    assert np.array_equal(xf[s.frozen], s.x[s.frozen])
    assert np.max(np.abs(xf[~s.frozen] - s.x[~s.frozen])) > 1e-3
