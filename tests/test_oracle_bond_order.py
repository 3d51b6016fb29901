"""Pins for the oracle's bond order (Sec. 2, Eq. 1-7) and elementary functions.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code: the normalisation b(0) = 1,
the p -> infinity limit (Eq. 6), the Tersoff form (Eq. 1), the expanded L = 2
form as printed (Eq. 7), monotonicity, derivative identities and the angular
minima quoted in Sec. 3.1.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def _rand_params(rng, L, shape=()):
    g = rng.uniform(0.3, 3.0, size=shape + (L,))
    n = rng.uniform(0.6, 1.6, size=shape + (L,))
    sigma = rng.uniform(0.4, 1.5, size=shape)
    p = rng.uniform(0.5, 4.0, size=shape)
    return g, n, sigma, p


@pytest.mark.parametrize("L", [1, 2, 3])
def test_b_is_one_without_environment(L):
    """Sec. 2 after Eq. 5: G normalises b to 1 when every zeta_l = 0."""
    rng = np.random.default_rng(10 + L)
    g, n, sigma, p = _rand_params(rng, L, (50,))
    b, db = O.bond_order(np.zeros((50, L)), g, n, sigma, p)
    assert np.allclose(b, GOLDEN["b_at_zero_zeta"]["value"], rtol=0, atol=1e-14)
    assert np.all(db == 0.0)


def test_b_maximum_is_one():
    """Sec. 2 after Eq. 7: the maximum of b_ij is 1 (b decreases in every zeta_l)."""
    rng = np.random.default_rng(3)
    g, n, sigma, p = _rand_params(rng, 2, (2000,))
    z = rng.exponential(2.0, size=(2000, 2))
    b, db = O.bond_order(z, g, n, sigma, p)
    assert np.all(b <= 1.0) and np.all(b > 0.0)
    assert np.all(db < 0.0)


def test_eq1_tersoff_reduction():
    """L = 1, g_1 = 1: Eq. 3-5 reduce to Eq. 1, b' = (1 + zeta^n)^(-1/(2 sigma))."""
    rng = np.random.default_rng(5)
    z = rng.exponential(1.5, size=(300, 1))
    n = rng.uniform(0.6, 1.6, size=(300, 1))
    sigma = rng.uniform(0.4, 1.5, size=300)
    p = rng.uniform(0.5, 4.0, size=300)
    b, _ = O.bond_order(z, np.ones((300, 1)), n, sigma, p)
    ref = (1.0 + z[:, 0] ** n[:, 0]) ** (-1.0 / (2.0 * sigma))
    assert np.allclose(b, ref, rtol=1e-13, atol=0)
    assert np.allclose(O.bond_order_tersoff(z[:, 0], n[:, 0], sigma), ref, rtol=1e-15)


def test_eq7_expanded_form_as_printed():
    """Eq. 7 (L = 2), with the exponent read as 1/(2 sigma p) and G from the
    b(0) = 1 normalisation, equals Eq. 3-5."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        g1, g2 = rng.uniform(0.3, 3.0, 2)
        n1, n2 = rng.uniform(0.6, 1.6, 2)
        sig = rng.uniform(0.4, 1.5)
        p = GOLDEN["p"]["value"]
        z1, z2 = rng.exponential(1.5, 2)
        G = (g1 ** -p + g2 ** -p) ** (-1.0 / (2 * sig * p))
        eq7 = G * ((g1 + z1 ** n1) ** -p + (g2 + z2 ** n2) ** -p) ** (1.0 / (2 * sig * p))
        b, _ = O.bond_order(np.array([z1, z2]), np.array([g1, g2]), np.array([n1, n2]), sig, p)
        assert abs(b - eq7) <= 1e-14 * eq7


@pytest.mark.parametrize("p", [8.0, 32.0, 96.0])
def test_eq6_p_to_infinity(p):
    """Eq. 6: as p -> inf, b -> max_l G (g_l + zeta_l^n_l)^(-1/(2 sigma)).
    For finite p, |log b_p - log b_inf| <= log(L) / (2 sigma p)."""
    rng = np.random.default_rng(int(p))
    g, n, sigma, _ = _rand_params(rng, 2, (500,))
    z = rng.exponential(1.0, size=(500, 2))
    b, _ = O.bond_order(z, g, n, sigma, np.full(500, p))
    binf = O.bond_order_pinf(z, g, n, sigma)
    bound = math.log(2.0) / (2.0 * sigma * p)
    assert np.all(np.abs(np.log(b) - np.log(binf)) <= bound + 1e-12)


def test_p1_reciprocal_sum_reading():
    """p = 1: Eq. 4 gives zhat_tot = 1 / sum_l (1/zhat_l) (reading of the
    'geometric mean' remark after Eq. 6: the equation governs)."""
    rng = np.random.default_rng(11)
    g, n, sigma, _ = _rand_params(rng, 2, (100,))
    z = rng.exponential(1.0, size=(100, 2))
    b, _ = O.bond_order(z, g, n, sigma, np.ones(100))
    zh = g + z ** n
    G = (1.0 / np.sum(1.0 / g, -1)) ** (1.0 / (2 * sigma))
    ref = G * (1.0 / np.sum(1.0 / zh, -1)) ** (-1.0 / (2 * sigma))
    assert np.allclose(b, ref, rtol=1e-13)


def test_db_dzeta_finite_difference():
    rng = np.random.default_rng(13)
    g, n, sigma, p = _rand_params(rng, 2, (200,))
    z = rng.uniform(0.2, 4.0, size=(200, 2))
    _, db = O.bond_order(z, g, n, sigma, p)
    h = 1e-6
    for l in range(2):
        e = np.zeros(2)
        e[l] = h
        bp, _ = O.bond_order(z + e, g, n, sigma, p)
        bm, _ = O.bond_order(z - e, g, n, sigma, p)
        assert np.allclose(db[:, l], (bp - bm) / (2 * h), rtol=1e-7, atol=1e-12)


def test_cutoff_function():
    R, S = 2.2, 2.55
    r = np.linspace(1.0, 3.0, 4001)
    f, df = O.cutoff(r, R, S)
    assert np.all(f[r < R] == 1.0) and np.all(f[r >= S] == 0.0)
    assert np.all(np.diff(f) <= 0.0)
    # continuity at R and S, midpoint value 1/2
    assert abs(O.cutoff(0.5 * (R + S), R, S)[0] - 0.5) < 1e-15
    h = 1e-6
    rr = np.linspace(R + 0.01, S - 0.01, 50)
    fd = (O.cutoff(rr + h, R, S)[0] - O.cutoff(rr - h, R, S)[0]) / (2 * h)
    assert np.allclose(O.cutoff(rr, R, S)[1], fd, rtol=1e-7, atol=1e-10)


def test_taper_polynomial():
    """T(0) = 1, T(1) = 0 and T', T'', T''' vanish at both ends; checked with
    numpy's polynomial class, not the oracle's closed forms."""
    poly = np.polynomial.Polynomial([1, 0, 0, 0, -35, 84, -70, 20])
    assert poly(0.0) == 1.0 and abs(poly(1.0)) < 1e-14
    for k in (1, 2, 3):
        d = poly.deriv(k)
        assert abs(d(0.0)) < 1e-12 and abs(d(1.0)) < 1e-10
    x = np.linspace(0, 0.999, 300)
    T, dT = O.taper(x)
    assert np.allclose(T, poly(x), rtol=0, atol=1e-13)
    assert np.allclose(dT, poly.deriv(1)(x), rtol=0, atol=1e-11)
    assert np.all(O.taper(np.array([1.0, 1.5]))[0] == 0.0)


def test_coulomb_kernel_limits():
    """Far inside a very large cutoff and with negligible shielding the kernel
    is Coulomb's law k_e / r; dK/dr matches a central difference."""
    r = np.linspace(1.0, 5.0, 50)
    K, _ = O.coulomb_kernel(r, 1e6, 1e6, 14.399645)
    assert np.allclose(K, 14.399645 / r, rtol=1e-12)
    h = 1e-6
    K1, dK = O.coulomb_kernel(r, 0.7, 8.0, 14.399645)
    fd = (O.coulomb_kernel(r + h, 0.7, 8.0, 14.399645)[0] - O.coulomb_kernel(r - h, 0.7, 8.0, 14.399645)[0]) / (2 * h)
    assert np.allclose(dK, fd, rtol=1e-7, atol=1e-10)
    assert O.coulomb_kernel(np.array([8.0, 9.0]), 0.7, 8.0, 14.399645)[0].max() == 0.0


def test_angular_minima_match_paper():
    """Sec. 3.1: the minimum bond angle of zeta_1 is 180 deg and that of
    zeta_2 is 127 deg. The synthetic parameter set honours both for every
    type triplet."""
    P = O.tables(st.load_params("p1"))
    theta = np.radians(np.linspace(60.0, 180.0, 120001))
    ct = np.cos(theta)
    want = [GOLDEN["angle_min_zeta1_deg"]["value"], GOLDEN["angle_min_zeta2_deg"]["value"]]
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for l in range(2):
                    val, _ = O.angular(ct, P.gam[a, b, c, l], P.c[a, b, c, l],
                                       P.d[a, b, c, l], P.h[a, b, c, l])
                    th_min = math.degrees(theta[np.argmin(val)])
                    assert abs(th_min - want[l]) < 0.01, (a, b, c, l, th_min)


def test_angular_derivative():
    ct = np.linspace(-1, 1, 101)
    h = 1e-6
    v, dv = O.angular(ct, 0.3, 3.0, 1.5, -0.6)
    fd = (O.angular(ct + h, 0.3, 3.0, 1.5, -0.6)[0] - O.angular(ct - h, 0.3, 3.0, 1.5, -0.6)[0]) / (2 * h)
    assert np.allclose(dv, fd, rtol=1e-7, atol=1e-10)
