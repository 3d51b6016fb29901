"""Pins of the oracle's Si-desorption screening (Sec. 3.3: the energy change
when one atom is eliminated, the rest held in place, charges re-minimised):
closed forms of small systems, and symmetry.

* Si-C dimer: removing either atom leaves one isolated neutral atom (q = 0,
  E = E0), so dE = E0_Si + E0_C - E_dimer, with E_dimer the 2x2 KKT closed
  form of the dimer.
* Linear Si3 (spacing d < R, ends beyond S of each other): all charges are
  zero (equal electronegativities: q = 0 solves H q + chi 1 = mu 1 with
  sum q = 0), the end bonds have b = 1 (no third atom in range) and the
  middle atom's bonds see the other end at 180 degrees. Removing an end
  atom therefore gives dE = -f_R(d) + b_mid f_A(d), with b_mid from Eq. 7
  at zeta_l = ang_l(-1).
* An all-Si cluster plus one Si far beyond every cutoff: q = 0 everywhere,
  so removing the far atom changes nothing: dE = 0.
* In an ideal 3C-SiC crystal every Si site is equivalent: equal dE.
"""
import math

import numpy as np
import pytest

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


@pytest.mark.parametrize("r", [1.75, 1.9, 2.15])   # inside R: f_c = 1
@pytest.mark.parametrize("i", [0, 1])
def test_dimer(r, i):
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    dE = O.removal_energy(x, np.array([0, 1]), np.full(3, 40.0), OPEN, P1, i)
    ref = P1["self"]["E0"][0] + P1["self"]["E0"][1] - _dimer_energy(r)
    assert dE == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("d", [2.2, 2.35, 2.44])
def test_linear_si3_end_atom(d):
    pr, bo, tp = P1["pair"]["SiSi"], P1["bond"]["SiSi"], P1["triplet"]["SiSiSi"]
    x = np.array([[10.0, 10.0, 10.0], [10.0 + d, 10.0, 10.0], [10.0 + 2 * d, 10.0, 10.0]])
    t = np.zeros(3, int)
    dE = O.removal_energy(x, t, np.full(3, 40.0), OPEN, P1, 2)
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
    assert dE == pytest.approx(-fR + b_mid * fA, rel=1e-12)


def test_far_atom_of_an_all_si_system():
    s = st.sic_3c(1, 4.36, 0.1, seed=5)
    si = s.types == 0
    x = np.concatenate([s.x[si] + 10.0, [[60.0, 60.0, 60.0]]])
    t = np.zeros(len(x), int)
    o = O.evaluate(x, t, np.full(3, 80.0), OPEN, P1)
    assert np.max(np.abs(o["q"])) < 1e-12
    dE = O.removal_energy(x, t, np.full(3, 80.0), OPEN, P1, len(x) - 1)
    assert abs(dE) < 1e-10


def test_equivalent_sites_in_ideal_crystal():
    s = st.sic_3c(2, 4.36, 0.0, seed=1)
    si = np.nonzero(s.types == 0)[0][:4]
    dE, _ = O.desorption_screen(s.x, s.types, s.box, s.pbc, P1, si)
    assert np.ptp(dE) < 1e-9 * abs(dE[0])


def test_coordination():
    s = st.sic_3c(2, 4.36, 0.05, seed=3)
    assert np.all(O.coordination(s.x, s.types, s.box, s.pbc, P1) == 4)
    slab = st.sic_4h_slab(4, 2, 3)
    c = O.coordination(slab.x, slab.types, slab.box, slab.pbc, P1)
    top = slab.x[:, 2] > slab.x[:, 2].max() - 0.1
    assert np.all(slab.types[top] == 0) and np.all(c[top] == 3)
    assert np.all(c[~top & (slab.x[:, 2] > slab.x[:, 2].min() + 0.1)] == 4)
