"""Pins that the synthetic parameter set P1 keeps the tetrahedral SiC
lattices the paper simulates (Sec. 3: 4H-SiC(0001) substrates held for
nanoseconds at 2500-3000 K; the fit of Sec. 2 targets SiC phases) as stable
minima, checked on the oracle:

* ideal 3C-SiC at a = 4.36 A: every vibration of a 64-atom cell (the zone
  centre and the zone-boundary points of the cubic cell) has a positive
  force constant; only the three translations are zero;
* ideal 4H-SiC (periodic, 32 atoms): a local minimum within 1e-3 A of the
  ideal sites, positive force constants there;
* the Born criteria of a cubic crystal, C11 - C12 > 0, C11 + 2 C12 > 0 and
  C44 > 0, with C44 from a [110]-oriented cell and the internal relaxation
  of the C sublattice included (checked against an explicit relaxation);
* a 64-atom crystal at 300 K releases no potential energy over 300 NVE steps;
* the same pins fail for sets with a planted defect: the channel-2 angle
  minimum at 60 degrees instead of the paper's 127, or both minima at 90
  degrees instead of 180 and 127 (negative force constants and C44).

Force constants are central differences of the oracle's analytic forces.
"""
import copy

import numpy as np

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")
EV_A3_TO_GPA = 160.21766208
KT_300 = O.KB * 300.0


def _force_constants(s, params, h=1e-3):
    """Phi[a, b] = -dF_b / dx_a (3N x 3N) by central differences."""
    n = s.n
    Phi = np.zeros((3 * n, 3 * n))
    for a in range(n):
        for d in range(3):
            xp, xm = s.x.copy(), s.x.copy()
            xp[a, d] += h
            xm[a, d] -= h
            Fp = O.evaluate(xp, s.types, s.box, s.pbc, params)["F"]
            Fm = O.evaluate(xm, s.types, s.box, s.pbc, params)["F"]
            Phi[3 * a + d] = -(Fp - Fm).ravel() / (2 * h)
    return Phi


def _stress_xx_slope(make, params, h=2e-3):
    """d sigma / d eps for the strain a structure factory applies:
    sigma = -W / V with W the oracle's virial (positive under compression)."""
    out = []
    for e in (h, -h):
        s = make(e)
        r = O.evaluate(s.x, s.types, s.box, s.pbc, params)
        out.append(r["virial"] / np.prod(s.box))
    return -(out[0] - out[1]) / (2 * h)


def _cubic_cell(f):
    s = st.sic_3c(1, 4.36, 0.0)
    return st.Structure("strained", s.x * f, s.types, s.box * f, s.pbc)


def _c11_c12(params):
    d = _stress_xx_slope(lambda e: _cubic_cell(np.array([1.0 + e, 1.0, 1.0])), params) * EV_A3_TO_GPA
    return d[0, 0], d[1, 1]


def _c44(params):
    """C44 from C'11 = (C11 + C12)/2 + C44 of the [110] cell, clamped and with
    the internal coordinates relaxed: C_relaxed = C_clamped - L Phi^+ L / V,
    L = dF/d eps at fixed fractional positions."""
    C11, C12 = _c11_c12(params)
    s0 = st.sic_3c_110()
    h = 1e-3
    rp = O.evaluate(*(lambda s: (s.x, s.types, s.box, s.pbc))(st.sic_3c_110(stretch_x=h)), params)
    rm = O.evaluate(*(lambda s: (s.x, s.types, s.box, s.pbc))(st.sic_3c_110(stretch_x=-h)), params)
    Vp = np.prod(st.sic_3c_110(stretch_x=h).box)
    Vm = np.prod(st.sic_3c_110(stretch_x=-h).box)
    c_clamped = -(rp["virial"][0, 0] / Vp - rm["virial"][0, 0] / Vm) / (2 * h)
    L = (rp["F"] - rm["F"]).ravel() / (2 * h)
    Phi = _force_constants(s0, params, h=1e-4)
    Phi = 0.5 * (Phi + Phi.T)
    c_relaxed = c_clamped - L @ np.linalg.pinv(Phi, rcond=1e-8) @ L / np.prod(s0.box)
    half = 0.5 * (C11 + C12)
    return c_relaxed * EV_A3_TO_GPA - half, c_clamped * EV_A3_TO_GPA - half


def test_3c_sic_every_vibration_of_a_64_atom_cell_is_stable():
    s = st.sic_3c(2, 4.36, 0.0)
    Phi = _force_constants(s, P1)
    # forces are exact derivatives of one energy: the constants are symmetric
    assert np.max(np.abs(Phi - Phi.T)) < 1e-5 * np.max(np.abs(Phi))
    ev = np.linalg.eigvalsh(0.5 * (Phi + Phi.T))
    assert np.all(np.abs(ev[:3]) < 1e-6), ev[:4]          # translations
    assert ev[3] > 1.0, ev[:8]                            # eV/A^2


def test_4h_sic_is_a_local_minimum():
    s = st.sic_4h_bulk(2, 1, 1)
    x = s.x.copy()
    # Newton steps on the ideal sites: the charge interaction of the 4H stacking
    # leaves small residual forces, so the minimum sits next to them
    for _ in range(3):
        r = O.evaluate(x, s.types, s.box, s.pbc, P1)
        cur = st.Structure("4H", x, s.types, s.box, s.pbc)
        Phi = _force_constants(cur, P1, h=1e-4)
        Phi = 0.5 * (Phi + Phi.T)
        x = x + (np.linalg.pinv(Phi, rcond=1e-8) @ r["F"].ravel()).reshape(-1, 3)
    r = O.evaluate(x, s.types, s.box, s.pbc, P1)
    assert np.max(np.abs(r["F"])) < 1e-6
    assert np.max(np.abs(x - s.x)) < 1e-3
    ev = np.linalg.eigvalsh(Phi)
    assert np.all(np.abs(ev[:3]) < 1e-5) and ev[3] > 1.0, ev[:6]


def test_born_criteria_3c_sic():
    C11, C12 = _c11_c12(P1)
    C44, C44_clamped = _c44(P1)
    assert C11 - C12 > 50.0 and C11 + 2 * C12 > 0.0 and C44 > 50.0, (C11, C12, C44)
    # internal relaxation can only soften the shear
    assert C44 < C44_clamped
    # the bulk modulus from a hydrostatic strain agrees with (C11 + 2 C12)/3
    B = np.trace(_stress_xx_slope(lambda e: _cubic_cell(np.full(3, 1.0 + e)), P1)) / 9.0 * EV_A3_TO_GPA
    assert abs(B - (C11 + 2 * C12) / 3) < 1e-3 * B


def test_c44_relaxation_matches_an_explicit_relaxation():
    """C'11 of the [110] cell with its atoms relaxed by Newton steps at each
    strain agrees with the force-constant formula used above."""
    h = 2e-3
    sig = []
    for e in (h, -h):
        s = st.sic_3c_110(stretch_x=e)
        x = s.x.copy()
        for _ in range(4):
            r = O.evaluate(x, s.types, s.box, s.pbc, P1)
            Phi = _force_constants(st.Structure("c", x, s.types, s.box, s.pbc), P1, h=1e-4)
            x = x + (np.linalg.pinv(0.5 * (Phi + Phi.T), rcond=1e-8) @ r["F"].ravel()).reshape(-1, 3)
        r = O.evaluate(x, s.types, s.box, s.pbc, P1)
        assert np.max(np.abs(r["F"])) < 1e-8
        sig.append(r["virial"][0, 0] / np.prod(s.box))
    c_relaxed = -(sig[0] - sig[1]) / (2 * h) * EV_A3_TO_GPA
    C11, C12 = _c11_c12(P1)
    C44, _ = _c44(P1)
    assert abs((c_relaxed - 0.5 * (C11 + C12)) - C44) < 1e-2 * C44


def test_crystal_at_300K_releases_no_potential_energy():
    s = st.sic_3c(2, 4.36, 0.05, seed=1)
    v = st.maxwell_boltzmann(s.types, 300.0, seed=101)
    e_pot0 = O.evaluate(s.x, s.types, s.box, s.pbc, P1)["E"]
    e_tot0 = e_pot0 + O.kinetic_energy(v, s.types, P1)
    x = s.x
    e_pot = []
    for _ in range(10):
        x, v, _, et = O.velocity_verlet(x, v, s.types, s.box, s.pbc, P1, 0.5, 30)
        e_pot.append(O.evaluate(x, s.types, s.box, s.pbc, P1)["E"])
        assert np.max(np.abs(et - e_tot0)) / s.n < 1e-4
    # equipartition moves E_pot up by about kT/2 per atom at most; a
    # collapsing lattice releases several kT
    assert abs(np.mean(e_pot) - e_pot0) / s.n < KT_300
    assert np.max(np.abs(np.array(e_pot) - e_pot0)) / s.n < 2 * KT_300


def _with_triplets(fn):
    """P1 with a change to every triplet row, A_SiC then re-solved so that
    ideal 3C-SiC stays stress-free at 4.36 A (the pressure is linear in A:
    only the repulsive term carries it)."""
    bad = copy.deepcopy(P1)
    for t in bad["triplet"].values():
        fn(t)
    s = st.sic_3c(1, 4.36, 0.0)

    def pressure(A):
        bad["pair"]["SiC"]["A"] = A
        return np.trace(O.evaluate(s.x, s.types, s.box, s.pbc, bad)["virial"])

    A0 = P1["pair"]["SiC"]["A"]
    p0, p1 = pressure(A0), pressure(2.0 * A0)
    bad["pair"]["SiC"]["A"] = A0 - p0 * A0 / (p1 - p0)
    return bad


def test_pins_catch_an_unstable_lattice():
    """Planted defects the pins above must reject: wrong angle minima."""
    s = st.sic_3c(1, 4.36, 0.0)
    ev1 = np.linalg.eigvalsh(_force_constants(s, P1))
    assert ev1[3] > 1.0
    for bad in (_with_triplets(lambda t: t.__setitem__("h", [t["h"][0], 0.5])),
                _with_triplets(lambda t: t.__setitem__("h", [0.0, 0.0]))):
        ev = np.linalg.eigvalsh(_force_constants(s, bad))
        assert ev[0] < -1.0, ev[:6]
        C44, _ = _c44(bad)
        assert C44 < 0.0, C44
