"""Pins for the oracle's energy, charges, forces and virial on whole systems.

Independent checks: a closed-form dimer (energy and the 2x2 charge KKT), a
pure-Python brute-force loop over atoms, images and triplets, the brute-force
vs k-d tree pair enumeration, periodic-supercell consistency, invariances,
Newton's third law, electronegativity equalisation, finite differences of the
energy (forces to 1e-6 relative, virial by homogeneous strain), zero pressure
of 3C-SiC at a = 4.36 A for the synthetic set, and positive-definiteness of
the charge Hessian.
"""
import math

import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")
T0 = O.tables(P1)


def _cluster(n, seed, box=30.0, min_sep=1.6, spread=4.0):
    rng = np.random.default_rng(seed)
    xs = []
    while len(xs) < n:
        c = rng.uniform(-spread, spread, 3)
        if all(np.linalg.norm(c - y) >= min_sep for y in xs):
            xs.append(c)
    x = np.array(xs) + box / 2
    t = rng.integers(0, 2, n).astype(np.int32)
    return x, t, np.full(3, box), np.array([False, False, False])


# ---------------------------------------------------------------------------
def test_pair_enumeration_brute_vs_kdtree():
    for s in (st.sic_3c(2, 4.36, 0.05, seed=2), st.sic_4h_slab(4, 2, 4, step="strip"),
              st.sic_3c(1, 4.36, 0.1, seed=3)):
        for rc in (2.9, 8.0):
            a = O.pairs_bruteforce(s.x, s.box, s.pbc, rc)
            b = O.pairs_kdtree(s.x, s.box, s.pbc, rc)
            for u, v in zip(a, b):
                assert np.array_equal(u.shape, v.shape)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            assert np.array_equal(a[2], b[2])
            assert np.allclose(a[3], b[3], atol=1e-12)


def test_self_images_in_small_box():
    """A 2-atom cell of edge 3 A holds periodic self-images inside 8 A."""
    x = np.array([[0.1, 0.2, 0.3], [1.5, 1.5, 1.5]])
    i, j, n, u = O.pairs_bruteforce(x, np.full(3, 3.0), np.array([True] * 3), 8.0)
    self_img = (i == j)
    assert self_img.sum() > 0
    r = np.linalg.norm(u[self_img], axis=1)
    assert np.allclose(np.sort(r)[:6], 3.0)


# ---------------------------------------------------------------------------
def test_dimer_closed_form():
    """Isolated Si-C dimer inside R: no third atom, so zeta = 0 and b = 1
    (Sec. 2). With q_Si = -q_C = q the energy is quadratic in q and the
    minimiser is q = (chi_C - chi_Si) / (2 J_Si + 2 J_C + 8 kappa f_A - 2 K)."""
    pr = P1["pair"]["SiC"]
    se, co = P1["self"], P1["coulomb"]
    for r in (1.7, 1.9, 2.1):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        res = O.evaluate(x, np.array([0, 1]), np.full(3, 40.0), np.array([False] * 3), P1)
        fA = pr["B"] * math.exp(-pr["lambda2"] * r)
        fR = pr["A"] * math.exp(-pr["lambda1"] * r)
        gam = math.sqrt(co["gamma"][0] * co["gamma"][1])
        xr = r / co["r_coul"]
        taper = 1 - 35 * xr ** 4 + 84 * xr ** 5 - 70 * xr ** 6 + 20 * xr ** 7
        K = co["k_e"] * taper / (r ** 3 + gam ** -3) ** (1 / 3)
        q = (se["chi"][1] - se["chi"][0]) / (2 * se["J"][0] + 2 * se["J"][1]
                                             + 8 * pr["kappa"] * fA - 2 * K)
        assert np.allclose(res["q"], [q, -q], rtol=1e-13, atol=1e-15)
        assert np.allclose(res["b"], 1.0, atol=1e-15)
        E = (se["E0"][0] + se["E0"][1] + (se["chi"][0] - se["chi"][1]) * q
             + (se["J"][0] + se["J"][1]) * q * q
             + fR - (1 - pr["kappa"] * 4 * q * q) * fA - q * q * K)
        assert abs(res["E"] - E) < 1e-12 * abs(E)


def _energy_bruteforce(x, types, box, pbc, q, P):
    """Pure-Python loops: every atom i, every image of every atom j, every
    third image-atom k; written independently of the vectorised oracle."""
    N = len(x)
    box = np.asarray(box, float)
    rmax = max(P.r_coul, float(P.S.max()))
    nimg = [int(math.ceil(rmax / box[d])) if pbc[d] else 0 for d in range(3)]
    imgs = [(a, b, c) for a in range(-nimg[0], nimg[0] + 1)
            for b in range(-nimg[1], nimg[1] + 1) for c in range(-nimg[2], nimg[2] + 1)]

    def nbrs(i, rc):
        out = []
        for j in range(N):
            for im in imgs:
                u = x[j] + np.array(im) * np.where(pbc, box, 0) - x[i]
                r = math.sqrt(u @ u)
                if 0 < r < rc:
                    out.append((j, u, r))
        return out

    E = 0.0
    for i in range(N):
        ti = types[i]
        E += P.E0[ti] + P.chi[ti] * q[i] + P.J[ti] * q[i] ** 2
        for j, u, r in nbrs(i, P.r_coul):
            tj = types[j]
            gam = math.sqrt(P.gam_c[ti] * P.gam_c[tj])
            xr = r / P.r_coul
            tap = 1 - 35 * xr ** 4 + 84 * xr ** 5 - 70 * xr ** 6 + 20 * xr ** 7
            E += 0.5 * q[i] * q[j] * P.k_e * tap / (r ** 3 + gam ** -3) ** (1 / 3)
        cov = [(j, u, r) for j, u, r in nbrs(i, float(P.S.max())) if r < P.S[ti, types[j]]]
        for a, (j, uj, rj) in enumerate(cov):
            tj = types[j]
            R, S = P.R[ti, tj], P.S[ti, tj]
            fc = 1.0 if rj < R else 0.5 * (1 + math.cos(math.pi * (rj - R) / (S - R)))
            zeta = [0.0] * P.L
            for bidx, (k, uk, rk) in enumerate(cov):
                if bidx == a:
                    continue
                tk = types[k]
                Rk, Sk = P.R[ti, tk], P.S[ti, tk]
                fck = 1.0 if rk < Rk else 0.5 * (1 + math.cos(math.pi * (rk - Rk) / (Sk - Rk)))
                cth = (uj @ uk) / (rj * rk)
                for l in range(P.L):
                    g_, c_, d_, h_ = (P.gam[ti, tj, tk, l], P.c[ti, tj, tk, l],
                                      P.d[ti, tj, tk, l], P.h[ti, tj, tk, l])
                    ang = g_ * (1 + c_ ** 2 / d_ ** 2 - c_ ** 2 / (d_ ** 2 + (h_ - cth) ** 2))
                    zeta[l] += fck * ang * math.exp(P.alpha[ti, tj, tk, l] * (rj - rk))
            sig, p = P.sigma[ti, tj], P.p[ti, tj]
            ssum = sum((P.g[ti, tj, l] + (zeta[l] ** P.n[ti, tj, l] if zeta[l] > 0 else 0.0)) ** -p
                       for l in range(P.L))
            s0 = sum(P.g[ti, tj, l] ** -p for l in range(P.L))
            b = (ssum / s0) ** (1 / (2 * sig * p))
            cq = 1 - P.kappa[ti, tj] * (q[i] - q[j]) ** 2
            E += 0.5 * fc * (P.A[ti, tj] * math.exp(-P.lam1[ti, tj] * rj)
                             - cq * b * P.B[ti, tj] * math.exp(-P.lam2[ti, tj] * rj))
    return E


@pytest.mark.parametrize("case", ["cluster", "periodic_small"])
def test_energy_bruteforce_loops(case):
    rng = np.random.default_rng(21)
    if case == "cluster":
        x, t, box, pbc = _cluster(9, 4, spread=2.5, min_sep=1.5)
    else:
        s = st.sic_3c(1, 4.36, 0.12, seed=5)
        x, t, box, pbc = s.x, s.types, s.box, s.pbc
        t = t.copy()
        t[[1, 6]] = 1 - t[[1, 6]]      # mixed-type environment
    q = rng.normal(0, 0.3, len(x))
    sysm = O.System(x, t, box, pbc, P1)
    E = sysm.energy(q)
    Eb = _energy_bruteforce(x, t, box, pbc, q, T0)
    assert abs(E - Eb) <= 1e-11 * max(1.0, abs(Eb))
    assert sysm.zeta.max() > 0.0


# ---------------------------------------------------------------------------
def _fd_forces(x, t, box, pbc, params, idx, h=1e-5):
    F = np.zeros((len(idx), 3))
    for a, i in enumerate(idx):
        for d in range(3):
            xp = x.copy(); xp[i, d] += h
            xm = x.copy(); xm[i, d] -= h
            Ep = O.evaluate(xp, t, box, pbc, params)["E"]
            Em = O.evaluate(xm, t, box, pbc, params)["E"]
            F[a, d] = -(Ep - Em) / (2 * h)
    return F


@pytest.mark.parametrize("case", ["sic_bulk", "slab", "cluster"])
def test_forces_match_finite_differences(case):
    """Forces at the charge minimiser equal -dE/dx of the minimised energy
    (charges re-solved at every displaced geometry), to 1e-6 relative."""
    if case == "sic_bulk":
        s = st.sic_3c(2, 4.36, 0.1, seed=8)
        x, t, box, pbc = s.x, s.types, s.box, s.pbc
    elif case == "slab":
        s = st.sic_4h_slab(3, 2, 4, step="strip")
        rng = np.random.default_rng(9)
        x = s.x + rng.uniform(-0.08, 0.08, s.x.shape)
        t, box, pbc = s.types, s.box, s.pbc
    else:
        x, t, box, pbc = _cluster(12, 6, spread=3.0, min_sep=1.45)
    res = O.evaluate(x, t, box, pbc, P1)
    idx = np.arange(0, len(x), max(1, len(x) // 6))[:6]
    Ffd = _fd_forces(x, t, box, pbc, P1, idx)
    Fan = res["F"][idx]
    scale = np.sqrt(np.mean(res["F"] ** 2))
    assert np.max(np.abs(Fan - Ffd)) <= 1e-6 * scale


def test_virial_matches_strain_derivative():
    """W = -dE/d(eps) under homogeneous strain of box and positions, with the
    charges re-minimised."""
    s = st.sic_3c(2, 4.36, 0.1, seed=12)
    res = O.evaluate(s.x, s.types, s.box, s.pbc, P1)
    W = res["virial"]
    h = 1e-6
    for a in range(3):
        e = np.zeros(3); e[a] = h
        Ep = O.evaluate(s.x * (1 + e), s.types, s.box * (1 + e), s.pbc, P1)["E"]
        Em = O.evaluate(s.x * (1 - e), s.types, s.box * (1 - e), s.pbc, P1)["E"]
        dE = (Ep - Em) / (2 * h)
        assert abs(W[a, a] + dE) <= 1e-6 * max(1.0, abs(dE))
    assert np.allclose(W, W.T, atol=1e-8 * np.abs(W).max())


def test_zero_pressure_3c_sic_at_4p36():
    """The synthetic set is tuned so that ideal 3C-SiC is stress-free at
    a = 4.36 A (the lattice constant of the 3C-SiC workload)."""
    s = st.sic_3c(3, 4.36, 0.0)
    res = O.evaluate(s.x, s.types, s.box, s.pbc, P1)
    V = np.prod(s.box)
    assert abs(np.trace(res["virial"]) / (3 * V)) < 1e-9
    assert res["q"][s.types == 0].min() > 0.1     # Si donates charge to C


def test_newton_third_law_and_torque():
    s = st.sic_3c(2, 4.36, 0.1, seed=14)
    res = O.evaluate(s.x, s.types, s.box, s.pbc, P1)
    assert np.abs(res["F"].sum(0)).max() < 1e-10 * np.abs(res["F"]).max() * len(s.x)
    x, t, box, pbc = _cluster(14, 15, spread=3.0, min_sep=1.45)
    r = O.evaluate(x, t, box, pbc, P1)
    assert np.abs(r["F"].sum(0)).max() < 1e-11 * len(x)
    torque = np.cross(x - x.mean(0), r["F"]).sum(0)
    assert np.abs(torque).max() < 1e-10 * len(x)


def test_invariances():
    x, t, box, pbc = _cluster(12, 17, spread=3.0, min_sep=1.45)
    r0 = O.evaluate(x, t, box, pbc, P1)
    # translation
    r1 = O.evaluate(x + np.array([0.37, -1.2, 0.9]), t, box, pbc, P1)
    assert abs(r1["E"] - r0["E"]) < 1e-12 * abs(r0["E"])
    # rotation about the centre
    th = 0.7
    Rm = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    ax = np.array([1.0, 2.0, 0.5]); ax /= np.linalg.norm(ax)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rm = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    c = x.mean(0)
    r2 = O.evaluate((x - c) @ Rm.T + c, t, box, pbc, P1)
    assert abs(r2["E"] - r0["E"]) < 1e-12 * abs(r0["E"])
    assert np.allclose(r2["F"], r0["F"] @ Rm.T, atol=1e-10)
    assert np.allclose(r2["q"], r0["q"], atol=1e-12)
    # permutation
    perm = np.random.default_rng(3).permutation(len(x))
    r3 = O.evaluate(x[perm], t[perm], box, pbc, P1)
    assert abs(r3["E"] - r0["E"]) < 1e-12 * abs(r0["E"])
    assert np.allclose(r3["F"], r0["F"][perm], atol=1e-11)


def test_periodic_supercell_consistency():
    """A 2x2x2 repetition of a periodic 16-atom cell (edge 4.36 A, far below
    the 8 A charge cutoff, so many images and self-images contribute) has 8x
    the energy, the same charges tiled and the same forces tiled."""
    s = st.sic_3c(1, 4.36, 0.08, seed=19)
    s2 = st.sic_3c(1, 4.36, 0.08, seed=19)
    t = s.types.copy(); t[3] = 1  # break the perfect stoichiometry
    x = s.x
    shifts = np.array([[a, b, c] for a in range(2) for b in range(2) for c in range(2)]) * s.box
    X = np.concatenate([x + sh for sh in shifts])
    Tt = np.tile(t, 8)
    r1 = O.evaluate(x, t, s.box, s.pbc, P1)
    r8 = O.evaluate(X, Tt, 2 * s.box, s.pbc, P1)
    assert abs(r8["E"] - 8 * r1["E"]) < 1e-10 * abs(r8["E"])
    assert np.allclose(r8["q"], np.tile(r1["q"], 8), atol=1e-12)
    assert np.allclose(r8["F"], np.tile(r1["F"], (8, 1)), atol=1e-9)


def test_charges_equalise_electronegativity():
    """At the minimiser dE/dq_i = mu for every i and sum q = Q (Sec. 2: the
    charges minimise E_tot), for Q = 0 and a charged system."""
    s = st.sic_4h_slab(3, 2, 4, step="strip")
    for Q in (0.0, 1.5):
        sysm = O.System(s.x, s.types, s.box, s.pbc, P1)
        q, mu = sysm.solve_charges(Q)
        g = sysm.dE_dq(q)
        assert abs(q.sum() - Q) < 1e-12
        assert np.max(np.abs(g - mu)) < 1e-11
        # the energy is minimal: any zero-sum perturbation raises it
        rng = np.random.default_rng(1)
        for _ in range(5):
            d = rng.normal(0, 1e-3, len(q)); d -= d.mean()
            assert sysm.energy(q + d) > sysm.energy(q)


def test_cg_matches_dense():
    s = st.sic_4h_slab(3, 2, 5, step="strip")
    sysm = O.System(s.x, s.types, s.box, s.pbc, P1)
    qd, mud = sysm.solve_charges(0.0, method="dense")
    qc, muc = sysm.solve_charges(0.0, method="cg")
    assert np.max(np.abs(qd - qc)) < 1e-10
    assert abs(mud - muc) < 1e-10


@pytest.mark.parametrize("pname", ["p1", "pt"])
def test_hessian_positive_definite(pname):
    """Sec. 2: the charges minimise E_tot, which has a unique minimum only
    when the charge Hessian is positive definite; every shipped parameter
    set satisfies it on the test shapes."""
    P = st.load_params(pname)
    for s in (st.sic_3c(2, 4.36, 0.05, seed=1), st.sic_4h_slab(3, 2, 4, step="strip"),
              st.stepped_slab_small(6, 3, 5), st.stepped_slab_small(8, 4, 6)):
        H = O.System(s.x, s.types, s.box, s.pbc, P).hessian_dense()
        assert np.allclose(H, H.T)
        assert np.linalg.eigvalsh(H).min() > 1.0


def test_energy_continuous_across_cutoffs():
    """Scanning a dimer across the covalent cutoff S and the charge cutoff
    Rc: energy and force have no jumps."""
    for typ, lo, hi in (((0, 1), 2.3, 2.8), ((1, 1), 1.8, 2.2), ((0, 1), 7.8, 8.2)):
        rs = np.linspace(lo, hi, 801)
        E = []
        F = []
        for r in rs:
            x = np.array([[10.0, 10, 10], [10.0 + r, 10, 10]])
            res = O.evaluate(x, np.array(typ), np.full(3, 40.0), np.array([False] * 3), P1)
            E.append(res["E"]); F.append(res["F"][1, 0])
        E, F = np.array(E), np.array(F)
        dr = rs[1] - rs[0]
        assert np.max(np.abs(np.diff(E))) < 5 * dr * (np.abs(F).max() + 1e-3)
        assert np.max(np.abs(np.diff(F))) < 0.05 * max(1e-2, np.abs(F).max())
