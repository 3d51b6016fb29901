"""FIRE energy minimisation on the GPU against the oracle's (same algorithm,
same order of operations): trajectories over a fixed number of iterations,
the closed-form minima of the SiC dimer and linear Si3, a stationary
crystal, replicas relaxed together versus alone, argument errors; at full
size (the 19,488-atom stepped slab) the invariants."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")
OPEN = np.array([False] * 3)


def _wrap(d, box, pbc):
    return d - np.where(pbc, np.round(d / box) * box, 0.0)


def _cluster(n, seed, spread=3.2, min_sep=1.6):
    rng = np.random.default_rng(seed)
    xs = []
    while len(xs) < n:
        c = rng.uniform(-spread, spread, 3)
        if all(np.linalg.norm(c - y) >= min_sep for y in xs):
            xs.append(c)
    t = rng.integers(0, 2, n).astype(np.int32)
    return st.Structure(f"cluster{n}", np.array(xs) + 15.0, t, np.full(3, 30.0), OPEN)


CASES = {
    "slab": lambda: st.stepped_slab_small(6, 3, 4),
    "bulk": lambda: st.sic_3c(1, 4.36, 0.12, seed=21),
    "cluster": lambda: _cluster(16, 22),
}


def _gpu_relax(structs, prec, **kw):
    sysm = ctbop.System(P1, precision=prec)
    sysm.load_replicas(structs)
    it, fm = sysm.minimize(**kw)
    x, v, E, F = sysm.get("positions"), sysm.get("velocities"), sysm.get("energy"), sysm.get("forces")
    sysm.close()
    return it, fm, x, v, E, F


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_trajectory_matches_oracle(case, prec):
    s = CASES[case]()
    n = 25
    it, fm, x, v, E, F = _gpu_relax([s], prec, max_iter=n, fmax=1e-12)
    xo, ito, Eo, ok = O.fire_minimize(s.x, s.types, s.box, s.pbc, P1, frozen=s.frozen, n_iter=n)
    assert it[0] == -1 and ito == n and not ok
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(_wrap(x - xo, s.box, s.pbc))) < tol
    # mixed: the stress-geometry bar of the single-point parity tests (cells
    # smaller than the charge cutoff round every image alike)
    assert E[0] == pytest.approx(Eo[-1], abs=(1e-9 if prec == "fp64" else 5e-6) * s.n)
    assert np.all(v == 0.0)
    Fm = np.where(s.frozen[:, None], 0.0, F)
    assert fm[0] == pytest.approx(np.sqrt(np.max(np.sum(Fm * Fm, axis=1))), rel=1e-9)


def _dimer():
    return st.Structure("SiC", np.array([[10.0, 10.0, 10.0], [12.0, 10.3, 9.8]]), np.array([0, 1], np.int32),
                        np.full(3, 40.0), OPEN)


def _si3(d0=2.3):
    x = np.array([[10.0, 10.0, 10.0], [10.0 + d0, 10.0, 10.0], [10.0 + 2 * d0, 10.0, 10.0]])
    return st.Structure("Si3", x, np.zeros(3, np.int32), np.full(3, 40.0), OPEN)


@pytest.mark.parametrize("prec,fmax,tol", [("fp64", 1e-7, 1e-6), ("mixed", 1e-3, 1e-3)])
def test_reaches_oracle_minima(prec, fmax, tol):
    """Dimer and Si3 relaxed together, as two replicas: each reaches the
    minimum the oracle's FIRE reaches (pinned there to closed forms)."""
    structs = [_dimer(), _si3()]
    it, fm, x, v, E, F = _gpu_relax(structs, prec, max_iter=5000, fmax=fmax)
    assert np.all(it > 0) and np.all(fm < fmax)
    xd, _, _, okd = O.fire_minimize(structs[0].x, structs[0].types, structs[0].box, OPEN, P1, fmax=1e-7,
                                    max_iter=5000)
    xs, _, _, oks = O.fire_minimize(structs[1].x, structs[1].types, structs[1].box, OPEN, P1, fmax=1e-7,
                                    max_iter=5000)
    assert okd and oks
    assert np.linalg.norm(x[1] - x[0]) == pytest.approx(np.linalg.norm(xd[1] - xd[0]), abs=tol)
    for a, b in ((2, 3), (3, 4)):
        assert np.linalg.norm(x[b] - x[a]) == pytest.approx(np.linalg.norm(xs[b - 2] - xs[a - 2]), abs=tol)


@pytest.mark.parametrize("n,fmax,xtol,etol,kind", [(25, 1e-12, 1e-9, 1e-10, "mixed bag"),
                                                   (2000, 1e-4, 1e-5, 1e-9, "unique minima")])
def test_replicas_relax_independently(n, fmax, xtol, etol, kind):
    """Replicas relaxed in one batch follow the paths they follow alone (up
    to periodic wrapping): to rounding over 25 iterations (a slab, a dimer, a random cluster; over
    hundreds the order of FP64 atomic sums, which depends on the batch,
    grows, and a random cluster's long path diverges); and to their
    converged minimum (dimer, Si3)."""
    if kind == "mixed bag":
        structs = [CASES["slab"](), _dimer(), CASES["cluster"]()]
    else:
        structs = [_dimer(), _si3()]
    it, fm, x, _, E, _ = _gpu_relax(structs, "fp64", max_iter=n, fmax=fmax)
    if kind == "unique minima":
        assert np.all(it > 0)
    off = np.cumsum([0] + [s.n for s in structs])
    for r, s in enumerate(structs):
        it1, fm1, x1, _, E1, _ = _gpu_relax([s], "fp64", max_iter=n, fmax=fmax)
        assert it[r] == it1[0]
        # positions are defined modulo the periodic box: list rebuilds wrap
        # them, and a batch rebuilds when any replica's atoms have moved far
        # enough, so the batch and the lone run may wrap at different times
        assert np.max(np.abs(_wrap(x[off[r]:off[r + 1]] - x1, s.box, s.pbc))) < xtol
        assert E[r] == pytest.approx(E1[0], abs=etol * s.n)


def test_stationary_crystal_and_arguments():
    s = st.sic_3c(2, 4.36, 0.0, seed=1)
    it, fm, x, v, E, F = _gpu_relax([s], "fp64", max_iter=100, fmax=1e-6)
    assert it[0] == 0 and np.max(np.abs(_wrap(x - s.x, s.box, s.pbc))) == 0.0
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    for kw in (dict(max_iter=-1), dict(fmax=0.0), dict(dt0=2.0, dt_max=1.0)):
        with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
            sysm.minimize(**kw)
    sysm.close()


def test_full_size_slab_invariants():
    """The 19,488-atom stepped slab, 60 iterations: the energy falls, frozen
    atoms stay, velocities end at zero, and the forces reported are the
    evaluation at the final positions."""
    s = st.stepped_slab_20k()
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    sysm.compute()
    E0 = sysm.get("energy")[0]
    it, fm = sysm.minimize(max_iter=60, fmax=1e-4)
    x, v, E1, F = sysm.get("positions"), sysm.get("velocities"), sysm.get("energy")[0], sysm.get("forces")
    sysm.compute()
    F2 = sysm.get("forces")
    sysm.close()
    assert it[0] == -1 and E1 < E0 - 1.0
    assert np.array_equal(_wrap(x[s.frozen] - s.x[s.frozen], s.box, s.pbc), np.zeros((s.frozen.sum(), 3)))
    assert np.all(v == 0.0)
    assert np.max(np.abs(F2 - F)) < 1e-4 * np.sqrt(np.mean(F2 ** 2))
