"""GPU neighbour lists against brute-force pair enumeration.

The lists are index work: the number of directed entries (i, j, image) with
r < S_ij + skin (covalent part) and r < Rc + skin (whole list) must equal the
oracle's enumeration over every periodic image, self-images included. The
FP64 path compares exactly. The mixed path tests distances in FP32, where a
pair within ~1e-6 A of a cutoff can fall either way, so it allows a couple
of entries per ten thousand atoms."""
import itertools

import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")
SKIN = 0.3
TYPES = ["Si", "C"]


def _s_matrix(params):
    S = np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            S[a, b] = params["pair"][TYPES[min(a, b)] + TYPES[max(a, b)]]["S"]
    return S


def _oracle_counts(s):
    rall = P1["coulomb"]["r_coul"] + SKIN
    i, j, n, u = O.pairs(s.x, s.box, s.pbc, rall)
    r = np.sqrt(np.einsum("ij,ij->i", u, u))
    S = _s_matrix(P1)
    cov = r < S[s.types[i], s.types[j]] + SKIN
    per_all = np.bincount(i, minlength=s.n)
    per_cov = np.bincount(i[cov], minlength=s.n)
    return int(cov.sum()), len(i), int(per_cov.max(initial=0)), int(per_all.max(initial=0))


def _gpu_counts(structs, prec):
    sysm = ctbop.System(P1, precision=prec, skin=SKIN)
    sysm.load_replicas(structs)
    sysm.compute()
    d = sysm.status()
    n = sum(s.n for s in structs)
    sysm.close()
    return int(round(d["mean_cov"] * n)), int(round(d["mean_all"] * n)), d["max_cov"], d["max_all"]


def _cluster(n, seed, spread=3.5, min_sep=1.45):
    rng = np.random.default_rng(seed)
    xs = []
    while len(xs) < n:
        c = rng.uniform(-spread, spread, 3)
        if all(np.linalg.norm(c - y) >= min_sep for y in xs):
            xs.append(c)
    x = np.array(xs) + 15.0
    t = rng.integers(0, 2, n).astype(np.int32)
    return st.Structure(f"cluster{n}", x, t, np.full(3, 30.0), np.array([False] * 3))


CASES = {
    "bulk512": lambda: [st.bulk_3c_512()],
    "small_box_1cell": lambda: [st.sic_3c(1, 4.36, 0.1, seed=31)],
    "small_box_2cell": lambda: [st.sic_3c(2, 4.36, 0.1, seed=32, strain=np.diag([0.03, -0.02, 0.01]))],
    "cluster": lambda: [_cluster(41, 3)],
    "stepped_slab": lambda: [st.stepped_slab_small(8, 4, 6)],
    "replicas": lambda: [st.sic_3c(2, 4.36, 0.05, seed=40), _cluster(17, 41), st.stepped_slab_small(6, 3, 4)],
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_list_counts_match_bruteforce(case, prec):
    structs = CASES[case]()
    ncov, nall, mcov, mall = 0, 0, 0, 0
    for s in structs:
        c, a, mc, ma = _oracle_counts(s)
        ncov, nall, mcov, mall = ncov + c, nall + a, max(mcov, mc), max(mall, ma)
    g = _gpu_counts(structs, prec)
    if prec == "fp64":
        assert g == (ncov, nall, mcov, mall), (g, (ncov, nall, mcov, mall))
    else:
        n = sum(s.n for s in structs)
        slack = 2 + n // 5000
        assert abs(g[0] - ncov) <= slack and abs(g[1] - nall) <= slack, (g, (ncov, nall))
        assert abs(g[2] - mcov) <= 1 and abs(g[3] - mall) <= 1, (g, (mcov, mall))


def test_list_counts_slab_20k_fp64():
    """The 19,488-atom stepped slab: every cell row of a large open-z grid."""
    s = st.stepped_slab_20k()
    c, a, mc, ma = _oracle_counts(s)
    assert _gpu_counts([s], "fp64") == (c, a, mc, ma)


def _boundary_structure():
    """Atoms 1e-9 (relative) inside the list radius of one centre atom and
    1e-9 outside that of another, in all 26 stencil directions, both centres
    on cell corners (the 90 A open box has 21^3 cells of 30/7 A); and a third
    centre with neighbours just inside and just outside the covalent list
    radii of each type pair."""
    rall = P1["coulomb"]["r_coul"] + SKIN
    S = _s_matrix(P1)
    dirs = [np.array(v, float) / np.linalg.norm(v)
            for v in itertools.product((-1, 0, 1), repeat=3) if any(v)]
    xs, ts = [], []
    for c, f, t0 in [((30.0 + 1e-9, 30.0 - 1e-9, 30.0), 1 - 1e-9, 0),
                     ((60.0, 30.0 + 1e-9, 30.0 - 1e-9), 1 + 1e-9, 1)]:
        c = np.array(c)
        xs.append(c)
        ts.append(t0)
        for k, d in enumerate(dirs):
            xs.append(c + d * rall * f)
            ts.append(k % 2)
    c1 = np.array([45.3, 60.7, 29.6])
    xs.append(c1)
    ts.append(1)
    for d, tj, inside in [((1, 0, 0), 0, True), ((-1, 0, 0), 0, False), ((0, 1, 0), 1, True),
                          ((0, -1, 0), 1, False), ((0, 0, 1), 0, False), ((0, 0, -1), 1, True)]:
        r = (S[1, tj] + SKIN) * ((1 - 1e-9) if inside else (1 + 1e-9))
        xs.append(c1 + np.array(d, float) * r)
        ts.append(tj)
    x = np.array(xs)
    return st.Structure("list_radius_boundary", x, np.array(ts, np.int32), np.full(3, 90.0),
                        np.array([False] * 3))


def test_boundary_structure_is_well_separated():
    """The boundary structure keeps its atoms apart (no accidental bonds or
    coincident atoms) and puts its boundary pairs where intended."""
    s = _boundary_structure()
    d = np.linalg.norm(s.x[:, None, :] - s.x[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    assert d.min() > 1.5, d.min()
    rall = P1["coulomb"]["r_coul"] + SKIN
    r0 = np.linalg.norm(s.x[1:27] - s.x[0], axis=1)
    r1 = np.linalg.norm(s.x[28:54] - s.x[27], axis=1)
    assert np.all(r0 < rall) and np.all(rall - r0 < 1e-7)
    assert np.all(r1 > rall) and np.all(r1 - rall < 1e-7)


def test_list_counts_at_the_list_radii_fp64():
    """Pairs 1e-9 inside the list radius and the covalent radii are listed,
    pairs 1e-9 outside are not: exact counts against brute force, for the
    candidate filter against each cell's bounding box as for the pair test."""
    s = _boundary_structure()
    c, a, mc, ma = _oracle_counts(s)
    assert _gpu_counts([s], "fp64") == (c, a, mc, ma)
