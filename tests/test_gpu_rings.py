"""Ring statistics on the GPU against the oracle (index work: every ring,
its size and centre, exact; 6-ring orientations to rounding): graphene,
a Stone-Wales defect, defected flakes on SiC, amorphous C clusters, lone
polygons as replicas of one batch; the 256-replica annealing ensemble at
full size, sampled replicas against the oracle; argument errors."""
import math

import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import rings as RG
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")
SCC = P1["pair"]["CC"]["S"]
OPEN = np.array([False] * 3)


def _pdist(a, b, box, pbc):
    d = a - b
    d = d - np.where(pbc, np.round(d / box) * box, 0.0)
    return float(np.sqrt(d @ d))


def _compare(structs, prec, bond_cut=0.0):
    """Every GPU ring matches one oracle ring of the same size and centre
    (periodic distance), one to one; 6-ring orientations agree."""
    sysm = ctbop.System(P1, precision=prec)
    sysm.load_replicas(structs)
    sysm.compute()
    rec = sysm.rings(bond_cut=bond_cut)
    sysm.close()
    cut = bond_cut or SCC
    ctol, otol = (1e-9, 1e-8) if prec == "fp64" else (1e-4, 1e-2)
    total = 0
    for r, s in enumerate(structs):
        ro = O.rings(s.x, s.types, s.box, s.pbc, cut)
        mine = rec[rec["replica"] == r]
        assert len(mine) == len(ro), (r, s.name, len(mine), len(ro))
        free = list(range(len(ro)))
        for m in mine:
            best = min(free, key=lambda k: (ro[k][0] != m["size"], _pdist(ro[k][1], m["centre"], s.box, s.pbc)))
            n, c, ao = ro[best]
            assert n == m["size"] and _pdist(c, m["centre"], s.box, s.pbc) < ctol, (r, n, m)
            if n == 6:
                d = abs(m["orientation"] - ao) % 60.0
                assert min(d, 60.0 - d) < otol
            else:
                assert math.isnan(m["orientation"]) and math.isnan(ao)
            free.remove(best)
        total += len(ro)
    return rec, total


def _polygon(n, b=1.42):
    R = b / (2.0 * math.sin(math.pi / n))
    a = 2 * math.pi * np.arange(n) / n
    x = np.stack([R * np.cos(a), R * np.sin(a), np.zeros(n)], 1) + 20.0
    return st.Structure(f"C{n}", x, np.ones(n, np.int32), np.full(3, 40.0), OPEN)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graphene_and_flakes(prec):
    structs = [st.graphene_sheet(200, seed=1, n_stone_wales=0, disp=0.0),
               st.graphene_sheet(300, seed=5, n_stone_wales=2),
               st.graphene_on_sic(1200, seed=7)]
    rec, total = _compare(structs, prec)
    c = RG.counts(rec, len(structs))
    assert c[0, 3] == structs[0].n // 2 and c[0].sum() == c[0, 3]
    assert total > 100


def test_stone_wales_at_a_shorter_cut():
    s = st.graphene_sheet(200, seed=3, n_stone_wales=1, disp=0.0)
    rec, _ = _compare([s], "fp64", bond_cut=1.7)
    c = RG.counts(rec, 1)[0]
    assert (c[2], c[3], c[4]) == (2, s.n // 2 - 4, 2)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amorphous_clusters(prec):
    structs = [st.amorphous_carbon_cluster(n, d, seed) for n, d, seed in ((150, 1.8, 1), (220, 2.1, 2), (300, 2.3, 3))]
    rec, total = _compare(structs, prec)
    assert total > 20 and len(set(rec["size"])) >= 3


def test_polygons_as_replicas():
    structs = [_polygon(n) for n in range(3, 9)]
    rec, _ = _compare(structs, "fp64", bond_cut=1.6)
    assert sorted(zip(rec["replica"], rec["size"])) == [(r, r + 3) for r in range(6)]


def test_annealing_ensemble_full_size():
    """All 256 replicas (410,978 atoms) in one call; the replicas of at most
    600 atoms against the oracle one by one (the rest: every record is a
    valid primitive-ring record of its replica's type mix)."""
    structs, _ = st.annealing_ensemble(256, seed=4)
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load_replicas(structs)
    sysm.compute()
    rec = sysm.rings()
    sysm.close()
    c = RG.counts(rec, len(structs))
    checked = 0
    for r, s in enumerate(structs):
        if s.n > 600:
            continue
        ro = O.rings(s.x, s.types, s.box, s.pbc, SCC)
        assert c[r].sum() == len(ro), (r, s.name)
        assert np.array_equal(c[r], O.ring_counts(ro)), (r, s.name)
        checked += 1
    assert checked >= 10
    no_c = [r for r, s in enumerate(structs) if not np.any(s.types == 1)]
    assert all(c[r].sum() == 0 for r in no_c)
    assert np.all((rec["size"] >= 3) & (rec["size"] <= 8))


def test_arguments_and_state():
    s = st.graphene_sheet(100, seed=1, n_stone_wales=0, disp=0.0)
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    with pytest.raises(ctbop.CtbopError, match="STATE"):
        sysm.rings()
    sysm.compute()
    for kw in (dict(bond_cut=SCC + 0.1), dict(max_size=9), dict(max_size=2), dict(bond_cut=-1.0)):
        with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
            sysm.rings(**kw)
    assert len(sysm.rings(max_size=5)) == 0
    sysm.close()
