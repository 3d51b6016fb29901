"""The autotuners of the CG matrix pass, the matrix assembly, the
charge-force gather, the covalent passes and the neighbour-list build: the
setting each keeps (list entries in flight per thread, lanes per atom, or
warps per block and stencil cells per batch) is the fastest it timed;
every matrix-pass depth gives the same charges and forces to
working-precision rounding (only the grouping of the row sums differs);
every gather depth gives bit-identical forces, energies and virials (it sums
the entries in the same order at any depth); every covalent lane count gives
bit-identical forces (one lane computes each bond whole) and per-atom
energies equal to the rounding of their cross-lane sum; every list-build
shape writes the same lists, so the forces and energies agree bit for bit."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")
BUILD_SHAPES = [(2, 64), (2, 128), (4, 64), (4, 128), (8, 64), (8, 128)]


def _run(s, prec):
    sysm = ctbop.System(P1, precision=prec)
    sysm.load(s)
    sysm.compute()
    out = sysm.get("forces"), sysm.get("charges"), sysm.status()
    sysm.close()
    return out


def test_tuner_keeps_the_fastest_depth():
    _, _, d = _run(st.stepped_slab_small(12, 6, 8), "mixed")
    ms = d["cg_mv_ms"]
    assert d["cg_mv_batch"] in (4, 8, 16)
    assert all(m > 0 for m in ms)
    # (the timed minimum; event timings of a small system can tie)
    assert ms[(4, 8, 16).index(d["cg_mv_batch"])] == min(ms)
    am = d["asm_ms"]
    assert d["asm_batch"] in (4, 8, 16) and all(m > 0 for m in am)
    # the assembly keeps its default depth 8 unless another is 10% faster
    k = int(np.argmin(am))
    assert d["asm_batch"] == ((4, 8, 16)[k] if am[k] < 0.9 * am[1] else 8)
    gm = d["gather_ms"]
    assert all(m > 0 for m in gm) and gm[(4, 6, 8).index(d["gather_batch"])] == min(gm)
    cm = d["cov_ms"]
    assert d["cov_lanes"] in (4, 8, 16) and all(m > 0 for m in cm)
    assert cm[(4, 8, 16).index(d["cov_lanes"])] == min(cm)
    bm = d["build_ms"]
    assert all(m > 0 for m in bm)
    assert bm[BUILD_SHAPES.index((d["build_warps"], d["build_batch"]))] == min(bm)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_every_depth_gives_the_same_result(prec, monkeypatch):
    s = st.stepped_slab_small(8, 4, 6)
    ref = None
    for depth in (4, 8, 16):
        monkeypatch.setenv("CTBOP_MV_BATCH", str(depth))
        F, q, d = _run(s, prec)
        assert d["cg_mv_batch"] == depth
        if ref is None:
            ref = (F, q)
            continue
        rms = np.sqrt(np.mean(ref[0] ** 2))
        ftol, qtol = (1e-9, 1e-10) if prec == "fp64" else (2e-5, 2e-6)
        assert np.max(np.abs(F - ref[0])) / rms < ftol
        assert np.max(np.abs(q - ref[1])) < qtol


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_every_gather_depth_gives_identical_results(prec, monkeypatch):
    """At fixed charges (no CG, whose reductions add in a varying order) the
    forces and per-atom energies of every gather depth agree bit for bit;
    the per-replica sums, added across blocks by atomics, to rounding."""
    s = st.stepped_slab_small(8, 4, 6)
    q = np.random.default_rng(8).normal(0.0, 0.2, s.n)
    q -= q.mean()
    monkeypatch.setenv("CTBOP_MV_BATCH", "8")
    ref = None
    for depth in (4, 6, 8):
        monkeypatch.setenv("CTBOP_GATHER_BATCH", str(depth))
        sysm = ctbop.System(P1, precision=prec)
        sysm.load(s)
        sysm.set_charges(q)
        sysm.compute(fixed_charges=True)
        out = [sysm.get(k) for k in ("forces", "e_atom", "energy", "virial")]
        assert sysm.status()["gather_batch"] == depth
        sysm.close()
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        np.testing.assert_allclose(out[2], ref[2], rtol=1e-13)
        np.testing.assert_allclose(out[3], ref[3], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_every_covalent_lane_count_gives_identical_results(prec, monkeypatch):
    """At fixed charges every lane count (4, 8, 16 lanes per atom) gives the
    same forces bit for bit, on a first evaluation (the mixed path's
    accurate mode, with its FP64 queue) and on a second one at moved
    positions; the per-atom energies agree to the rounding of the lanes'
    partial sums."""
    s = st.stepped_slab_small(8, 4, 6)
    q = np.random.default_rng(9).normal(0.0, 0.2, s.n)
    q -= q.mean()
    x2 = s.x + np.random.default_rng(10).normal(0.0, 0.03, s.x.shape)
    monkeypatch.setenv("CTBOP_MV_BATCH", "8")
    monkeypatch.setenv("CTBOP_GATHER_BATCH", "8")
    ref = None
    for lanes in (4, 8, 16):
        monkeypatch.setenv("CTBOP_COV_LANES", str(lanes))
        sysm = ctbop.System(P1, precision=prec)
        sysm.load(s)
        sysm.set_charges(q)
        out = []
        for x in (s.x, x2):
            sysm.set_positions(x)
            sysm.compute(fixed_charges=True)
            out += [sysm.get("forces"), sysm.get("e_atom")]
        assert sysm.status()["cov_lanes"] == lanes
        sysm.close()
        if ref is None:
            ref = out
            continue
        etol = 1e-12 if prec == "fp64" else 1e-6
        for k in (0, 2):
            assert np.array_equal(out[k], ref[k])
            np.testing.assert_allclose(out[k + 1], ref[k + 1], rtol=0, atol=etol)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_every_list_build_shape_gives_identical_lists(prec, monkeypatch):
    """Every list-build shape gives the same list counts and, at fixed
    charges, bit-identical forces and per-atom energies (the forces sum the
    list entries in list order, so equal forces mean equal lists); on three
    replicas of different kinds, so the cells of several grids are spread
    over the blocks."""
    structs = [st.stepped_slab_small(8, 4, 6), st.sic_3c(2, 4.36, 0.05, seed=40), st.bulk_3c_512()]
    n = sum(s.n for s in structs)
    q = np.random.default_rng(11).normal(0.0, 0.2, n)
    monkeypatch.setenv("CTBOP_MV_BATCH", "8")
    monkeypatch.setenv("CTBOP_GATHER_BATCH", "8")
    monkeypatch.setenv("CTBOP_COV_LANES", "8")
    ref = None
    for w, b in BUILD_SHAPES:
        monkeypatch.setenv("CTBOP_BUILD_SHAPE", f"{w},{b}")
        sysm = ctbop.System(P1, precision=prec)
        sysm.load_replicas(structs)
        sysm.set_charges(q)
        sysm.compute(fixed_charges=True)
        d = sysm.status()
        assert (d["build_warps"], d["build_batch"]) == (w, b)
        out = [sysm.get("forces"), sysm.get("e_atom"), d["mean_cov"], d["mean_all"], d["max_cov"], d["max_all"]]
        sysm.close()
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        assert out[2:] == ref[2:]
