"""The autotuners of the CG matrix pass, the matrix assembly and the
charge-force gather: the depth each keeps (list entries in flight per
thread) is the fastest it timed; every matrix-pass depth gives the same
charges and forces to working-precision rounding (only the grouping of the
row sums differs); every gather depth gives bit-identical forces, energies
and virials (it sums the entries in the same order at any depth)."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")


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
    assert d["cg_mv_batch"] == (4, 8, 16)[int(np.argmin(ms))]
    am = d["asm_ms"]
    assert d["asm_batch"] in (4, 8, 16) and all(m > 0 for m in am)
    # the assembly keeps its default depth 8 unless another is 10% faster
    k = int(np.argmin(am))
    assert d["asm_batch"] == ((4, 8, 16)[k] if am[k] < 0.9 * am[1] else 8)
    gm = d["gather_ms"]
    assert all(m > 0 for m in gm) and d["gather_batch"] == (4, 6, 8)[int(np.argmin(gm))]


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
