"""The autotuners of the CG matrix pass and of the matrix assembly: the
depth each keeps (list entries in flight per thread) is the fastest it
timed, and every matrix-pass depth gives the same charges and forces to
working-precision rounding (only the grouping of the row sums differs; the
assembly computes every entry alike at any depth)."""
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
