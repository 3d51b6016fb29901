"""Error paths of the C ABI, all raised on the host side or through the
library's device error word. Nothing here faults the GPU: bad values are
rejected by argument checks, and non-finite positions are caught by the
binning kernel, which records them and substitutes zero."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")


def _system(s, **kw):
    sysm = ctbop.System(P1, **kw)
    sysm.load(s)
    return sysm


def test_cg_iteration_limit_is_reported():
    """Too few CG iterations: status says CG_NOT_CONVERGED, the solve stopped
    at the limit, and the results are still written (finite)."""
    s = st.bulk_3c_512()
    sysm = _system(s, precision="fp64", cg_max_iter=3)
    sysm.compute()
    d = sysm.status()
    assert d["rc"] == "CG_NOT_CONVERGED"
    assert d["cg_iters_last"] == 3
    q = sysm.get("charges")
    assert np.all(np.isfinite(q)) and abs(q.sum()) < 1e-10
    with pytest.raises(ctbop.CtbopError, match="CG_NOT_CONVERGED"):
        sysm.step(1, 0.5)
    sysm.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tiny_capacities_regrow(prec):
    """Capacities far below the need: the first build measures the counts and
    the lists regrow; results equal a default run (entry order inside a
    list may differ, so only rounding changes)."""
    s = st.stepped_slab_small(8, 4, 6)
    a = _system(s, precision=prec)
    a.compute()
    Fa, qa = a.get("forces"), a.get("charges")
    b = _system(s, precision=prec, cap_cov=4, cap_all=8)
    b.compute()
    Fb, qb = b.get("forces"), b.get("charges")
    tol = 1e-10 if prec == "fp64" else 2e-4
    rms = np.sqrt(np.mean(Fa ** 2))
    assert np.max(np.abs(Fa - Fb)) / rms < tol
    assert np.max(np.abs(qa - qb)) < (1e-10 if prec == "fp64" else 1e-5)
    assert b.status()["rc"] == "OK"
    a.close()
    b.close()


def test_nonfinite_position_is_reported():
    s = st.bulk_3c_512()
    x = s.x.copy()
    x[7, 1] = np.nan
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(st.Structure("bad", x, s.types, s.box, s.pbc))
    with pytest.raises(ctbop.CtbopError, match="NONFINITE"):
        sysm.compute()
    sysm.close()


def test_invalid_arguments_are_rejected():
    s = st.bulk_3c_512()
    sysm = ctbop.System(P1, precision="mixed")
    with pytest.raises(ctbop.CtbopError, match="STATE"):
        sysm.set_types(s.types)                    # before set_layout
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.set_layout([0, 10, 5])                # offsets decrease
    sysm.set_layout([0, s.n])
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.set_box([[-1.0, 5.0, 5.0]], [[True, True, True]])
    bad = s.types.copy()
    bad[3] = 2
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.set_types(bad)
    sysm.load(s)
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.step(1, 0.0)
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.step(1, float("nan"))
    sysm.compute()
    assert sysm.status()["rc"] == "OK"
    sysm.close()


def test_caller_buffers_are_checked_before_the_library_sees_them():
    """Buffers shorter than the system, or of a narrower element type, are
    rejected on the host: the library would read or write past them."""
    torch = pytest.importorskip("torch")
    s = st.bulk_3c_512()
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    with pytest.raises(ValueError, match="elements"):
        sysm.set_positions(s.x[:-1])
    with pytest.raises(ValueError, match="elements"):
        sysm.set_velocities(torch.zeros((s.n - 1, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError, match="float64"):
        sysm.set_positions(torch.tensor(s.x, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError, match="boxes"):
        sysm.set_box(np.ones((2, 3)) * 20.0, np.ones((2, 3), bool))
    sysm.compute()
    with pytest.raises(ValueError, match="elements"):
        sysm.get("forces", torch.empty((s.n, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError, match="float64"):
        sysm.get("charges", np.empty(s.n, np.float32))
    F = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    sysm.get("forces", F)
    torch.cuda.synchronize()
    assert np.array_equal(F.cpu().numpy(), sysm.get("forces"))
    sysm.close()


def test_create_rejects_bad_options():
    with pytest.raises(ctbop.CtbopError):
        ctbop.System(P1, cg_max_iter=0)
    with pytest.raises(ctbop.CtbopError):
        ctbop.System(P1, skin=-0.1)


def test_empty_system_runs_every_entry_point():
    """A layout with no atoms at all: every entry point returns cleanly with
    empty results (zero energy)."""
    empty = st.Structure("empty", np.zeros((0, 3)), np.zeros(0, np.int32), np.full(3, 20.0), np.array([True] * 3))
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(empty)
    sysm.compute()
    assert sysm.get("energy").tolist() == [0.0]
    assert sysm.get("forces").shape == (0, 3)
    sysm.step(3, 0.5)
    it, fm = sysm.minimize(max_iter=5, fmax=1e-3)
    assert it[0] == 0
    assert len(sysm.rings()) == 0
    assert sysm.removal_energies([]).shape == (0,)
    assert sysm.get("coordination").shape == (0,)
    L, G = sysm.param_grad(w_E=[1.0], E_ref=[0.0])
    assert L == 0.0
    sysm.close()


def test_triclinic_cell_is_refused():
    """Cells are orthorhombic (a reading the library documents): a cell
    matrix with an off-diagonal entry is refused through the C ABI with
    INVALID_ARG and a message, and nothing of the box is changed."""
    import ctypes as C
    s = st.bulk_3c_512()
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    h = np.ascontiguousarray(np.diag(s.box).reshape(1, 3, 3))
    h[0, 0, 1] = 0.2                              # a shear of the first cell vector
    p = np.ones((1, 3), dtype=np.uint8)
    L = ctbop.lib()
    rc = L.ctbop_set_box(sysm._h, h.ctypes.data_as(C.c_void_p), p.ctypes.data_as(C.c_void_p))
    assert ctbop.ERR[rc] == "INVALID_ARG"
    assert b"orthorhombic" in L.ctbop_last_error(sysm._h)
    sysm.compute()                                # the previous box still holds
    assert sysm.status()["rc"] == "OK"
    sysm.close()
