"""Storage order: atoms stored along a Morton curve, in a random order, or
as given, give the same results in the caller's order (energies, forces,
charges, velocities after steps, coordination, removal energies, the
force-matching loss and gradient), to rounding; orders that cross replicas
or come after the per-atom arrays are refused."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")


def _structs():
    return [st.stepped_slab_small(6, 3, 4), st.sic_3c(1, 4.36, 0.1, seed=31), st.amorphous_carbon_cluster(40, 2.0, 5)]


def _run(structs, order, prec="fp64"):
    sysm = ctbop.System(P1, precision=prec)
    if order == "random":
        off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
        sysm.load_replicas(structs, order=None)
        rng = np.random.default_rng(0)
        perm = np.concatenate([o + rng.permutation(s.n) for o, s in zip(off, structs)])
        sysm2 = ctbop.System(P1, precision=prec)
        sysm2.set_layout(off)
        sysm2.set_order(perm)
        sysm2.set_box(np.array([s.box for s in structs]), np.array([s.pbc for s in structs]))
        sysm2.set_types(np.concatenate([s.types for s in structs]))
        sysm2.set_positions(np.concatenate([s.x for s in structs]))
        sysm2.set_frozen(np.concatenate([s.frozen for s in structs]).astype(np.uint8))
        sysm.close()
        sysm = sysm2
    else:
        sysm.load_replicas(structs, order=order)
    v = np.concatenate([st.maxwell_boltzmann(s.types, 1200.0, seed=40 + k, frozen=s.frozen)
                        for k, s in enumerate(structs)])
    sysm.set_velocities(v)
    sysm.compute()
    out = {k: sysm.get(k) for k in ("energy", "forces", "charges", "coordination")}
    cand = np.nonzero((out["coordination"] < 4) & (np.concatenate([s.types for s in structs]) == 0))[0][:12]
    out["cand"] = cand
    out["dE"] = sysm.removal_energies(cand)
    F_ref = out["forces"] * 1.01 + 0.01
    nr = np.array([s.n for s in structs], float)
    L, G = sysm.param_grad(w_E=1.0 / nr ** 2, E_ref=out["energy"] + 0.5, w_F=1.0 / (3 * nr), F_ref=F_ref)
    out["loss"], out["grad"] = L, ctbop.params_vector(G)
    sysm.step(10, 0.5)
    out["x"], out["v"] = sysm.get("positions"), sysm.get("velocities")
    sysm.close()
    return out


@pytest.mark.parametrize("order", ["morton", "random"])
def test_results_do_not_depend_on_storage_order(order):
    structs = _structs()
    a, b = _run(structs, None), _run(structs, order)
    np.testing.assert_allclose(b["energy"], a["energy"], rtol=0, atol=1e-9 * 200)
    assert np.max(np.abs(b["forces"] - a["forces"])) < 1e-8
    assert np.max(np.abs(b["charges"] - a["charges"])) < 1e-9
    assert np.array_equal(b["coordination"], a["coordination"]) and np.array_equal(b["cand"], a["cand"])
    np.testing.assert_allclose(b["dE"], a["dE"], rtol=0, atol=1e-7)
    assert b["loss"] == pytest.approx(a["loss"], rel=1e-9)
    np.testing.assert_allclose(b["grad"], a["grad"], rtol=0, atol=1e-7 * np.max(np.abs(a["grad"])))
    box = np.concatenate([np.tile(s.box, (s.n, 1)) for s in structs])
    pbc = np.concatenate([np.tile(s.pbc, (s.n, 1)) for s in structs])
    d = b["x"] - a["x"]
    d = d - np.where(pbc, np.round(d / box) * box, 0.0)
    assert np.max(np.abs(d)) < 1e-8 and np.max(np.abs(b["v"] - a["v"])) < 1e-9


def test_bad_orders_are_refused():
    structs = _structs()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    sysm = ctbop.System(P1, precision="mixed")
    sysm.set_layout(off)
    bad = np.arange(off[-1])
    bad[0], bad[-1] = bad[-1], bad[0]          # swaps atoms of two replicas
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.set_order(bad)
    dup = np.arange(off[-1])
    dup[1] = 0
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.set_order(dup)
    sysm.set_types(np.concatenate([s.types for s in structs]))
    with pytest.raises(ctbop.CtbopError, match="STATE"):
        sysm.set_order(np.arange(off[-1]))
    sysm.close()
