"""Pins of the oracle's force-matching gradient (central differences of the
loss, the definition) against closed forms that follow from the energy's
structure, not from the difference machinery itself:
  * E0_t enters E as a count: dE/dE0_t = number of atoms of type t;
  * chi_t, J_t enter E as chi q + J q^2 at the minimiser, whose charge
    response drops out (envelope theorem): dE/dchi_t = sum q_i, dE/dJ_t =
    sum q_i^2 over type t;
  * A enters linearly through 1/2 fc e^{-lambda1 r} per directed bond;
  * k_e scales the charge kernel: dE/dk_e = E_Coulomb / k_e at the minimiser;
  * no force depends on E0, so the force term's derivative with respect to
    E0 is zero."""
import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")


def _cell():
    return st.sic_3c(1, 4.36, 0.12, seed=61, strain=np.diag([0.02, -0.01, 0.015]))


def _energy_grad(s, paths):
    o = O.evaluate(s.x, s.types, s.box, s.pbc, P1)
    # loss = 1/2 (E - (E - 1))^2 -> dloss/dtheta = dE/dtheta
    return o, O.loss_grad_fd([s], P1, w_E=[0.5], E_ref=[o["E"] - 1.0], paths=paths)


def test_self_energy_parameters_closed_form():
    s = _cell()
    paths = [("self", f, t) for f in ("E0", "chi", "J") for t in (0, 1)]
    o, g = _energy_grad(s, paths)
    q = o["q"]
    for t in (0, 1):
        m = s.types == t
        assert g[("self", "E0", t)] == pytest.approx(m.sum(), rel=1e-9)
        assert g[("self", "chi", t)] == pytest.approx(q[m].sum(), rel=1e-6, abs=1e-9)
        assert g[("self", "J", t)] == pytest.approx((q[m] ** 2).sum(), rel=1e-6, abs=1e-9)


def test_repulsion_prefactor_closed_form():
    s = _cell()
    paths = [("pair", k, "A") for k in ("SiSi", "SiC", "CC")]
    _, g = _energy_grad(s, paths)
    i, j, n, u = O.pairs(s.x, s.box, s.pbc, 3.5)
    r = np.linalg.norm(u, axis=1)
    names = {(0, 0): "SiSi", (0, 1): "SiC", (1, 0): "SiC", (1, 1): "CC"}
    ref = {"SiSi": 0.0, "SiC": 0.0, "CC": 0.0}
    for a, b, rr in zip(s.types[i], s.types[j], r):
        pr = P1["pair"][names[(a, b)]]
        if rr < pr["R"]:
            fc = 1.0
        elif rr < pr["S"]:
            fc = 0.5 * (1.0 + np.cos(np.pi * (rr - pr["R"]) / (pr["S"] - pr["R"])))
        else:
            fc = 0.0
        ref[names[(a, b)]] += 0.5 * fc * np.exp(-pr["lambda1"] * rr)
    for k in ref:
        assert g[("pair", k, "A")] == pytest.approx(ref[k], rel=1e-7, abs=1e-10)


def test_coulomb_constant_closed_form():
    s = _cell()
    o, g = _energy_grad(s, [("coulomb", "k_e")])
    no_c = O.evaluate(s.x, s.types, s.box, s.pbc, O.with_leaf(P1, ("coulomb", "k_e"), 0.0), q=o["q"])["E"]
    ke = P1["coulomb"]["k_e"]
    assert g[("coulomb", "k_e")] == pytest.approx((o["E"] - no_c) / ke, rel=1e-6)


def test_force_term_does_not_depend_on_self_energy_constant():
    s = _cell()
    o = O.evaluate(s.x, s.types, s.box, s.pbc, P1)
    F_ref = o["F"] + 0.1
    g = O.loss_grad_fd([s], P1, w_F=[1.0], F_ref=F_ref, paths=[("self", "E0", 0), ("self", "E0", 1)])
    assert abs(g[("self", "E0", 0)]) < 1e-9 and abs(g[("self", "E0", 1)]) < 1e-9


def test_leaves_cover_every_parameter_once():
    leaves = O.param_leaves(P1)
    paths = [p for p, _ in leaves]
    assert len(paths) == len(set(paths))
    # 3 pairs x 7 + 4 bonds x 6 + 8 triplets x 5 x 2 + 6 self + 2 gamma_c + r_coul + k_e
    assert len(paths) == 21 + 24 + 80 + 6 + 2 + 2
