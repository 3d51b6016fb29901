"""Force-matching gradient on the GPU (FP64 policy) against the oracle's
central differences of the same loss, over every parameter of the set, on a
batch of two uneven replicas (a strained 64-atom 3C-SiC cell and a random
20-atom Si/C cluster)."""
import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P0 = st.load_params("p0")


def _cluster(n, seed, spread=3.2, min_sep=1.45):
    rng = np.random.default_rng(seed)
    xs = []
    while len(xs) < n:
        c = rng.uniform(-spread, spread, 3)
        if all(np.linalg.norm(c - y) >= min_sep for y in xs):
            xs.append(c)
    x = np.array(xs) + 15.0
    t = rng.integers(0, 2, n).astype(np.int32)
    return st.Structure(f"cluster{n}", x, t, np.full(3, 30.0), np.array([False] * 3))


def _batch():
    return [st.sic_3c(2, 4.36, 0.1, seed=71, strain=np.diag([0.04, -0.03, 0.02])), _cluster(20, 72)]


def _leaf(d, path):
    node = d
    for k in path:
        node = node[k]
    return float(node)


def _gpu_grad(structs, **loss):
    sysm = ctbop.System(P0, precision="fp64")
    sysm.load_replicas(structs)
    L, G = sysm.param_grad(**loss)
    out = ctbop.grad_to_dict(G, P0)
    F = sysm.get("forces")
    sysm.close()
    return L, out, F


def _compare(structs, loss, rtol):
    L, g, _ = _gpu_grad(structs, **loss)
    Lo = O.force_matching_loss(structs, P0, **loss)
    assert L == pytest.approx(Lo, rel=1e-9, abs=1e-12)
    fd = O.loss_grad_fd(structs, P0, **loss)
    scale = max(abs(v) for v in fd.values())
    worst = sorted(((abs(_leaf(g, p) - v) / (abs(v) + 1e-3 * scale), p, _leaf(g, p), v) for p, v in fd.items()),
                   reverse=True)[:5]
    print("worst", worst)
    assert worst[0][0] <= rtol, worst


def test_energy_loss_gradient_matches_oracle():
    structs = _batch()
    E = [O.evaluate(s.x, s.types, s.box, s.pbc, P0)["E"] for s in structs]
    _compare(structs, dict(w_E=[0.5, 0.3], E_ref=[E[0] - 1.0, E[1] + 2.0]), rtol=1e-8)


def test_force_matching_gradient_matches_oracle():
    """Targets from a perturbed parameter set (the fitting situation): the
    loss has energy and force terms, and the force term's gradient carries
    the charge response through the adjoint solve."""
    structs = _batch()
    Pt = O.with_leaf(P0, ("pair", "SiC", "A"), P0["pair"]["SiC"]["A"] * 1.03)
    Pt = O.with_leaf(Pt, ("self", "chi", 1), P0["self"]["chi"][1] * 0.97)
    Pt = O.with_leaf(Pt, ("triplet", "SiCSi", "h", 1), P0["triplet"]["SiCSi"]["h"][1] + 0.05)
    ref = [O.evaluate(s.x, s.types, s.box, s.pbc, Pt) for s in structs]
    loss = dict(w_E=[0.2, 0.1], E_ref=[o["E"] for o in ref], w_F=[1.0, 0.5],
                F_ref=np.concatenate([o["F"] for o in ref]))
    # the force term adds a directional central difference (O(h^2) at h =
    # 1e-4 A): measured worst 4.4e-7 relative, on the cutoff radii
    _compare(structs, loss, rtol=2e-6)


def test_energy_constant_gradient_exact():
    """dE/dE0_t is the count of type-t atoms, from the analytic kernel."""
    structs = _batch()
    sysm = ctbop.System(P0, precision="fp64")
    sysm.load_replicas(structs)
    sysm.compute()
    E = sysm.get("energy")
    L, G = sysm.param_grad(w_E=[0.5, 0.5], E_ref=E - 1.0)
    sysm.close()
    types = np.concatenate([s.types for s in structs])
    for t in (0, 1):
        assert G.E0[t] == pytest.approx(float((types == t).sum()), rel=1e-12)
    assert G.mass[0] == 0.0 and G.mass[1] == 0.0


def test_autograd_energy_backward_is_minus_force():
    import torch
    from paper_1802_07871_gb300.autograd import Energy
    structs = _batch()
    sysm = ctbop.System(P0, precision="fp64")
    sysm.load_replicas(structs)
    x = torch.tensor(np.concatenate([s.x for s in structs]), dtype=torch.float64, requires_grad=True)
    E = Energy.apply(x, sysm)
    (E * torch.tensor([1.0, -2.0], dtype=torch.float64)).sum().backward()
    F = sysm.get("forces")
    rep = sysm.replica_index()
    w = np.array([1.0, -2.0])[rep][:, None]
    np.testing.assert_allclose(x.grad.numpy(), -w * F, rtol=0, atol=0)
    # and against central differences of the energy itself
    x0 = x.detach().clone()
    idx = [(0, 0), (5, 2), (70, 1)]
    for a, k in idx:
        h = 1e-5
        xp, xm = x0.clone(), x0.clone()
        xp[a, k] += h
        xm[a, k] -= h
        d = (Energy.apply(xp, sysm) - Energy.apply(xm, sysm)) / (2 * h)
        assert float(d[rep[a]]) == pytest.approx(-F[a, k], rel=1e-6, abs=1e-7)
    sysm.close()


def test_autograd_force_matching_step_reduces_loss():
    """One gradient step on the parameter vector through the autograd
    wrapper: the loss decreases by about what the gradient predicts."""
    import torch
    from paper_1802_07871_gb300.autograd import ForceMatchingLoss
    structs = _batch()
    Pt = O.with_leaf(P0, ("pair", "SiC", "B"), P0["pair"]["SiC"]["B"] * 1.02)
    ref = [O.evaluate(s.x, s.types, s.box, s.pbc, Pt) for s in structs]
    kw = dict(w_E=[0.1, 0.1], E_ref=[o["E"] for o in ref], w_F=[1.0, 1.0],
              F_ref=np.concatenate([o["F"] for o in ref]))
    sysm = ctbop.System(P0, precision="fp64")
    sysm.load_replicas(structs)
    theta = torch.tensor(ctbop.params_vector(ctbop.params_struct(P0)), dtype=torch.float64, requires_grad=True)
    L0 = ForceMatchingLoss.apply(theta, sysm, *kw.values())
    L0.backward()
    g = theta.grad.clone()
    step = 1e-3 * float(L0) / float((g * g).sum())
    with torch.no_grad():
        L1 = ForceMatchingLoss.apply(theta - step * g, sysm, *kw.values())
    predicted = float(L0) - step * float((g * g).sum())
    assert float(L1) < float(L0)
    assert float(L1) == pytest.approx(predicted, rel=1e-4)
    sysm.close()
