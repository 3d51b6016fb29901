"""Si desorption screening on the GPU (Sec. 3.3) against the oracle: the
covalent coordination (index work: exact in FP64), the removal energies of
every surface-Si candidate (batched leave-one-out replicas) and the
screening's decisions; chunking, multi-replica sources, a one-atom replica,
argument errors; at full size (the 19,488-atom stepped slab) sampled
candidates against separately built systems without the atom."""
import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import desorption as D
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")
# removal energies are differences of two total energies, each within 1e-6
# eV/atom (mixed) or 1e-9 (FP64) of the oracle
TOL = {"fp64": 1e-7, "mixed": 1e-6}


def _system(structs, prec):
    sysm = ctbop.System(P1, precision=prec)
    sysm.load_replicas(structs)
    sysm.compute()
    return sysm


def _oracle_candidates(s):
    c = O.coordination(s.x, s.types, s.box, s.pbc, P1)
    return np.nonzero((s.types == 0) & (c < 4) & ~s.frozen)[0], c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_coordination_matches_oracle(prec):
    for s in (st.stepped_slab_small(8, 4, 6), st.sic_3c(2, 4.36, 0.1, seed=3)):
        sysm = _system([s], prec)
        c = sysm.get("coordination")
        sysm.close()
        co = O.coordination(s.x, s.types, s.box, s.pbc, P1)
        bad = np.count_nonzero(c != co)
        assert bad == 0 if prec == "fp64" else bad <= 1, (bad, np.nonzero(c != co))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_removal_energies_match_oracle(prec):
    s = st.stepped_slab_small(6, 3, 4)
    cand, _ = _oracle_candidates(s)
    dEo, rmo = O.desorption_screen(s.x, s.types, s.box, s.pbc, P1, cand, threshold=4.3)
    sysm = _system([s], prec)
    dE = sysm.removal_energies(cand)
    sysm.close()
    np.testing.assert_allclose(dE, dEo, rtol=0, atol=TOL[prec] * s.n)
    # the decisions at a threshold away from every energy
    assert np.min(np.abs(dEo - 4.3)) > 10 * TOL[prec] * s.n
    assert set(cand[dE < 4.3]) == set(rmo)


def test_chunking_and_padding_do_not_change_results():
    s = st.stepped_slab_small(6, 3, 4)
    cand, _ = _oracle_candidates(s)
    sysm = _system([s], "fp64")
    whole = sysm.removal_energies(cand)
    small = sysm.removal_energies(cand, max_atoms=4 * (s.n - 1))   # 4 per chunk, last one padded
    again = sysm.removal_energies(cand[::-1])                      # reuses the batch system
    sysm.close()
    np.testing.assert_allclose(small, whole, rtol=0, atol=1e-9)
    np.testing.assert_allclose(again[::-1], whole, rtol=0, atol=1e-9)


def test_several_source_replicas_and_a_single_atom():
    a = st.stepped_slab_small(6, 3, 4)
    b = st.sic_3c(1, 4.36, 0.1, seed=8)
    one = st.Structure("atom", np.array([[5.0, 5.0, 5.0]]), np.array([0], np.int32), np.full(3, 20.0),
                       np.array([False] * 3))
    structs = [a, b, one]
    off = np.cumsum([0] + [x.n for x in structs])
    ca, _ = _oracle_candidates(a)
    picks = [(0, int(i)) for i in ca[:5]] + [(1, 0), (1, 5), (2, 0)]
    cand = np.array([off[r] + i for r, i in picks])
    sysm = _system(structs, "fp64")
    dE = sysm.removal_energies(cand[::-1])[::-1]                   # mixed order of sources
    sysm.close()
    for (r, i), d in zip(picks, dE):
        s = structs[r]
        ref = O.removal_energy(s.x, s.types, s.box, s.pbc, P1, i)
        assert d == pytest.approx(ref, abs=TOL["fp64"] * s.n), (r, i)


def test_arguments_and_state():
    s = st.stepped_slab_small(6, 3, 4)
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(s)
    with pytest.raises(ctbop.CtbopError, match="STATE"):
        sysm.get("coordination")                                   # no evaluation yet
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.removal_energies([0, s.n])
    assert sysm.removal_energies([]).shape == (0,)
    sysm.close()


def test_full_size_sampled_against_separate_systems():
    """The 19,488-atom stepped slab, every surface Si in one call (in
    chunks); eight sampled candidates against systems built without the atom
    (another code path: host-side removal, a fresh evaluation each)."""
    s = st.stepped_slab_20k()
    sysm = _system([s], "mixed")
    types, frozen = s.types, s.frozen
    cand, coord = D.surface_si(sysm, types, frozen)
    E = sysm.get("energy")[0]
    dE = sysm.removal_energies(cand)
    sysm.close()
    assert len(cand) > 300 and np.all(np.isfinite(dE))
    rng = np.random.default_rng(3)
    for i in rng.choice(len(cand), 8, replace=False):
        a = int(cand[i])
        keep = np.ones(s.n, bool)
        keep[a] = False
        sub = ctbop.System(P1, precision="mixed")
        sub.load(st.Structure("minus one", s.x[keep], s.types[keep], s.box, s.pbc, s.frozen[keep]))
        sub.compute()
        ref = sub.get("energy")[0] + P1["self"]["E0"][0] - E
        sub.close()
        assert dE[i] == pytest.approx(ref, abs=2 * TOL["mixed"] * s.n), (a, dE[i], ref)


def test_desorption_run_removes_and_continues():
    s = st.stepped_slab_small(6, 3, 4)
    v = st.maxwell_boltzmann(s.types, 1500.0, seed=4, frozen=s.frozen)
    run = D.DesorptionRun(s, P1, v, precision="mixed", T0=1500.0, tau=50.0, threshold=100.0)
    ev = run.run(1, steps_per_interval=20)
    n_cand = ev[0].candidates
    assert len(ev[0].removed) == n_cand > 0                       # every candidate is below 100 eV
    assert run.system.n == s.n - n_cand
    ev = run.run(1, steps_per_interval=20)
    assert run.system.status()["rc"] == "OK"
    run.threshold = -100.0
    ev = run.run(1, steps_per_interval=20)
    assert len(ev[-1].removed) == 0
    run.close()
