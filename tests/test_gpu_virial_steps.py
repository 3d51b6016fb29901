"""MD steps leave the virial out of their force pass; reading it after steps
recomputes it from the state the steps left. It must equal the virial of a
fresh evaluation at the same positions and charges (and reading it must not
change any other result)."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_virial_after_steps_matches_fresh_evaluation(prec):
    s = st.stepped_slab_small(8, 4, 6)
    md = ctbop.System(P1, precision=prec)
    md.load(s, velocities=st.maxwell_boltzmann(s.types, 1500.0, seed=7, frozen=s.frozen))
    md.compute()
    md.step(30, 0.5)
    E0, F0, K0 = md.get("energy"), md.get("forces"), md.get("kinetic")
    W = md.get("virial")
    # the other results are untouched by the recomputation
    assert np.array_equal(md.get("forces"), F0)
    np.testing.assert_allclose(md.get("energy"), E0, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(md.get("kinetic"), K0, rtol=1e-14, atol=1e-12)
    x, q = md.get("positions"), md.get("charges")
    md.close()
    ref = ctbop.System(P1, precision=prec)
    ref.load(s)
    ref.set_positions(x)
    ref.set_charges(q)
    ref.compute(fixed_charges=True)
    Wr = ref.get("virial")
    ref.close()
    scale = max(np.max(np.abs(Wr)), 1.0)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert np.max(np.abs(W - Wr)) / scale < tol, (W, Wr)
    assert np.max(np.abs(Wr)) > 1.0   # a real check: the slab's virial is not small


def test_virial_after_profiled_steps():
    s = st.stepped_slab_small(8, 4, 6)
    md = ctbop.System(P1, precision="fp64")
    md.load(s, velocities=st.maxwell_boltzmann(s.types, 1500.0, seed=8, frozen=s.frozen))
    md.compute()
    md.profile_steps(2, 0.5)
    W = md.get("virial")
    x, q = md.get("positions"), md.get("charges")
    md.close()
    ref = ctbop.System(P1, precision="fp64")
    ref.load(s)
    ref.set_positions(x)
    ref.set_charges(q)
    ref.compute(fixed_charges=True)
    Wr = ref.get("virial")
    ref.close()
    assert np.max(np.abs(W - Wr)) / max(np.max(np.abs(Wr)), 1.0) < 1e-10
