"""Pins for the oracle's velocity-Verlet integrator (the MD of Sec. 3.3):
energy fluctuation scales as dt^2, the FP64 trajectory is time-reversible,
and frozen atoms never move."""
import numpy as np

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")


def _run(dt, nsteps, s, v):
    x, v2, q, et = O.velocity_verlet(s.x, v, s.types, s.box, s.pbc, P1, dt, nsteps, s.frozen)
    return x, v2, et


def test_energy_error_scales_as_dt_squared():
    s = st.sic_3c(2, 4.36, 0.05, seed=1)
    v = st.maxwell_boltzmann(s.types, 600.0, seed=101)
    e0 = O.evaluate(s.x, s.types, s.box, s.pbc, P1)["E"] + O.kinetic_energy(v, s.types, P1)
    _, _, e1 = _run(0.5, 40, s, v)
    _, _, e2 = _run(0.25, 80, s, v)
    d1 = np.max(np.abs(e1 - e0))
    d2 = np.max(np.abs(e2 - e0))
    assert 2.5 < d1 / d2 < 6.0
    assert d1 / len(s.x) < 1e-4


def test_time_reversibility_and_frozen():
    s = st.sic_4h_slab(3, 2, 4, step="strip")
    v = st.maxwell_boltzmann(s.types, 1500.0, seed=7, frozen=s.frozen)
    x1, v1, _ = _run(0.5, 20, s, v)
    assert np.array_equal(x1[s.frozen], s.x[s.frozen])
    s_back = st.Structure("back", x1, s.types, s.box, s.pbc, s.frozen)
    x2, v2, _ = _run(0.5, 20, s_back, -v1)
    assert np.max(np.abs(x2 - s.x)) < 1e-9
    assert np.max(np.abs(v2 + v)) < 1e-9
