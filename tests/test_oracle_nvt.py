"""Pins of the oracle's Nose-Hoover integrator:
  * with a very heavy thermostat (tau -> infinity) it reduces to NVE velocity
    Verlet (the thermostat never acts);
  * its extended energy E + K + Qm xi^2/2 + g kB T0 eta is conserved, with a
    drift that falls as dt^2 (the splitting is second order);
  * a cold start driven by a hotter bath gains kinetic energy."""
import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")


def _small():
    s = st.sic_3c(1, 4.36, 0.05, seed=81)
    v = st.maxwell_boltzmann(s.types, 300.0, seed=82)
    return s, v


def test_heavy_thermostat_is_nve():
    s, v = _small()
    x1, v1, q1, _ = O.velocity_verlet(s.x, v, s.types, s.box, s.pbc, P1, 0.5, 12)
    x2, v2, q2, xi, eta, _ = O.nose_hoover(s.x, v, s.types, s.box, s.pbc, P1, 0.5, 12, T0=300.0, tau=1e12)
    assert np.max(np.abs(x1 - x2)) < 1e-12 and np.max(np.abs(v1 - v2)) < 1e-12
    assert abs(xi) < 1e-20


def test_extended_energy_drift_scales_as_dt_squared():
    s, v = _small()
    drift = []
    for dt, n in ((0.5, 40), (0.25, 80)):
        *_, ext = O.nose_hoover(s.x, v, s.types, s.box, s.pbc, P1, dt, n, T0=900.0, tau=10.0)
        drift.append(np.max(np.abs(ext - ext[0])))
    assert drift[0] < 1e-3 * s.n
    assert 2.5 < drift[0] / drift[1] < 6.0, drift


def test_hot_bath_heats_a_cold_start():
    s, v = _small()
    K0 = O.kinetic_energy(v, s.types, P1)
    _, v1, *_ = O.nose_hoover(s.x, v, s.types, s.box, s.pbc, P1, 0.5, 60, T0=3000.0, tau=5.0)
    assert O.kinetic_energy(v1, s.types, P1) > 2.0 * K0
