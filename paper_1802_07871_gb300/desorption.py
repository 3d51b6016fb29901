"""Si desorption during MD (Sec. 3.3): at fixed intervals (1 ps in the paper)
the surface Si atoms are screened by the energy change their elimination
would cause, and those below a threshold are removed, so that the order and
timing of the removals follow from the dynamics rather than being chosen in
advance.

Host orchestration only: the coordination, the removal energies (one batch
of leave-one-out replicas) and the MD run in the library's kernels.

Readings (the paper states neither):
* surface Si = mobile Si atoms with covalent coordination (neighbours within
  the cutoff S of the pair) below 4;
* the removed atoms of one screening are all those below the threshold,
  each evaluated alone from the same state.
Threshold: the paper uses 6.5 eV, 3.5 eV below its typical terrace Si
(about 10 eV). The synthetic parameter set puts terrace Si much lower, so
threshold="relative" takes the median removal energy of the 3-coordinated
candidates (terrace Si) minus 3.5 eV.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ctbop
from . import structures as st

TERRACE_MARGIN = 3.5   # eV below the terrace Si removal energy (Sec. 3.3)


def surface_si(system: ctbop.System, types: np.ndarray, frozen: np.ndarray):
    """Candidates of the screening (mobile Si with coordination < 4) and
    every atom's coordination."""
    coord = system.get("coordination")
    return np.nonzero((types == st.SI) & (coord < 3.5) & ~frozen)[0], coord


def screen(system: ctbop.System, types: np.ndarray, frozen: np.ndarray, threshold=6.5, max_atoms: int = 0):
    """One screening of the current state: (candidates, their removal
    energies, the candidates to remove, the threshold used)."""
    cand, coord = surface_si(system, types, frozen)
    dE = system.removal_energies(cand, max_atoms) if len(cand) else np.empty(0)
    if isinstance(threshold, str):
        if threshold != "relative":
            raise ValueError("threshold: a number (eV) or 'relative'")
        terrace = dE[coord[cand] == 3]
        ref = terrace if len(terrace) else dE
        thr = float(np.median(ref)) - TERRACE_MARGIN if len(ref) else 0.0
    else:
        thr = float(threshold)
    return cand, dE, cand[dE < thr], thr


@dataclass
class Event:
    time_fs: float
    removed: np.ndarray          # original ids of the atoms removed
    energies: np.ndarray         # their removal energies (eV)
    threshold: float
    candidates: int


@dataclass
class DesorptionRun:
    """MD of one structure with Si desorption screening every interval.

    The system is rebuilt from the kept atoms (positions, velocities,
    charges) after each removal; a Nose-Hoover thermostat, if set, restarts
    from xi = eta = 0 then."""
    structure: st.Structure
    params: dict
    velocities: np.ndarray
    precision: str = "mixed"
    T0: float | None = None
    tau: float = 100.0
    threshold: float | str = 6.5
    max_atoms: int = 0
    ids: np.ndarray = field(init=False)
    events: list = field(default_factory=list)
    time_fs: float = 0.0

    def __post_init__(self):
        s = self.structure
        self.ids = np.arange(s.n)
        self._x, self._v = s.x.copy(), np.asarray(self.velocities, float).copy()
        self._t, self._f = s.types.copy(), s.frozen.copy()
        self._q = None
        self._sys = None
        self._make()

    def _make(self):
        if self._sys is not None:
            self._sys.close()
        s = self.structure
        sysm = ctbop.System(self.params, precision=self.precision)
        sysm.load(st.Structure(s.name, self._x, self._t, s.box, s.pbc, self._f), velocities=self._v)
        if self._q is not None:
            sysm.set_charges(self._q)
        if self.T0:
            sysm.set_thermostat(self.T0, self.tau)
        self._sys = sysm

    @property
    def system(self) -> ctbop.System:
        return self._sys

    def run(self, n_intervals: int, steps_per_interval: int = 2000, dt: float = 0.5):
        """n_intervals times: steps_per_interval MD steps, then a screening
        and the removals it decides."""
        for _ in range(n_intervals):
            self._sys.step(steps_per_interval, dt)
            self.time_fs += steps_per_interval * dt
            cand, dE, rm, thr = screen(self._sys, self._t, self._f, self.threshold, self.max_atoms)
            if len(rm) == 0:
                self.events.append(Event(self.time_fs, np.empty(0, int), np.empty(0), thr, len(cand)))
                continue
            self.events.append(Event(self.time_fs, self.ids[rm], dE[np.isin(cand, rm)], thr, len(cand)))
            keep = np.ones(len(self._t), bool)
            keep[rm] = False
            self._x = self._sys.get("positions")[keep]
            self._v = self._sys.get("velocities")[keep]
            self._q = self._sys.get("charges")[keep]
            self._t, self._f, self.ids = self._t[keep], self._f[keep], self.ids[keep]
            self._make()
        return self.events

    def close(self):
        if self._sys is not None:
            self._sys.close()
            self._sys = None
