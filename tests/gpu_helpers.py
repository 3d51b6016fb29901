"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare them."""
import numpy as np

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

# Tolerances. FP64 path: limited by the CG stopping rule (rms stationarity
# residual 1e-10 eV/e). Mixed path: the stated targets, force error relative
# to the RMS force 1e-4, energy 1e-6 eV/atom, charges 1e-5 e.
TOL = {
    "fp64": dict(force=1e-8, energy=1e-9, charge=1e-8, virial=1e-8, eatom=1e-8, mu=1e-8),
    "mixed": dict(force=1e-4, energy=1e-6, charge=1e-5, virial=1e-4, eatom=2e-5, mu=1e-5),
    # Stress geometries in mixed precision: FP32 cell-local positions carry
    # ~5e-7 A of rounding, so a term's energy error is about |dE_term/dr| x
    # 5e-7 A, and each stored FP32 charge-matrix entry is rounded by ~6e-8
    # relative. In cells smaller than the charge cutoff every periodic image
    # of a pair rounds alike (~240 correlated terms per atom), and random
    # clusters hold pairs compressed to 1.45 A with 50 eV repulsive terms;
    # there the errors no longer average out. Forces keep the 1e-4 bar.
    "mixed_stress": dict(force=1e-4, energy=5e-6, charge=3e-5, virial=1e-4, eatom=1e-4, mu=3e-5),
}


def gpu_eval(structures, params, precision, Q=None, charges=None, fixed=False, **kw):
    if not isinstance(structures, (list, tuple)):
        structures = [structures]
    sysm = ctbop.System(params, precision=precision, **kw)
    sysm.load_replicas(structures)
    if Q is not None:
        sysm.set_total_charge(Q)
    if charges is not None:
        sysm.set_charges(np.asarray(charges, float))
    sysm.compute(fixed_charges=fixed)
    out = {k: sysm.get(k) for k in ("energy", "forces", "charges", "virial", "e_atom", "mu")}
    out["status"] = sysm.status()
    sysm.close()
    return out


def oracle_eval(s, params, Q=0.0, q=None):
    return O.evaluate(s.x, s.types, s.box, s.pbc, params, Q=Q, q=q)


def compare(g, o, n, precision, sl=slice(None), r=0, check_charges=True, check_mu=True, stress=False):
    """Compare replica r of a GPU result (atoms sl) with an oracle result."""
    t = TOL["mixed_stress" if (stress and precision == "mixed") else precision]
    F, Fo = g["forces"][sl], o["F"]
    rms = max(np.sqrt(np.mean(Fo ** 2)), 1e-3)
    ferr = np.max(np.abs(F - Fo)) / rms if len(Fo) else 0.0
    eerr = abs(g["energy"][r] - o["E"]) / max(n, 1)
    res = {"force": ferr, "energy": eerr}
    assert ferr <= t["force"], (precision, "force", ferr)
    assert eerr <= t["energy"], (precision, "energy", eerr)
    if check_charges and len(Fo):
        qerr = np.max(np.abs(g["charges"][sl] - o["q"]))
        res["charge"] = qerr
        assert qerr <= t["charge"], (precision, "charge", qerr)
    W, Wo = g["virial"][r], o["virial"]
    werr = np.max(np.abs(W - Wo)) / max(np.max(np.abs(Wo)), 1.0)
    res["virial"] = werr
    assert werr <= t["virial"], (precision, "virial", werr)
    if len(Fo):
        aerr = np.max(np.abs(g["e_atom"][sl] - o["e_atom"]))
        res["eatom"] = aerr
        assert aerr <= t["eatom"], (precision, "e_atom", aerr)
    if check_mu and o.get("mu") is not None and len(Fo) > 1:
        merr = abs(g["mu"][r] - o["mu"])
        res["mu"] = merr
        assert merr <= t["mu"], (precision, "mu", merr)
    return res


def local_cut(s, i, rcut):
    """Atoms within rcut of atom i (minimum image along periodic axes), atom
    i first, as an open cluster. Returns (x, types, index map)."""
    d = s.x - s.x[i]
    for a in range(3):
        if s.pbc[a]:
            d[:, a] -= np.round(d[:, a] / s.box[a]) * s.box[a]
    r = np.linalg.norm(d, axis=1)
    idx = np.nonzero(r < rcut)[0]
    idx = np.concatenate([[i], idx[idx != i]])
    return d[idx] + 500.0, s.types[idx], idx


def sampled_local_check(s, params, g, precision, samples, rcut=9.0):
    """Full-size check one atom at a time: with the GPU's charges held fixed,
    the force, per-atom energy and dE/dq of a sampled atom depend only on
    atoms within max(Rc, 2 S_max) of it, so the oracle evaluates a local cut
    exactly. Returns the worst errors."""
    t = TOL[precision]
    q = g["charges"]
    rmsF = np.sqrt(np.mean(g["forces"] ** 2))
    worst = {"force": 0.0, "eatom": 0.0, "stationarity": 0.0}
    for i in samples:
        x, ty, idx = local_cut(s, int(i), rcut)
        sysm = O.System(x, ty, np.full(3, 1000.0), np.array([False] * 3), params)
        Fo = sysm.forces(q[idx])[0]
        eo = sysm.energy(q[idx], per_atom=True)[0]
        dq = sysm.dE_dq(q[idx])[0]
        worst["force"] = max(worst["force"], np.max(np.abs(g["forces"][i] - Fo)) / rmsF)
        worst["eatom"] = max(worst["eatom"], abs(g["e_atom"][i] - eo))
        worst["stationarity"] = max(worst["stationarity"], abs(dq - g["mu"][0]))
    assert worst["force"] <= t["force"], worst
    assert worst["eatom"] <= t["eatom"], worst
    assert worst["stationarity"] <= 10 * t["mu"], worst
    return worst


def oracle_EF(args):
    """(E, F) of one structure from the oracle; a top-level function so a
    spawn pool can run it."""
    s, params = args
    o = O.evaluate(s.x, s.types, s.box, s.pbc, params)
    return o["E"], o["F"]


def oracle_EF_many(structs, params, workers=None):
    """oracle_EF over many structures in a spawn process pool (one BLAS
    thread per worker)."""
    import multiprocessing as mp
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(oracle_EF, [(s, params) for s in structs], chunksize=8)
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [e for e, _ in out], [f for _, f in out]
