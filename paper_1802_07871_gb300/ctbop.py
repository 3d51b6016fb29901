"""Thin ctypes binding of libctbop (include/ctbop.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. Host arrays are numpy arrays; device arrays are torch CUDA tensors
(their data_ptr() is passed with CTBOP_DEVICE). There is no CPU fallback: if
the library is not built this module raises on first use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .structures import TYPE_NAMES

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libctbop.so")

OK = 0
ERR = {
    -1: "INVALID_ARG", -2: "OOM", -3: "NEIGH_OVERFLOW", -4: "CG_NOT_CONVERGED",
    -5: "NONFINITE", -6: "CUDA", -7: "STATE",
}
HOST, DEVICE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
FIXED_CHARGES = 1
GET = {"energy": 0, "forces": 1, "charges": 2, "positions": 3, "velocities": 4,
       "virial": 5, "e_atom": 6, "mu": 7, "kinetic": 8, "thermostat": 9, "coordination": 10}

# every symbol include/ctbop.h declares
EXPORTS = (
    "ctbop_default_options", "ctbop_create", "ctbop_destroy", "ctbop_last_error",
    "ctbop_set_stream", "ctbop_set_layout", "ctbop_set_box", "ctbop_set_types",
    "ctbop_set_positions", "ctbop_set_velocities", "ctbop_set_charges", "ctbop_set_frozen",
    "ctbop_set_total_charge", "ctbop_compute", "ctbop_step", "ctbop_get", "ctbop_status",
    "ctbop_profile_steps", "ctbop_energy_noalloc", "ctbop_param_grad", "ctbop_set_params", "ctbop_set_thermostat",
    "ctbop_removal_energies", "ctbop_minimize", "ctbop_rings", "ctbop_set_order",
    "ctbop_measure_peaks",
)
# one record of ctbop_rings (struct ctbop_ring)
RING_DTYPE = np.dtype([("replica", "<i4"), ("size", "<i4"), ("centre", "<f8", 3), ("orientation", "<f8")])
NPHASE = 10
PHASES = ("kick_drift", "lists", "bond", "assemble", "cg_start", "cg_matvec", "cg_update",
          "cg_charges", "cov_force", "coul_gather_kick")

D4 = C.c_double * 4
D2x4 = (C.c_double * 2) * 4
D2x8 = (C.c_double * 2) * 8
D2 = C.c_double * 2


class Params(C.Structure):
    _fields_ = [
        ("A", D4), ("B", D4), ("lambda1", D4), ("lambda2", D4), ("R", D4), ("S", D4), ("kappa", D4),
        ("sigma", D4), ("p", D4), ("g", D2x4), ("n", D2x4),
        ("gamma", D2x8), ("c", D2x8), ("d", D2x8), ("h", D2x8), ("alpha", D2x8),
        ("E0", D2), ("chi", D2), ("J", D2), ("gamma_c", D2), ("mass", D2),
        ("r_coul", C.c_double), ("k_e", C.c_double),
    ]


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("cg_max_iter", C.c_int32), ("cg_tol", C.c_double),
        ("skin", C.c_double), ("cap_cov", C.c_int32), ("cap_all", C.c_int32),
        ("device", C.c_int32), ("precond", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("rebuilds", C.c_int64), ("cg_iters_last", C.c_int32),
        ("max_cov", C.c_int32), ("cg_iters_total", C.c_int64), ("solves", C.c_int64),
        ("cg_residual_last", C.c_double), ("max_all", C.c_int32), ("error_bits", C.c_uint32),
        ("mean_cov", C.c_double), ("mean_all", C.c_double), ("cg_residual_start", C.c_double),
        ("cg_mv_batch", C.c_int32), ("asm_batch", C.c_int32), ("cg_mv_ms", C.c_double * 3),
        ("mean_mat", C.c_double), ("asm_ms", C.c_double * 3),
        ("gather_batch", C.c_int32), ("fp64_atoms", C.c_int32), ("fp64_bonds", C.c_int32), ("pad", C.c_int32),
        ("gather_ms", C.c_double * 3), ("cov_lanes", C.c_int32), ("pad2", C.c_int32), ("cov_ms", C.c_double * 3),
        ("build_warps", C.c_int32), ("build_batch", C.c_int32), ("build_ms", C.c_double * 6),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["cg_mv_ms"] = list(self.cg_mv_ms)
        d["asm_ms"] = list(self.asm_ms)
        d["gather_ms"] = list(self.gather_ms)
        d["cov_ms"] = list(self.cov_ms)
        d["build_ms"] = list(self.build_ms)
        d.pop("pad", None)
        d.pop("pad2", None)
        return d


class Peaks(C.Structure):
    _fields_ = [
        ("fp32_tflops", C.c_double), ("mufu_ex2_tops", C.c_double), ("mufu_rsq_tops", C.c_double),
        ("fp64_tflops", C.c_double), ("ms", C.c_double * 4), ("sm_mhz", C.c_double),
        ("sms", C.c_int32), ("pad", C.c_int32),
    ]


_lib = None


def lib():
    """Load libctbop.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is not built; run paper_1802_07871_gb300.build.build()")
    L = C.CDLL(_LIB_PATH)
    vp = C.c_void_p
    sig = {
        "ctbop_default_options": ([C.POINTER(Options)], C.c_int),
        "ctbop_create": ([C.POINTER(Params), C.POINTER(Options), C.POINTER(vp)], C.c_int),
        "ctbop_destroy": ([vp], C.c_int),
        "ctbop_last_error": ([vp], C.c_char_p),
        "ctbop_set_stream": ([vp, vp], C.c_int),
        "ctbop_set_layout": ([vp, C.c_int32, vp], C.c_int),
        "ctbop_set_box": ([vp, vp, vp], C.c_int),
        "ctbop_set_types": ([vp, vp, C.c_int], C.c_int),
        "ctbop_set_positions": ([vp, vp, C.c_int], C.c_int),
        "ctbop_set_velocities": ([vp, vp, C.c_int], C.c_int),
        "ctbop_set_charges": ([vp, vp, C.c_int], C.c_int),
        "ctbop_set_frozen": ([vp, vp, C.c_int], C.c_int),
        "ctbop_set_total_charge": ([vp, vp], C.c_int),
        "ctbop_compute": ([vp, C.c_uint32], C.c_int),
        "ctbop_step": ([vp, C.c_int64, C.c_double], C.c_int),
        "ctbop_get": ([vp, C.c_int, vp, C.c_int], C.c_int),
        "ctbop_status": ([vp, C.POINTER(Stats)], C.c_int),
        "ctbop_profile_steps": ([vp, C.c_int64, C.c_double, vp, vp], C.c_int),
        "ctbop_removal_energies": ([vp, C.c_int64, vp, C.c_int64, vp], C.c_int),
        "ctbop_minimize": ([vp, C.c_int64, C.c_double, C.c_double, C.c_double, vp, vp], C.c_int),
        "ctbop_rings": ([vp, C.c_double, C.c_int32, C.c_int64, vp, vp], C.c_int),
        "ctbop_set_order": ([vp, vp], C.c_int),
        "ctbop_measure_peaks": ([C.c_int32, vp, C.POINTER(Peaks)], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def measure_peaks(device: int = 0, stream=None) -> dict:
    """FP32 FMA, special-function (ex2, rsqrt) and FP64 FMA rates of the GPU
    (ctbop_measure_peaks), with the SM clock they were taken at."""
    out = Peaks()
    ptr = None if stream is None else int(stream)
    rc = lib().ctbop_measure_peaks(int(device), ptr, C.byref(out))
    if rc != OK:
        raise CtbopError(f"ctbop_measure_peaks: {ERR.get(rc, rc)}")
    return {"fp32_tflops": out.fp32_tflops, "mufu_ex2_tops": out.mufu_ex2_tops,
            "mufu_rsq_tops": out.mufu_rsq_tops, "fp64_tflops": out.fp64_tflops,
            "ms": list(out.ms), "sm_mhz": out.sm_mhz, "sms": out.sms}


def params_struct(d: dict) -> Params:
    """Marshal a parameter dictionary (the JSON layout of params/*.json) into
    the C struct. A set with L = 1 gets an inert second component
    (g_2 = 1e30, n_2 = 1, gamma_2 = 0), which leaves Eq. 7 equal to the L = 1
    form to far below double rounding."""
    P = Params()
    T = TYPE_NAMES
    for a in range(2):
        for b in range(2):
            k = a * 2 + b
            pr = d["pair"][T[min(a, b)] + T[max(a, b)]]
            P.A[k], P.B[k] = pr["A"], pr["B"]
            P.lambda1[k], P.lambda2[k] = pr["lambda1"], pr["lambda2"]
            P.R[k], P.S[k], P.kappa[k] = pr["R"], pr["S"], pr["kappa"]
            bo = d["bond"][T[a] + T[b]]
            P.sigma[k], P.p[k] = bo["sigma"], bo["p"]
            g, n = list(bo["g"]), list(bo["n"])
            if len(g) == 1:
                g, n = g + [1e30], n + [1.0]
            P.g[k][0], P.g[k][1] = g
            P.n[k][0], P.n[k][1] = n
            for c in range(2):
                t = (a * 2 + b) * 2 + c
                tp = d["triplet"][T[a] + T[b] + T[c]]
                for key, dst in (("gamma", P.gamma), ("c", P.c), ("d", P.d), ("h", P.h), ("alpha", P.alpha)):
                    vals = list(tp[key])
                    if len(vals) == 1:
                        vals = vals + ([0.0] if key == "gamma" else [1.0 if key in ("c", "d") else 0.0])
                    dst[t][0], dst[t][1] = vals
    se, co = d["self"], d["coulomb"]
    for t in range(2):
        P.E0[t], P.chi[t], P.J[t] = se["E0"][t], se["chi"][t], se["J"][t]
        P.gamma_c[t], P.mass[t] = co["gamma"][t], d["mass"][t]
    P.r_coul, P.k_e = co["r_coul"], co["k_e"]
    return P


def morton_order(x, box, pbc, cell: float = 2.5) -> np.ndarray:
    """Indices of the atoms along a Morton (Z-order) curve over a grid of
    `cell` A cells (periodic axes wrapped into the box first): neighbouring
    indices are then neighbouring atoms. A storage order for
    System.set_order."""
    x = np.asarray(x, float).copy()
    box, pbc = np.asarray(box, float), np.asarray(pbc, bool)
    x = np.where(pbc, np.mod(x, np.where(pbc, box, 1.0)), x)
    c = np.floor((x - x.min(axis=0)) / cell).astype(np.int64) if len(x) else np.zeros((0, 3), np.int64)
    c = np.clip(c, 0, (1 << 20) - 1)
    key = np.zeros(len(x), dtype=np.int64)
    for b in range(20):
        for d in range(3):
            key |= ((c[:, d] >> b) & 1) << (3 * b + d)
    return np.argsort(key, kind="stable")


def params_vector(P: Params) -> np.ndarray:
    """The struct as its 144 doubles (field order of ctbop_params)."""
    return np.frombuffer(bytes(P), dtype=np.float64).copy()


def params_from_vector(v) -> Params:
    """A struct from 144 doubles in field order."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    if v.size != C.sizeof(Params) // 8:
        raise ValueError("need 144 parameters")
    return Params.from_buffer_copy(v.tobytes())


def grad_to_dict(G: Params, d: dict) -> dict:
    """Map a gradient in the layout of the C struct back onto the keys of the
    parameter dictionary d (the JSON layout): every struct entry is a copy of
    one dictionary entry, so a dictionary entry's derivative is the sum over
    the struct entries copied from it (a symmetric pair constant feeds both
    ordered pairs; the inert second component of an L = 1 set feeds none)."""
    T = TYPE_NAMES
    out = {"pair": {}, "bond": {}, "triplet": {}, "self": {}, "coulomb": {}}
    for key, pr in d["pair"].items():
        out["pair"][key] = {f: 0.0 for f in ("A", "B", "lambda1", "lambda2", "R", "S", "kappa")}
    fmap = {"A": "A", "B": "B", "lambda1": "lambda1", "lambda2": "lambda2", "R": "R", "S": "S", "kappa": "kappa"}
    for a in range(2):
        for b in range(2):
            k = a * 2 + b
            pk = T[min(a, b)] + T[max(a, b)]
            for f, sf in fmap.items():
                out["pair"][pk][f] += getattr(G, sf)[k]
            bo = d["bond"][T[a] + T[b]]
            L = len(bo["g"])
            out["bond"][T[a] + T[b]] = {"sigma": G.sigma[k], "p": G.p[k],
                                         "g": [G.g[k][l] for l in range(L)], "n": [G.n[k][l] for l in range(L)]}
            for c in range(2):
                t = (a * 2 + b) * 2 + c
                tp = d["triplet"][T[a] + T[b] + T[c]]
                out["triplet"][T[a] + T[b] + T[c]] = {
                    key: [getattr(G, key)[t][l] for l in range(len(tp[key]))]
                    for key in ("gamma", "c", "d", "h", "alpha")}
    out["self"] = {"E0": [G.E0[t] for t in range(2)], "chi": [G.chi[t] for t in range(2)],
                   "J": [G.J[t] for t in range(2)]}
    out["coulomb"] = {"gamma": [G.gamma_c[t] for t in range(2)], "r_coul": G.r_coul, "k_e": G.k_e}
    return out


def _ptr(a):
    """(pointer, mem) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_buffer(a, dtype, count: int, what: str):
    """A caller's buffer (numpy array or torch tensor) that the library will
    read or write `count` elements of `dtype` from: its element type and its
    size must match, or the library would read or write past it."""
    dt = np.dtype(dtype)
    if isinstance(a, np.ndarray):
        if a.dtype != dt:
            raise TypeError(f"{what}: need {dt.name} elements, got {a.dtype}")
        n = a.size
    elif hasattr(a, "data_ptr"):
        tn = str(a.dtype).replace("torch.", "")
        if not (tn == dt.name or (dt == np.uint8 and tn == "bool")):
            raise TypeError(f"{what}: need {dt.name} elements, got {tn}")
        n = a.numel()
    else:
        raise TypeError(f"{what}: unsupported array type {type(a)}")
    if n != count:
        raise ValueError(f"{what}: need {count} elements, got {n}")


class CtbopError(RuntimeError):
    pass


class System:
    """One simulation (one or more replicas) on one GPU."""

    def __init__(self, params: dict, precision: str = "mixed", skin: float = 0.3,
                 cg_tol: float = 0.0, cg_max_iter: int = 200, device: int = 0,
                 cap_cov: int = 0, cap_all: int = 0, precond: str = "block"):
        L = lib()
        self._L = L
        o = Options()
        L.ctbop_default_options(C.byref(o))
        o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        o.skin, o.cg_tol, o.cg_max_iter, o.device = skin, cg_tol, cg_max_iter, device
        o.cap_cov, o.cap_all = cap_cov, cap_all
        if precond not in ("block", "jacobi"):
            raise ValueError("precond: 'block' or 'jacobi'")
        o.precond = 0 if precond == "block" else 1
        self._p = params_struct(params)
        h = C.c_void_p()
        rc = L.ctbop_create(C.byref(self._p), C.byref(o), C.byref(h))
        if rc != OK:
            raise CtbopError(f"ctbop_create failed: {ERR.get(rc, rc)}")
        self._h = h
        self.n = 0
        self.R = 0
        self.precision = precision
        self.device = device

    def _check(self, rc, what):
        if rc != OK:
            msg = self._L.ctbop_last_error(self._h).decode()
            raise CtbopError(f"{what}: {ERR.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.ctbop_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup
    def set_stream(self, stream_handle: int):
        self._check(self._L.ctbop_set_stream(self._h, C.c_void_p(stream_handle)), "set_stream")

    def set_params_struct(self, P: Params):
        """Replace the parameters from a filled struct (e.g. one built from a
        parameter vector, see params_from_vector)."""
        self._p = P
        self._check(self._L.ctbop_set_params(self._h, C.byref(self._p)), "set_params")

    def replica_index(self) -> np.ndarray:
        """Replica of every atom (from the layout)."""
        return np.repeat(np.arange(self.R), np.diff(self._offsets))

    def set_thermostat(self, T0, tau):
        """Nose-Hoover thermostat per replica (T0 in K, tau in fs; T0 <= 0:
        NVE for that replica; T0=None: all NVE)."""
        if T0 is None:
            self._check(self._L.ctbop_set_thermostat(self._h, None, None), "set_thermostat")
            return
        t0 = np.ascontiguousarray(np.broadcast_to(np.asarray(T0, float), (self.R,)))
        ta = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, float), (self.R,)))
        self._check(self._L.ctbop_set_thermostat(self._h, t0.ctypes.data_as(C.c_void_p),
                                                 ta.ctypes.data_as(C.c_void_p)), "set_thermostat")

    def set_params(self, params: dict):
        """Replace the potential's parameters (the next evaluation rebuilds
        lists and graphs as needed)."""
        self._p = params_struct(params)
        self._check(self._L.ctbop_set_params(self._h, C.byref(self._p)), "set_params")

    def param_grad(self, w_E=None, E_ref=None, w_F=None, F_ref=None):
        """Force-matching loss and its gradient with respect to every field
        of the parameter struct, in the system's precision policy: returns
        (loss, Params)."""
        def arr(a, n):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(n)
            return a, a.ctypes.data_as(C.c_void_p)
        wE, pwE = arr(w_E, self.R)
        Er, pEr = arr(E_ref, self.R)
        wF, pwF = arr(w_F, self.R)
        Fr, pFr = arr(F_ref, 3 * self.n)
        loss = C.c_double(0.0)
        G = Params()
        self._check(self._L.ctbop_param_grad(self._h, pwE, pEr, pwF, pFr, C.byref(loss), C.byref(G)),
                    "param_grad")
        return loss.value, G

    def set_layout(self, offsets):
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self._L.ctbop_set_layout(self._h, len(off) - 1, off.ctypes.data_as(C.c_void_p)), "set_layout")
        self._offsets = off.copy()
        self.n = int(off[-1])
        self.R = len(off) - 1

    def set_box(self, lengths, pbc):
        lengths = np.asarray(lengths, dtype=np.float64).reshape(-1, 3)
        h = np.zeros((len(lengths), 3, 3))
        for r in range(len(lengths)):
            h[r] = np.diag(lengths[r])
        h = np.ascontiguousarray(h)
        p = np.ascontiguousarray(np.asarray(pbc).reshape(-1, 3), dtype=np.uint8)
        if self.R > 0 and (len(h) != self.R or len(p) != self.R):
            raise ValueError(f"set_box: need {self.R} boxes and pbc rows, got {len(h)} and {len(p)}")
        self._check(self._L.ctbop_set_box(self._h, h.ctypes.data_as(C.c_void_p), p.ctypes.data_as(C.c_void_p)),
                    "set_box")

    def _set(self, fn, a, dtype, what, per_atom=1):
        if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(a, dtype=dtype)
        if self.R > 0:   # without a layout the library reports the state error
            _check_buffer(a, dtype, per_atom * self.n, what)
        if getattr(a, "is_cuda", False) and a.device.index != self.device:
            raise ValueError(f"{what}: tensor on cuda:{a.device.index}, system on cuda:{self.device}")
        ptr, mem = _ptr(a)
        self._keep = a
        self._check(fn(self._h, ptr, mem), what)

    def set_types(self, t):
        self._set(self._L.ctbop_set_types, t, np.int32, "set_types")

    def set_positions(self, x):
        self._set(self._L.ctbop_set_positions, x, np.float64, "set_positions", 3)

    def set_velocities(self, v):
        self._set(self._L.ctbop_set_velocities, v, np.float64, "set_velocities", 3)

    def set_charges(self, q):
        self._set(self._L.ctbop_set_charges, q, np.float64, "set_charges")

    def set_frozen(self, f):
        self._set(self._L.ctbop_set_frozen, f, np.uint8, "set_frozen")

    def set_total_charge(self, Q):
        Q = np.atleast_1d(np.asarray(Q, dtype=np.float64))
        if self.R > 0:
            Q = np.ascontiguousarray(np.broadcast_to(Q, (self.R,)))
        self._check(self._L.ctbop_set_total_charge(self._h, Q.ctypes.data_as(C.c_void_p)), "set_total_charge")

    def set_order(self, order):
        """Storage order (after set_layout, before the per-atom arrays):
        order[k] is the caller's index of the atom stored in slot k. Inputs
        and outputs stay in the caller's order."""
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        if o is not None and self.R > 0:
            _check_buffer(o, np.int64, self.n, "set_order")
        self._check(self._L.ctbop_set_order(self._h, None if o is None else o.ctypes.data_as(C.c_void_p)),
                    "set_order")

    def load(self, structure, velocities=None, charges=None, order="morton"):
        """Set layout, box, types, positions and frozen mask of one structure
        (stored along a Morton curve unless order=None)."""
        s = structure
        self.set_layout([0, s.n])
        if order == "morton":
            self.set_order(morton_order(s.x, s.box, s.pbc))
        self.set_box(s.box, s.pbc)
        self.set_types(s.types)
        self.set_positions(s.x)
        self.set_frozen(s.frozen.astype(np.uint8))
        if velocities is not None:
            self.set_velocities(velocities)
        if charges is not None:
            self.set_charges(charges)

    def load_replicas(self, structures, order="morton"):
        """Set the layout and every array of a batch of structures (each
        replica stored along a Morton curve unless order=None)."""
        off = np.concatenate([[0], np.cumsum([s.n for s in structures])])
        self.set_layout(off)
        if order == "morton":
            self.set_order(np.concatenate([o + morton_order(s.x, s.box, s.pbc) for o, s in zip(off, structures)]))
        self.set_box(np.array([s.box for s in structures]), np.array([s.pbc for s in structures]))
        self.set_types(np.concatenate([s.types for s in structures]))
        self.set_positions(np.concatenate([s.x for s in structures]))
        self.set_frozen(np.concatenate([s.frozen for s in structures]).astype(np.uint8))

    # ---- run
    def compute(self, fixed_charges: bool = False):
        self._check(self._L.ctbop_compute(self._h, FIXED_CHARGES if fixed_charges else 0), "compute")

    def step(self, n: int, dt: float):
        self._check(self._L.ctbop_step(self._h, int(n), float(dt)), "step")

    def profile_steps(self, n: int, dt: float) -> dict:
        """Per-phase GPU time (ms, summed) and launch counts over n steps."""
        ms = np.zeros(NPHASE)
        cnt = np.zeros(NPHASE, dtype=np.int64)
        self._check(self._L.ctbop_profile_steps(self._h, int(n), float(dt), ms.ctypes.data_as(C.c_void_p),
                                                cnt.ctypes.data_as(C.c_void_p)), "profile_steps")
        return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(PHASES)}

    def energy_noalloc(self) -> np.ndarray:
        """Per-replica energy through the entry point that allocates nothing
        on the device (at most 64 replicas), for callers that cannot allocate
        while reading energies (GPU memory held by another framework's
        caching allocator; monitoring code that must not synchronise the
        device through a cudaFree)."""
        out = np.empty(self.R, dtype=np.float64)
        self._check(self._L.ctbop_energy_noalloc(self._h, out.ctypes.data_as(C.c_void_p)), "energy_noalloc")
        return out

    def removal_energies(self, candidates, max_atoms: int = 0) -> np.ndarray:
        """Energy change (eV) when each candidate atom (global index) is
        eliminated alone from the current state, the rest in place, charges
        re-minimised, the atom leaving neutral (E0 of its type): the
        stability measure of the desorption screening."""
        c = np.ascontiguousarray(candidates, dtype=np.int64).reshape(-1)
        out = np.empty(len(c), dtype=np.float64)
        self._check(self._L.ctbop_removal_energies(self._h, len(c), c.ctypes.data_as(C.c_void_p), int(max_atoms),
                                                   out.ctypes.data_as(C.c_void_p)), "removal_energies")
        return out

    def minimize(self, max_iter: int = 1000, fmax: float = 1e-3, dt0: float = 1.0, dt_max: float = 5.0):
        """FIRE relaxation of every replica (charges re-minimised at every
        force evaluation). Returns (iterations per replica, -1 where max_iter
        was reached first; max |F_i| per replica at the end)."""
        it = np.empty(self.R, dtype=np.int64)
        fm = np.empty(self.R, dtype=np.float64)
        self._check(self._L.ctbop_minimize(self._h, int(max_iter), float(fmax), float(dt0), float(dt_max),
                                           it.ctypes.data_as(C.c_void_p), fm.ctypes.data_as(C.c_void_p)),
                    "minimize")
        return it, fm

    def rings(self, bond_cut: float = 0.0, max_size: int = 8) -> np.ndarray:
        """Primitive C rings of the current state (records of RING_DTYPE, in
        no particular order); bond_cut 0 = the C-C covalent cutoff."""
        cap = max(1024, self.n)
        while True:
            out = np.empty(cap, dtype=RING_DTYPE)
            n = C.c_int64(0)
            self._check(self._L.ctbop_rings(self._h, float(bond_cut), int(max_size), cap,
                                            out.ctypes.data_as(C.c_void_p), C.byref(n)), "rings")
            if n.value <= cap:
                return out[:n.value].copy()
            cap = n.value

    def status(self) -> dict:
        st = Stats()
        rc = self._L.ctbop_status(self._h, C.byref(st))
        d = st.as_dict()
        d["rc"] = ERR.get(rc, rc) if rc else "OK"
        return d

    def get(self, what: str, out=None):
        """Copy a result out. Without `out` returns a numpy array (synchronises);
        `out` may be a numpy array or a torch tensor (device copy is
        stream-ordered)."""
        sel = GET[what]
        shape = {"energy": (self.R,), "mu": (self.R,), "kinetic": (self.R,), "virial": (self.R, 3, 3),
                 "forces": (self.n, 3), "positions": (self.n, 3), "velocities": (self.n, 3),
                 "charges": (self.n,), "e_atom": (self.n,), "thermostat": (self.R, 4),
                 "coordination": (self.n,)}[what]
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        _check_buffer(out, np.float64, int(np.prod(shape)), f"get {what}")
        if getattr(out, "is_cuda", False) and out.device.index != self.device:
            raise ValueError(f"get {what}: tensor on cuda:{out.device.index}, system on cuda:{self.device}")
        ptr, mem = _ptr(out)
        self._check(self._L.ctbop_get(self._h, sel, ptr, mem), f"get {what}")
        return out
