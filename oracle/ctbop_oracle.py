"""FP64 CPU oracle for the charge-transfer bond-order potential.

TEST INFRASTRUCTURE ONLY. Only the test-suite, the package smoke check and the
benchmark's CPU-baseline leg may import this module. The product path (the
CUDA library and its binding) never calls it and has no CPU fallback.

Plain, slow and direct: every quantity is the definition written out in
float64 with numpy, with library primitives (a k-d tree for neighbour search,
a dense linear solve, scipy's CG) as single steps. It shares no code with the
CUDA library.

What it computes (paper sections and equations; readings R1-R3 and numbered
readings are the model card, stated where used):

* Bond order, Sec. 2 Eq. 3-5 for any L and p (the GPU implements the L = 2
  expanded form, Eq. 7). The normalisation G makes b = 1 when every zeta_l = 0
  (Sec. 2, text after Eq. 5). Eq. 6 (p -> inf) and Eq. 1 (Tersoff) are
  provided for the pins.
* Environment sums zeta_l,ij (Eq. 2, one per l): sum over k != i, j of
  f_c(r_ik) ang_l(cos theta_ijk) exp(alpha_l (r_ij - r_ik))   [reading R1].
* Pair energy per directed bond (reading R1, Tersoff 1988 philosophy kept as
  Sec. 2 asks):
      E_ij = 1/2 f_c(r) [ A e^(-lambda1 r) - c_ij b_ij B e^(-lambda2 r) ]
  with the covalent-ionic factor c_ij = 1 - kappa (q_i - q_j)^2   [reading R2,
  the f_q mixing the paper names but does not print].
* Self energy U_i = E0_t + chi_t q_i + J_t q_i^2 (the constant E0 is the term
  Sec. 2 adds to U^Self) and shielded, tapered charge interaction
      1/2 sum_i sum_j' q_i q_j k_e T(r/Rc) / (r^3 + gamma_ij^-3)^(1/3)
  over every periodic image inside Rc, self-images included   [reading R3].
* Charges minimise E_tot at fixed positions (Sec. 2): with E quadratic in q,
  the minimiser under sum q = Q solves H q + chi = mu 1 (dense KKT solve, or
  CG for large systems).
* Forces -dE/dx at fixed q (exact at the minimiser because dE/dq_i = mu for
  all i and sum_i dq_i/dx = 0), virial W = -sum_u u (x) dE/du over every
  relative vector u, per-atom energies.
* Velocity-Verlet NVE with frozen atoms (the paper runs MD with a fixed
  substrate bottom, Sec. 3.3).
* NVT by one Nose-Hoover thermostat per system (the paper's MD is NVT,
  Sec. 3.3, with no thermostat named). Pinned: a heavy thermostat gives the
  NVE trajectory, the extended energy drifts as dt^2, and a hot bath heats a
  cold start.
* Parameter gradients of a force-matching loss on E and F (the paper fits
  its parameters to energies, forces and charges, Sec. 2, without a method):
  central differences of the loss, Richardson-extrapolated. Pinned: closed
  forms for the self-energy parameters, the repulsion prefactor and the
  Coulomb constant; F does not depend on E0.
* Si desorption screening (Sec. 3.3): covalent coordination and the energy
  change on removing one atom with the charges re-solved. Pinned: the SiC
  dimer and linear Si3 in closed form, a far atom of an all-Si system,
  equivalent sites of an ideal crystal.
* FIRE minimisation (Bitzek et al. 2006; the paper relaxes structures
  without naming a method). Pinned: closed-form minima of the dimer and of
  linear Si3, an ideal crystal takes no iteration, descent with frozen
  atoms.
* Primitive rings of the C network and the 6-ring orientation (Sec. 3.3
  follows 5-, 6- and 7-rings). Pinned: perfect graphene, a Stone-Wales
  defect, lone polygons, two squares sharing an edge, rotation, and a path
  around a periodic box that is no ring.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TYPE_KEYS = ("Si", "C")
ACC = 9.648533212e-3          # 1 eV/(A u) in A/fs^2
KB = 8.617333262e-5           # eV/K


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------
@dataclass
class Tables:
    """Parameter tables indexed by type: pair [ti,tj], bond-order [ti,tj],
    triplet [ti,tj,tk,l], per type [t]."""
    A: np.ndarray
    B: np.ndarray
    lam1: np.ndarray
    lam2: np.ndarray
    R: np.ndarray
    S: np.ndarray
    kappa: np.ndarray
    sigma: np.ndarray
    p: np.ndarray
    g: np.ndarray        # [2,2,L]
    n: np.ndarray        # [2,2,L]
    gam: np.ndarray      # [2,2,2,L]
    c: np.ndarray
    d: np.ndarray
    h: np.ndarray
    alpha: np.ndarray
    E0: np.ndarray
    chi: np.ndarray
    J: np.ndarray
    gam_c: np.ndarray
    mass: np.ndarray
    r_coul: float
    k_e: float
    L: int


def tables(params: dict) -> Tables:
    """Unpack a parameter dictionary (the JSON layout) into index tables."""
    L = len(next(iter(params["bond"].values()))["g"])
    z2 = lambda: np.zeros((2, 2))
    A, B, l1, l2, R, S, kap = (z2() for _ in range(7))
    for a in range(2):
        for b in range(2):
            key = TYPE_KEYS[min(a, b)] + TYPE_KEYS[max(a, b)]
            pr = params["pair"][key]
            A[a, b], B[a, b] = pr["A"], pr["B"]
            l1[a, b], l2[a, b] = pr["lambda1"], pr["lambda2"]
            R[a, b], S[a, b], kap[a, b] = pr["R"], pr["S"], pr["kappa"]
    sig, p = z2(), z2()
    g, n = np.zeros((2, 2, L)), np.zeros((2, 2, L))
    for a in range(2):
        for b in range(2):
            bo = params["bond"][TYPE_KEYS[a] + TYPE_KEYS[b]]
            sig[a, b], p[a, b] = bo["sigma"], bo["p"]
            g[a, b], n[a, b] = bo["g"], bo["n"]
    trip = {k: np.zeros((2, 2, 2, L)) for k in ("gamma", "c", "d", "h", "alpha")}
    for a in range(2):
        for b in range(2):
            for c in range(2):
                tp = params["triplet"][TYPE_KEYS[a] + TYPE_KEYS[b] + TYPE_KEYS[c]]
                for k in trip:
                    trip[k][a, b, c] = tp[k]
    se = params["self"]
    co = params["coulomb"]
    return Tables(A, B, l1, l2, R, S, kap, sig, p, g, n,
                  trip["gamma"], trip["c"], trip["d"], trip["h"], trip["alpha"],
                  np.array(se["E0"], float), np.array(se["chi"], float),
                  np.array(se["J"], float), np.array(co["gamma"], float),
                  np.array(params["mass"], float), float(co["r_coul"]),
                  float(co["k_e"]), L)


# ----------------------------------------------------------------------------
# elementary functions of the model card
# ----------------------------------------------------------------------------
def cutoff(r, R, S):
    """Tersoff cutoff (reading R1): 1 below R, 1/2[1 + cos(pi (r-R)/(S-R))]
    between R and S, 0 beyond S. Returns (f_c, df_c/dr)."""
    r = np.asarray(r, float)
    t = np.clip((r - R) / (S - R), 0.0, 1.0)
    f = np.where(r < R, 1.0, np.where(r >= S, 0.0, 0.5 * (1.0 + np.cos(np.pi * t))))
    df = np.where((r > R) & (r < S), -0.5 * np.pi / (S - R) * np.sin(np.pi * t), 0.0)
    return f, df


def angular(ct, gam, c, d, h):
    """Angular function of the environment sum (reading R1):
    gam [1 + c^2/d^2 - c^2/(d^2 + (h - cos)^2)], minimal at cos = h.
    Returns (value, d value / d cos)."""
    den = d * d + (h - ct) ** 2
    val = gam * (1.0 + c * c / (d * d) - c * c / den)
    dval = -2.0 * gam * c * c * (h - ct) / (den * den)
    return val, dval


def taper(x):
    """Degree-7 taper T(x) = 20x^7 - 70x^6 + 84x^5 - 35x^4 + 1 on [0,1), 0
    beyond (reading R3). Returns (T, dT/dx)."""
    x = np.asarray(x, float)
    inside = x < 1.0
    T = np.where(inside, 1.0 + x ** 4 * (-35.0 + x * (84.0 + x * (-70.0 + 20.0 * x))), 0.0)
    dT = np.where(inside, 140.0 * x ** 3 * (x - 1.0) ** 3, 0.0)
    return T, dT


def coulomb_kernel(r, gam_ij, r_coul, k_e):
    """Shielded, tapered charge-charge kernel K(r) = k_e T(r/Rc) /
    (r^3 + gam_ij^-3)^(1/3) (reading R3). Returns (K, dK/dr)."""
    T, dT = taper(r / r_coul)
    D = np.cbrt(r ** 3 + gam_ij ** -3.0)
    K = k_e * T / D
    dK = k_e * (dT / r_coul / D - T * r * r / D ** 4)
    return K, dK


def bond_order(zeta, g, n, sigma, p):
    """Vectorised bond order, Sec. 2 Eq. 3-5, for any L and p.

    zeta: (..., L) environment sums; g, n: (..., L); sigma, p: (...).
        zhat_l   = g_l + zeta_l^(n_l)                      (Eq. 5)
        zhat_tot = (sum_l zhat_l^-p)^(-1/p)                 (Eq. 4)
        b        = G zhat_tot^(-1/(2 sigma))                (Eq. 3)
    with G fixing b = 1 when every zeta_l = 0. Returns (b, db/dzeta_l (..., L)).
    The derivative of zeta^n at zeta = 0 is taken as 0 (reading: it is only
    ever multiplied by d zeta/dx, which is 0 there).
    """
    zeta = np.asarray(zeta, float)
    sigma = np.asarray(sigma, float)[..., None]
    p = np.asarray(p, float)[..., None]
    pos = zeta > 0.0
    zn = np.where(pos, np.power(np.where(pos, zeta, 1.0), n), 0.0)
    dzn = np.where(pos, n * np.power(np.where(pos, zeta, 1.0), n - 1.0), 0.0)
    zhat = g + zn
    ztot = np.sum(zhat ** (-p), axis=-1) ** (-1.0 / p[..., 0])
    G = np.sum(g ** (-p), axis=-1) ** (-1.0 / (2.0 * sigma[..., 0] * p[..., 0]))
    b = G * ztot ** (-1.0 / (2.0 * sigma[..., 0]))
    # db/dzeta_l = b/(2 sigma) * ztot^p * zhat_l^(-p-1) * n zeta^(n-1) * (-1)
    db = -(b[..., None] / (2.0 * sigma)) * (ztot[..., None] ** p) \
        * zhat ** (-p - 1.0) * dzn
    return b, db


def bond_order_pinf(zeta, g, n, sigma):
    """Eq. 6, the p -> infinity limit: b = max_l G (g_l + zeta_l^n_l)^(-1/(2 sigma))
    with G = (min_l g_l)^(1/(2 sigma))."""
    zeta = np.asarray(zeta, float)
    zhat = g + np.where(zeta > 0, np.power(np.maximum(zeta, 0.0), n), 0.0)
    G = np.min(g, axis=-1) ** (1.0 / (2.0 * np.asarray(sigma)))
    return np.max(G[..., None] * zhat ** (-1.0 / (2.0 * np.asarray(sigma)[..., None])), axis=-1)


def bond_order_tersoff(zeta, n, sigma):
    """Eq. 1: b' = (1 + zeta^n)^(-1/(2 sigma))."""
    return (1.0 + np.power(zeta, n)) ** (-1.0 / (2.0 * sigma))


# ----------------------------------------------------------------------------
# neighbour enumeration over periodic images
# ----------------------------------------------------------------------------
def _image_range(box, pbc, rcut):
    nmax = [int(math.ceil(rcut / box[d])) if pbc[d] else 0 for d in range(3)]
    rng = [np.arange(-m, m + 1) for m in nmax]
    return np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)


def pairs_bruteforce(x, box, pbc, rcut):
    """Every directed pair (i, j, image n) with 0 < |x_j + n*box - x_i| < rcut,
    by testing all N^2 pairs against all images that can reach rcut.
    Self-images (j == i, n != 0) are included. Returns (i, j, n, u) with
    u = x_j + n*box - x_i."""
    x = np.asarray(x, float)
    N = len(x)
    imgs = _image_range(box, pbc, rcut)
    I, J, Nn, U = [], [], [], []
    for img in imgs:
        shift = img * np.where(pbc, box, 0.0)
        u = x[None, :, :] + shift - x[:, None, :]
        r2 = np.einsum("ijk,ijk->ij", u, u)
        ok = (r2 < rcut * rcut) & (r2 > 0.0)
        ii, jj = np.nonzero(ok)
        I.append(ii)
        J.append(jj)
        Nn.append(np.repeat(img[None, :], len(ii), 0))
        U.append(u[ii, jj])
    i = np.concatenate(I)
    j = np.concatenate(J)
    n = np.concatenate(Nn).astype(np.int64)
    u = np.concatenate(U)
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], j, i))
    return i[order], j[order], n[order], u[order]


def pairs_kdtree(x, box, pbc, rcut):
    """Same set as pairs_bruteforce, found with a k-d tree over the atoms and
    their periodic copies that can lie within rcut of the primary cell."""
    from scipy.spatial import cKDTree

    x = np.asarray(x, float)
    N = len(x)
    imgs = _image_range(box, pbc, rcut)
    lo = x.min(0) - rcut
    hi = x.max(0) + rcut
    cx, ci, cn = [], [], []
    for img in imgs:
        shift = img * np.where(pbc, box, 0.0)
        y = x + shift
        keep = np.all((y > lo) & (y < hi), axis=1)
        cx.append(y[keep])
        ci.append(np.nonzero(keep)[0])
        cn.append(np.repeat(img[None, :], int(keep.sum()), 0))
    cx = np.concatenate(cx)
    ci = np.concatenate(ci)
    cn = np.concatenate(cn).astype(np.int64)
    t_all = cKDTree(cx)
    t_own = cKDTree(x)
    sdm = t_own.sparse_distance_matrix(t_all, rcut, output_type="ndarray")
    i = sdm["i"].astype(np.int64)
    k = sdm["j"].astype(np.int64)
    j = ci[k]
    n = cn[k]
    u = cx[k] - x[i]
    r2 = np.einsum("ij,ij->i", u, u)
    ok = (r2 > 0.0) & (r2 < rcut * rcut)
    i, j, n, u = i[ok], j[ok], n[ok], u[ok]
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], j, i))
    return i[order], j[order], n[order], u[order]


def pairs(x, box, pbc, rcut, method="auto"):
    if method == "brute" or (method == "auto" and len(x) <= 600):
        return pairs_bruteforce(x, box, pbc, rcut)
    return pairs_kdtree(x, box, pbc, rcut)


# ----------------------------------------------------------------------------
# the potential
# ----------------------------------------------------------------------------
class System:
    """Geometry-dependent pieces of E(x, q) for one configuration.

    Builds the covalent bonds (r < S of the pair), the triplets, the
    environment sums, the bond orders and the charge-interaction pairs; then
    energy(q), hessian(), gradient terms and forces at any q.
    """

    def __init__(self, x, types, box, pbc, params, method="auto"):
        self.P = P = tables(params) if isinstance(params, dict) else params
        self.x = np.asarray(x, float)
        self.types = t = np.asarray(types, np.int64)
        self.box = np.asarray(box, float)
        self.pbc = np.asarray(pbc, bool)
        self.N = N = len(self.x)

        # ---- covalent bonds: directed (i -> j image) with r < S(ti,tj)
        smax = float(P.S.max())
        bi, bj, bn, bu = pairs(self.x, self.box, self.pbc, smax, method)
        br = np.sqrt(np.einsum("ij,ij->i", bu, bu))
        keep = br < P.S[t[bi], t[bj]]
        self.bi, self.bj, self.bu, self.br = bi[keep], bj[keep], bu[keep], br[keep]
        self.bn = bn[keep]
        ti, tj = t[self.bi], t[self.bj]
        self.fc, self.dfc = cutoff(self.br, P.R[ti, tj], P.S[ti, tj])
        self.fR = P.A[ti, tj] * np.exp(-P.lam1[ti, tj] * self.br)
        self.fA = P.B[ti, tj] * np.exp(-P.lam2[ti, tj] * self.br)
        self.kap = P.kappa[ti, tj]

        # ---- triplets (a = bond i->j, b = bond i->k, same i, b != a)
        nb = len(self.bi)
        start = np.searchsorted(self.bi, np.arange(N + 1))
        cnt = np.diff(start)[self.bi]
        a_idx = np.repeat(np.arange(nb), cnt)
        offs = np.arange(len(a_idx)) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        b_idx = start[self.bi[a_idx]] + offs
        m = a_idx != b_idx
        self.ta, self.tb = a_idx[m], b_idx[m]
        ua, ub = self.bu[self.ta], self.bu[self.tb]
        ra, rb = self.br[self.ta], self.br[self.tb]
        self.ct = np.einsum("ij,ij->i", ua, ub) / (ra * rb)
        tI, tJ, tK = t[self.bi[self.ta]], t[self.bj[self.ta]], t[self.bj[self.tb]]
        L = P.L
        self.zeta = np.zeros((nb, L))
        self._trip = []
        for l in range(L):
            ang, dang = angular(self.ct, P.gam[tI, tJ, tK, l], P.c[tI, tJ, tK, l],
                                P.d[tI, tJ, tK, l], P.h[tI, tJ, tK, l])
            al = P.alpha[tI, tJ, tK, l]
            ex = np.exp(al * (ra - rb))
            fck = self.fc[self.tb]
            tau = fck * ang * ex
            np.add.at(self.zeta[:, l], self.ta, tau)
            self._trip.append((ang, dang, al, ex, tau))
        self.b, self.db = bond_order(self.zeta, P.g[ti, tj], P.n[ti, tj],
                                     P.sigma[ti, tj], P.p[ti, tj])

        # ---- charge-interaction pairs (all images, r < Rc)
        ci, cj, cn, cu = pairs(self.x, self.box, self.pbc, P.r_coul, method)
        self.ci, self.cj, self.cu = ci, cj, cu
        self.cr = np.sqrt(np.einsum("ij,ij->i", cu, cu))
        gij = np.sqrt(P.gam_c[t[ci]] * P.gam_c[t[cj]])
        self.K, self.dK = coulomb_kernel(self.cr, gij, P.r_coul, P.k_e)

        # ---- charge-independent pieces
        self.chi = P.chi[t]
        self.Jt = P.J[t]
        self.E0 = P.E0[t]

    # ---------------- charges
    def bond_weights(self):
        """a_ij = 1/2 kappa f_c f_A b_ij: coefficient of (q_i - q_j)^2 in E_ij."""
        return 0.5 * self.kap * self.fc * self.fA * self.b

    def hessian_dense(self):
        """H = d^2 E / dq^2 (dense, N x N)."""
        N = self.N
        H = np.diag(2.0 * self.Jt)
        aw = self.bond_weights()
        np.add.at(H, (self.bi, self.bi), 2.0 * aw)
        np.add.at(H, (self.bj, self.bj), 2.0 * aw)
        np.add.at(H, (self.bi, self.bj), -2.0 * aw)
        np.add.at(H, (self.bj, self.bi), -2.0 * aw)
        np.add.at(H, (self.ci, self.cj), 0.5 * self.K)
        np.add.at(H, (self.cj, self.ci), 0.5 * self.K)
        return H

    def hessian_sparse(self):
        import scipy.sparse as sp
        N = self.N
        aw = self.bond_weights()
        rows = np.concatenate([np.arange(N), self.bi, self.bj, self.bi, self.bj, self.ci, self.cj])
        cols = np.concatenate([np.arange(N), self.bi, self.bj, self.bj, self.bi, self.cj, self.ci])
        vals = np.concatenate([2.0 * self.Jt, 2 * aw, 2 * aw, -2 * aw, -2 * aw,
                               0.5 * self.K, 0.5 * self.K])
        return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))

    def solve_charges(self, Q=0.0, method="auto", tol=1e-13, q0=None):
        """Minimise E over q subject to sum q = Q (Sec. 2: charges minimise
        E_tot). E is quadratic in q, so the minimiser solves the KKT system
        [H, -1; 1^T, 0][q; mu] = [-chi; Q]. Dense solve for N <= 4000,
        otherwise two CG solves H s = -chi, H t = 1 (scipy CG) and
        q = s + mu t with mu fixing the total charge."""
        N = self.N
        if method == "dense" or (method == "auto" and N <= 4000):
            H = self.hessian_dense()
            KKT = np.zeros((N + 1, N + 1))
            KKT[:N, :N] = H
            KKT[:N, N] = -1.0
            KKT[N, :N] = 1.0
            rhs = np.concatenate([-self.chi, [Q]])
            sol = np.linalg.solve(KKT, rhs)
            return sol[:N], float(sol[N])
        from scipy.sparse.linalg import cg
        H = self.hessian_sparse()
        d = H.diagonal()
        import scipy.sparse.linalg as spl
        M = spl.LinearOperator((N, N), matvec=lambda v: v / d)
        s, i1 = cg(H, -self.chi, rtol=tol, atol=0.0, M=M, maxiter=5000)
        tt, i2 = cg(H, np.ones(N), rtol=tol, atol=0.0, M=M, maxiter=5000)
        if i1 or i2:
            raise RuntimeError("oracle CG did not converge")
        mu = (Q - s.sum()) / tt.sum()
        return s + mu * tt, float(mu)

    # ---------------- energy
    def energy(self, q, per_atom=False):
        """E(x, q) of the model card (pair + bond order + self + charge terms)."""
        q = np.asarray(q, float)
        t = self.types
        dq = q[self.bi] - q[self.bj]
        cq = 1.0 - self.kap * dq * dq
        e_bond = 0.5 * self.fc * (self.fR - cq * self.b * self.fA)
        e_self = self.E0 + self.chi * q + self.Jt * q * q
        e_pair = 0.5 * q[self.ci] * q[self.cj] * self.K
        if not per_atom:
            return float(e_bond.sum() + e_self.sum() + e_pair.sum())
        ea = e_self.copy()
        np.add.at(ea, self.bi, e_bond)
        np.add.at(ea, self.ci, e_pair)
        return ea

    def dE_dq(self, q):
        q = np.asarray(q, float)
        g = self.chi + 2.0 * self.Jt * q
        aw = self.bond_weights()
        dq = q[self.bi] - q[self.bj]
        np.add.at(g, self.bi, 2.0 * aw * dq)
        np.add.at(g, self.bj, -2.0 * aw * dq)
        np.add.at(g, self.ci, 0.5 * self.K * q[self.cj])
        np.add.at(g, self.cj, 0.5 * self.K * q[self.ci])
        return g

    # ---------------- gradients at fixed q
    def gradients(self, q):
        """dE/du for every covalent bond vector and every charge-pair vector,
        at fixed charges. Returns (g_bond (nb,3), g_pair (np,3))."""
        P = self.P
        q = np.asarray(q, float)
        t = self.types
        ti, tj = t[self.bi], t[self.bj]
        dq = q[self.bi] - q[self.bj]
        cq = 1.0 - self.kap * dq * dq
        uhat = self.bu / self.br[:, None]
        # pair part, b held fixed
        dE_dr = 0.5 * (self.dfc * (self.fR - cq * self.b * self.fA)
                       + self.fc * (-P.lam1[ti, tj] * self.fR
                                    + cq * self.b * P.lam2[ti, tj] * self.fA))
        gb = dE_dr[:, None] * uhat
        # bond-order part: D_l = dE_ij/dzeta_l
        D = -0.5 * (cq * self.fc * self.fA)[:, None] * self.db
        ua, ub = uhat[self.ta], uhat[self.tb]
        ra, rb = self.br[self.ta], self.br[self.tb]
        ct = self.ct[:, None]
        fck, dfck = self.fc[self.tb], self.dfc[self.tb]
        for l, (ang, dang, al, ex, tau) in enumerate(self._trip):
            Dl = D[self.ta, l]
            # d tau / d u_a and d tau / d u_b
            dcos_a = (ub - ct * ua) / ra[:, None]
            dcos_b = (ua - ct * ub) / rb[:, None]
            w_cos = (fck * dang * ex)[:, None]
            g_a = (al * tau)[:, None] * ua + w_cos * dcos_a
            g_b = (dfck * ang * ex - al * tau)[:, None] * ub + w_cos * dcos_b
            np.add.at(gb, self.ta, Dl[:, None] * g_a)
            np.add.at(gb, self.tb, Dl[:, None] * g_b)
        # charge pairs
        chat = self.cu / self.cr[:, None]
        gp = (0.5 * q[self.ci] * q[self.cj] * self.dK)[:, None] * chat
        return gb, gp

    def forces(self, q):
        gb, gp = self.gradients(q)
        F = np.zeros((self.N, 3))
        # E depends on u = x_j - x_i: dE/dx_j += g, dE/dx_i -= g
        np.add.at(F, self.bj, -gb)
        np.add.at(F, self.bi, gb)
        np.add.at(F, self.cj, -gp)
        np.add.at(F, self.ci, gp)
        return F

    def virial(self, q):
        """W = -sum_u u (x) dE/du (3x3)."""
        gb, gp = self.gradients(q)
        return -(np.einsum("ia,ib->ab", self.bu, gb) + np.einsum("ia,ib->ab", self.cu, gp))


def evaluate(x, types, box, pbc, params, Q=0.0, q=None, charge_method="auto",
             method="auto"):
    """One energy/force/charge evaluation: charges minimised (unless q is
    given), then energy, forces, virial and per-atom energies at those
    charges."""
    s = System(x, types, box, pbc, params, method=method)
    mu = None
    if q is None:
        q, mu = s.solve_charges(Q, method=charge_method)
    q = np.asarray(q, float)
    return {
        "E": s.energy(q),
        "F": s.forces(q),
        "q": q,
        "mu": mu,
        "virial": s.virial(q),
        "e_atom": s.energy(q, per_atom=True),
        "zeta": s.zeta,
        "b": s.b,
        "system": s,
    }


def kinetic_energy(v, types, params, frozen=None):
    m = np.asarray(params["mass"] if isinstance(params, dict) else params.mass)[types]
    ke = 0.5 * np.sum(m[:, None] * v * v) / ACC
    return float(ke)


def velocity_verlet(x, v, types, box, pbc, params, dt, nsteps, frozen=None,
                    Q=0.0, record=None):
    """NVE velocity Verlet (dt in fs), charges re-minimised every step (Sec. 2:
    the charge is minimised in every timestep). Frozen atoms keep v = 0 and
    never move; their forces are still computed. Returns final (x, v, q) and
    a list of total energies E_pot + KE after each step."""
    P = tables(params)
    x = np.array(x, float)
    v = np.array(v, float)
    types = np.asarray(types)
    frozen = np.zeros(len(x), bool) if frozen is None else np.asarray(frozen, bool)
    inv_m = (ACC / P.mass[types])[:, None]
    mob = (~frozen)[:, None]
    res = evaluate(x, types, box, pbc, params, Q)
    F = res["F"]
    etot = []
    for _ in range(nsteps):
        v = np.where(mob, v + 0.5 * dt * F * inv_m, 0.0)
        x = np.where(mob, x + dt * v, x)
        res = evaluate(x, types, box, pbc, params, Q)
        F = res["F"]
        v = np.where(mob, v + 0.5 * dt * F * inv_m, 0.0)
        etot.append(res["E"] + kinetic_energy(v, types, params))
    return x, v, res["q"], np.array(etot)


def thermostat_dof(types, frozen=None):
    """Degrees of freedom a thermostat controls: 3 per mobile atom, less the 3
    of the centre-of-mass motion when no atom is frozen (then the total
    momentum is conserved)."""
    n = len(types)
    fr = np.zeros(n, bool) if frozen is None else np.asarray(frozen, bool)
    g = 3 * int((~fr).sum())
    return g - 3 if not fr.any() else g


def nose_hoover(x, v, types, box, pbc, params, dt, nsteps, T0, tau, frozen=None, Q=0.0, xi=0.0, eta=0.0):
    """NVT velocity Verlet with one Nose-Hoover thermostat (reading of the
    paper's "NVT ensemble", Sec. 3.3, which names no thermostat).
    Equations of motion: dx/dt = v, dv/dt = F/m - xi v, dxi/dt = (2K - g kB T0)/Qm,
    deta/dt = xi, with thermostat mass Qm = g kB T0 tau^2; the extended energy
    E + K + Qm xi^2 / 2 + g kB T0 eta is conserved. One step is the symmetric
    splitting: xi and eta half-steps, velocity scaling by exp(-xi dt/2), the
    velocity-Verlet kick/drift/force/kick, velocity scaling, eta and xi
    half-steps. Frozen atoms keep v = 0 and count in neither K nor g.
    Returns (x, v, q, xi, eta, extended energies after each step)."""
    P = tables(params)
    x = np.array(x, float)
    v = np.array(v, float)
    types = np.asarray(types)
    frozen = np.zeros(len(x), bool) if frozen is None else np.asarray(frozen, bool)
    inv_m = (ACC / P.mass[types])[:, None]
    mob = (~frozen)[:, None]
    g = thermostat_dof(types, frozen)
    gkT = g * KB * T0
    Qm = gkT * tau * tau
    res = evaluate(x, types, box, pbc, params, Q)
    F = res["F"]
    ext = []
    for _ in range(nsteps):
        K = kinetic_energy(v, types, params)
        xi = xi + 0.5 * dt * (2.0 * K - gkT) / Qm
        eta = eta + 0.5 * dt * xi
        v = np.where(mob, v * np.exp(-0.5 * dt * xi), 0.0)
        v = np.where(mob, v + 0.5 * dt * F * inv_m, 0.0)
        x = np.where(mob, x + dt * v, x)
        res = evaluate(x, types, box, pbc, params, Q)
        F = res["F"]
        v = np.where(mob, v + 0.5 * dt * F * inv_m, 0.0)
        v = np.where(mob, v * np.exp(-0.5 * dt * xi), 0.0)
        eta = eta + 0.5 * dt * xi
        K = kinetic_energy(v, types, params)
        xi = xi + 0.5 * dt * (2.0 * K - gkT) / Qm
        ext.append(res["E"] + K + 0.5 * Qm * xi * xi + gkT * eta)
    return x, v, res["q"], xi, eta, np.array(ext)


# ----------------------------------------------------------------------------
# force-matching loss and its parameter gradient (the definition, by central
# differences; the paper fits its parameters to DFT energies, forces and
# charges, Sec. 2, without printing a method)
# ----------------------------------------------------------------------------
def param_leaves(params):
    """Every scalar of a parameter dictionary the energy depends on, as
    (path, value): pair, bond, triplet, self and charge-kernel entries (the
    masses and labels are not parameters of E)."""
    out = []
    for sec in ("pair", "bond", "triplet"):
        for key in sorted(params[sec]):
            for f in sorted(params[sec][key]):
                v = params[sec][key][f]
                if isinstance(v, (list, tuple)):
                    out += [((sec, key, f, l), float(x)) for l, x in enumerate(v)]
                else:
                    out.append(((sec, key, f), float(v)))
    for f in ("E0", "chi", "J"):
        out += [(("self", f, t), float(x)) for t, x in enumerate(params["self"][f])]
    out += [(("coulomb", "gamma", t), float(x)) for t, x in enumerate(params["coulomb"]["gamma"])]
    out += [(("coulomb", "r_coul"), float(params["coulomb"]["r_coul"])),
            (("coulomb", "k_e"), float(params["coulomb"]["k_e"]))]
    return out


def with_leaf(params, path, value):
    """A deep copy of params with the scalar at path set to value."""
    import copy
    p = copy.deepcopy(params)
    node = p
    for k in path[:-1]:
        node = node[k]
    node[path[-1]] = value
    return p


def force_matching_loss(structs, params, w_E=None, E_ref=None, w_F=None, F_ref=None):
    """loss = sum_r w_E[r] (E_r - E_ref[r])^2 + sum_r w_F[r] sum_i |F_i - F_ref_i|^2
    with every structure's charges at their minimiser (total charge 0)."""
    loss = 0.0
    off = 0
    for r, s in enumerate(structs):
        o = evaluate(s.x, s.types, s.box, s.pbc, params)
        if w_E is not None:
            loss += w_E[r] * (o["E"] - E_ref[r]) ** 2
        if w_F is not None:
            d = o["F"] - F_ref[off:off + s.n]
            loss += w_F[r] * float(np.sum(d * d))
        off += s.n
    return loss


def loss_grad_fd(structs, params, w_E=None, E_ref=None, w_F=None, F_ref=None, paths=None, h=1e-4):
    """d loss / d theta for every leaf (or the given paths) by central
    differences with step h * max(|theta|, 1), Richardson-extrapolated from
    that step and half of it (error O(h^4)): the loss is quadratic in E and
    F, whose derivatives reach hundreds of eV per unit of some parameters,
    so a single central difference at h = 1e-4 keeps ~1e-4 relative error."""
    leaves = dict(param_leaves(params))
    out = {}

    def central(path, v, step):
        lp = force_matching_loss(structs, with_leaf(params, path, v + step), w_E, E_ref, w_F, F_ref)
        lm = force_matching_loss(structs, with_leaf(params, path, v - step), w_E, E_ref, w_F, F_ref)
        return (lp - lm) / (2.0 * step)

    for path in (paths if paths is not None else list(leaves)):
        v = leaves[path]
        step = h * max(abs(v), 1.0)
        d1, d2 = central(path, v, step), central(path, v, 0.5 * step)
        out[path] = (4.0 * d2 - d1) / 3.0
    return out


# ----------------------------------------------------------------------------
# Si desorption screening (Sec. 3.3)
# ----------------------------------------------------------------------------
def coordination(x, types, box, pbc, params):
    """Covalent coordination of every atom: neighbours (every periodic image)
    closer than the cutoff S of the pair, i.e. with f_c > 0."""
    s = System(x, types, box, pbc, params)
    return np.bincount(s.bi, minlength=s.N)


def removal_energy(x, types, box, pbc, params, i, Q=0.0, E_full=None):
    """Energy change when atom i is eliminated (Sec. 3.3 screens surface Si
    atoms by it every 1 ps and removes those below a threshold, 6.5 eV):

        dE_i = E(system without i) + E0_{t_i} - E(system),

    every other atom held in place and both energies at their charge
    minimiser with total charge Q. Reading (the paper defines the change but
    not its reference state): the atom leaves as an isolated neutral atom,
    whose energy is its self-energy constant E0 (U at q = 0), so the rest
    keeps the total charge. E_full may pass E(system) when already known."""
    x = np.asarray(x, float)
    types = np.asarray(types)
    keep = np.ones(len(x), bool)
    keep[i] = False
    P = tables(params) if isinstance(params, dict) else params
    if E_full is None:
        E_full = evaluate(x, types, box, pbc, params, Q=Q)["E"]
    if keep.sum() == 0:
        E_rest = 0.0
    else:
        E_rest = evaluate(x[keep], types[keep], box, pbc, params, Q=Q)["E"]
    return E_rest + float(P.E0[int(types[i])]) - E_full


def desorption_screen(x, types, box, pbc, params, candidates, threshold=6.5, Q=0.0):
    """Removal energies of the candidate atoms, each taken alone from the
    same configuration, and the candidates whose energy is below the
    threshold (the ones the screening removes together)."""
    E_full = evaluate(x, types, box, pbc, params, Q=Q)["E"]
    dE = np.array([removal_energy(x, types, box, pbc, params, int(i), Q=Q, E_full=E_full) for i in candidates])
    return dE, np.asarray(candidates)[dE < threshold]


# ----------------------------------------------------------------------------
# Energy minimisation ("relaxed", "energy minimization", Sec. 3)
# ----------------------------------------------------------------------------
# FIRE constants as published by Bitzek et al., Phys. Rev. Lett. 97, 170201
# (2006): N_min, f_inc, f_dec, alpha_start, f_alpha.
FIRE_NMIN, FIRE_FINC, FIRE_FDEC, FIRE_ALPHA0, FIRE_FALPHA = 5, 1.1, 0.5, 0.1, 0.99


def fire_minimize(x, types, box, pbc, params, frozen=None, fmax=1e-3, max_iter=1000, dt0=1.0, dt_max=5.0,
                  Q=0.0, n_iter=None):
    """Relax positions to a local minimum of E(x) = min_q E(x, q) (the paper
    relaxes structures but names no method; reading: FIRE, Bitzek et al.
    2006, with the semi-implicit Euler step). One iteration, with F the
    forces at the current positions (charges at their minimiser) and v the
    velocities (zero at the start), over the mobile atoms:
      * stop when max_i |F_i| < fmax;
      * P = F . v. Downhill (P >= 0, so a start from rest counts): n+ += 1;
        once n+ > N_min, dt = min(f_inc dt, dt_max) and alpha *= f_alpha;
        then v = (1 - alpha) v + alpha |v| F / |F|. Uphill (P < 0): n+ = 0,
        dt *= f_dec, alpha = alpha_start, v = 0;
      * v += dt F / m; x += dt v.
    Frozen atoms never move. n_iter, if given, stops after that many
    iterations whatever the forces. Returns (x, iterations taken, the
    energies at every evaluation, converged)."""
    P = tables(params)
    x = np.array(x, float)
    types = np.asarray(types)
    frozen = np.zeros(len(x), bool) if frozen is None else np.asarray(frozen, bool)
    mob = (~frozen)[:, None]
    inv_m = (ACC / P.mass[types])[:, None]
    v = np.zeros_like(x)
    dt, alpha, npos = dt0, FIRE_ALPHA0, 0
    res = evaluate(x, types, box, pbc, params, Q)
    energies = [res["E"]]
    it = 0
    limit = max_iter if n_iter is None else n_iter
    while True:
        F = np.where(mob, res["F"], 0.0)
        fm = float(np.sqrt(np.max(np.sum(F * F, axis=1)))) if len(F) else 0.0
        if (n_iter is None and fm < fmax) or it >= limit:
            return x, it, np.array(energies), fm < fmax
        Pw = float(np.sum(F * v))
        if Pw >= 0.0:
            npos += 1
            if npos > FIRE_NMIN:
                dt = min(dt * FIRE_FINC, dt_max)
                alpha *= FIRE_FALPHA
            vn, fn = math.sqrt(float(np.sum(v * v))), math.sqrt(float(np.sum(F * F)))
            v = (1.0 - alpha) * v + (alpha * vn / fn if fn > 0 else 0.0) * F
        else:
            npos = 0
            dt *= FIRE_FDEC
            alpha = FIRE_ALPHA0
            v = np.zeros_like(v)
        v = np.where(mob, v + dt * F * inv_m, 0.0)
        x = np.where(mob, x + dt * v, x)
        it += 1
        res = evaluate(x, types, box, pbc, params, Q)
        energies.append(res["E"])


# ----------------------------------------------------------------------------
# Ring statistics of the C network (Sec. 3.3: counts of 5-, 6- and 7-membered
# rings over time, and the in-plane orientation of 6-membered rings)
# ----------------------------------------------------------------------------
def carbon_bonds(x, types, box, pbc, bond_cut):
    """C-C bonds (every periodic image) shorter than bond_cut: for each C
    atom, the list of (neighbour, bond vector)."""
    x = np.asarray(x, float)
    types = np.asarray(types)
    i, j, _, u = pairs(x, np.asarray(box, float), np.asarray(pbc, bool), bond_cut)
    r = np.sqrt(np.einsum("ij,ij->i", u, u))
    nb = [[] for _ in range(len(x))]
    for a, b, v, rr in zip(i, j, u, r):
        if types[a] == 1 and types[b] == 1 and rr < bond_cut:
            nb[a].append((int(b), v))
    return nb


def rings(x, types, box, pbc, bond_cut, max_size=8, close_tol=0.1):
    """Primitive rings of the C bond graph, sizes 3..max_size (a reading of
    the paper's "n-membered rings"; it gives no ring criterion). A ring is a
    closed path of distinct atoms whose bond vectors sum to zero (so a path
    around a periodic box does not count), and is primitive when no two of
    its atoms are joined in the graph by a path shorter than their distance
    along the ring (with the same displacement). Each ring once: starting at
    its lowest atom index, second atom below the last. Returns a list of
    (size, centre (3,), orientation in degrees or nan): the orientation of a
    6-ring is the in-plane angle of its three vertex diagonals taken modulo
    60 degrees (their circular mean in that period), zero when a diagonal
    points along x."""
    x = np.asarray(x, float)
    nb = carbon_bonds(x, types, box, pbc, bond_cut)
    out = []

    def has_shortcut(a, b, disp, k):
        # a walk of length < k from a reaching b with displacement disp
        frontier = [(a, np.zeros(3))]
        for _ in range(k - 1):
            nxt = []
            for v, d in frontier:
                for w, bv in nb[v]:
                    dw = d + bv
                    if w == b and np.linalg.norm(dw - disp) < close_tol:
                        return True
                    nxt.append((w, dw))
            frontier = nxt
        return False

    def primitive(path, pos):
        n = len(path)
        for s in range(n):
            for t in range(s + 2, n):
                k = min(t - s, n - (t - s))
                if k >= 2 and has_shortcut(path[s], path[t], pos[t] - pos[s], k):
                    return False
        return True

    def orientation(pos):
        psi = []
        for k in range(3):
            d = pos[k + 3] - pos[k]
            psi.append(6.0 * math.atan2(d[1], d[0]))
        m = math.atan2(sum(math.sin(p) for p in psi), sum(math.cos(p) for p in psi)) / 6.0
        return math.degrees(m) % 60.0

    def dfs(path, pos):
        v, d = path[-1], pos[-1]
        for w, bv in nb[v]:
            dw = d + bv
            if w == path[0] and len(path) >= 3:
                if np.linalg.norm(dw) < close_tol and path[1] < path[-1] and primitive(path, pos):
                    P = np.array(pos)
                    c = x[path[0]] + P.mean(axis=0)
                    out.append((len(path), c, orientation(P) if len(path) == 6 else float("nan")))
                continue
            if w <= path[0] or w in path or len(path) >= max_size:
                continue
            dfs(path + [w], pos + [dw])

    for a in range(len(x)):
        if nb[a]:
            dfs([a], [np.zeros(3)])
    return out


def ring_counts(ring_list, max_size=8):
    """Number of rings of each size 3..max_size."""
    c = np.zeros(max_size - 2, dtype=np.int64)
    for n, _, _ in ring_list:
        c[n - 3] += 1
    return c
