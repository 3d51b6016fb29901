/*
 * ctbop.h — C ABI of libctbop: one MD step of the charge-transfer
 * bond-order Si/C potential of Takamoto et al. (arXiv:1802.07871) on one GPU.
 *
 * What a step computes (paper references are sections and equations of the
 * paper; "reading" marks choices the paper leaves open, documented with the
 * library):
 *   - environment sums zeta_1, zeta_2 of every directed bond (Sec. 2, Eq. 2)
 *     and the vectorised bond order b_ij (Eq. 7, L = 2, p = 2);
 *   - Tersoff-type pair energies with the covalent-ionic factor
 *     1 - kappa (q_i - q_j)^2 on the attractive term (reading of f_q, Sec. 2);
 *   - self energy E0 + chi q + J q^2 (Sec. 2 adds the constant E0) and a
 *     shielded, tapered charge interaction over all periodic images;
 *   - charges minimising the total energy at every step (Sec. 2), solved by
 *     preconditioned conjugate gradients on the device;
 *   - forces -dE/dx at the minimising charges, virial, per-atom energies;
 *   - NVE velocity Verlet with frozen atoms (Sec. 3.3 fixes the substrate
 *     bottom).
 *
 * Conventions
 *   Units: Angstrom, fs, u, eV, e. Atom types: 0 = Si, 1 = C.
 *   Every function returns CTBOP_OK (0) or a negative CTBOP_ERR_* code;
 *   ctbop_last_error() gives a message for the last failure of that system.
 *   A system handle is used from one host thread at a time (not reentrant).
 *   Array arguments are plain pointers. `mem` says where a pointer lives:
 *   CTBOP_HOST (pageable or pinned host memory) or CTBOP_DEVICE (device
 *   memory of the system's GPU). Inputs are copied in; the caller keeps
 *   ownership of every buffer it passes. The library owns its device memory.
 *   Device-pointer transfers and compute/step calls are ordered on the
 *   system's stream; host-pointer transfers and ctbop_status synchronise it.
 *   Atoms are laid out replica by replica: atom_offsets[r]..atom_offsets[r+1]-1
 *   belong to replica r; atoms of different replicas never interact.
 */
#ifndef CTBOP_H
#define CTBOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CTBOP_OK                    0
#define CTBOP_ERR_INVALID_ARG      -1   /* null pointer, size mismatch, bad type or box */
#define CTBOP_ERR_OOM              -2   /* device allocation failed */
#define CTBOP_ERR_NEIGH_OVERFLOW   -3   /* neighbour capacity exceeded and could not grow */
#define CTBOP_ERR_CG_NOT_CONVERGED -4   /* charge solve hit max_iter; results still written */
#define CTBOP_ERR_NONFINITE        -5   /* non-finite energy, force or position */
#define CTBOP_ERR_CUDA             -6   /* a CUDA runtime call failed */
#define CTBOP_ERR_STATE            -7   /* call out of order (e.g. compute before positions) */

/* ---- memory location of a pointer argument ----------------------------- */
#define CTBOP_HOST   0
#define CTBOP_DEVICE 1

/* ---- precision policy --------------------------------------------------- */
/* FP64: every quantity in double precision.
 * MIXED: bond-order, cutoff, three-body, charge-kernel arithmetic and the
 * CG matrix-vector products in float; positions as float offsets from the
 * owning cell's origin (exact FP64 master copy kept); per-atom energies,
 * virial, CG vectors, dot products and residual norms in double. */
#define CTBOP_PREC_FP64  0
#define CTBOP_PREC_MIXED 1

/* ---- compute flags ------------------------------------------------------ */
#define CTBOP_FIXED_CHARGES 1u   /* use the charges last set; skip the solve */

/* ---- ctbop_get selectors (dst layouts) ---------------------------------- */
#define CTBOP_GET_ENERGY    0   /* double[R]   total potential energy per replica (eV) */
#define CTBOP_GET_FORCES    1   /* double[N*3] forces (eV/A) */
#define CTBOP_GET_CHARGES   2   /* double[N]   charges (e) */
#define CTBOP_GET_POSITIONS 3   /* double[N*3] positions (A); wrapped into the box along periodic axes at list rebuilds */
#define CTBOP_GET_VELOCITIES 4  /* double[N*3] velocities (A/fs) */
#define CTBOP_GET_VIRIAL    5   /* double[R*9] virial W = -sum_u u (x) dE/du, row-major 3x3 (eV); MD steps
                                   leave it out of their force pass, so the first read after ctbop_step
                                   recomputes it from the current state (one covalent-force and charge-force
                                   pass, no kick) */
#define CTBOP_GET_E_ATOM    6   /* double[N]   per-atom energies (eV) */
#define CTBOP_GET_MU        7   /* double[R]   electronegativity (Lagrange multiplier of sum q = Q), eV/e */
#define CTBOP_GET_KINETIC   8   /* double[R]   kinetic energy of the current velocities (eV) */
#define CTBOP_GET_THERMOSTAT 9  /* double[R*4] Nose-Hoover state per replica: xi (1/fs), eta (fs), thermostat
                                   mass Qm (eV fs^2), g kB T0 (eV); zeros when the replica has none */
#define CTBOP_GET_COORDINATION 10 /* double[N] covalent coordination: neighbours (every periodic image) closer
                                   than the cutoff S of the pair, f_c > 0; needs a completed compute or step
                                   (CTBOP_ERR_STATE otherwise) */

/* ---- parameters --------------------------------------------------------- */
/* Index conventions: pair tables [ti*2+tj] (symmetric for the pair block),
 * ordered pair [ti*2+tj] for the bond-order block, ordered triplet
 * [(ti*2+tj)*2+tk] (i centre, j bond partner, k third atom), then l = 0,1. */
typedef struct ctbop_params {
    /* pair: E_ij = 1/2 fc(r)[A e^{-lambda1 r} - c_ij b_ij B e^{-lambda2 r}],
     * fc from R to S; c_ij = 1 - kappa (q_i - q_j)^2 */
    double A[4], B[4], lambda1[4], lambda2[4], R[4], S[4], kappa[4];
    /* bond order (Eq. 7): b = G[(g1+z1^n1)^-p + (g2+z2^n2)^-p]^(1/(2 sigma p)) */
    double sigma[4], p[4], g[4][2], n[4][2];
    /* environment sums (Eq. 2): zeta_l = sum_k fc(r_ik) ang_l(cos) e^{alpha_l (r_ij - r_ik)},
     * ang_l(c) = gamma_l [1 + c_l^2/d_l^2 - c_l^2/(d_l^2 + (h_l - c)^2)] */
    double gamma[8][2], c[8][2], d[8][2], h[8][2], alpha[8][2];
    /* per type: self energy E0 + chi q + J q^2, charge shielding gamma_c, mass (u) */
    double E0[2], chi[2], J[2], gamma_c[2], mass[2];
    /* charge kernel k_e T(r/r_coul) / (r^3 + (gamma_ci gamma_cj)^(-3/2))^(1/3) */
    double r_coul, k_e;
} ctbop_params;

/* Preconditioners of the charge CG (ctbop_options.precond). BLOCK: the
 * exact inverse of each 32 x 32 diagonal block of H (atoms 32b .. 32b+31 in
 * the order they were given; atoms listed in spatially coherent order make
 * the blocks compact and the preconditioner strong). JACOBI: 1 / diag(H). */
#define CTBOP_PRECOND_BLOCK 0
#define CTBOP_PRECOND_JACOBI 1

typedef struct ctbop_options {
    int32_t precision;    /* CTBOP_PREC_FP64 or CTBOP_PREC_MIXED */
    int32_t cg_max_iter;  /* charge-solve iteration cap (default 200) */
    double  cg_tol;       /* stop when max_i |H q + chi - mu|_i over a replica (the max-norm of
                           the stationarity residual) is below cg_tol (eV/e); 0 = policy default
                           (FP64 1e-11, MIXED 1e-5) */
    double  skin;         /* neighbour-list skin (A, default 0.3) */
    int32_t cap_cov;      /* covalent entries per atom; 0 = sized from the first configuration */
    int32_t cap_all;      /* all entries (charge cutoff) per atom; 0 = sized automatically */
    int32_t device;       /* CUDA device ordinal */
    int32_t precond;      /* charge-solve preconditioner: CTBOP_PRECOND_BLOCK (default) or CTBOP_PRECOND_JACOBI */
} ctbop_options;

/* Counters, and the shapes the autotuners keep. The tuners time every
 * candidate on the live lists after each list allocation and keep the
 * fastest; environment
 * variables force a choice instead: CTBOP_MV_BATCH (4, 8, 16: matrix-pass
 * depth), CTBOP_GATHER_BATCH (4, 6, 8), CTBOP_COV_LANES (4, 8, 16),
 * CTBOP_BUILD_SHAPE ("warps,batch"). CTBOP_NO_GRAPH=1 runs steps as direct
 * launches with a host-polled charge loop instead of CUDA graphs. */
typedef struct ctbop_stats {
    int64_t steps;            /* MD steps taken */
    int64_t rebuilds;         /* neighbour-list rebuilds */
    int32_t cg_iters_last;    /* CG iterations of the last charge solve */
    int32_t max_cov;          /* largest covalent entry count at the last rebuild */
    int64_t cg_iters_total;   /* summed over all solves */
    int64_t solves;           /* number of charge solves */
    double  cg_residual_last; /* max_i |H q + chi - mu|_i after the last solve, replica 0 (eV/e) */
    int32_t max_all;          /* largest total entry count at the last rebuild */
    uint32_t error_bits;      /* device-side error bits seen (see ctbop_last_error) */
    double  mean_cov;         /* mean covalent entries (incl. skin) at the last rebuild */
    double  mean_all;         /* mean total entries at the last rebuild */
    double  cg_residual_start; /* max_i |H q0 + chi - mu|_i of the last solve's starting guess, replica 0 (eV/e) */
    int32_t cg_mv_batch;      /* list entries in flight per thread in the CG matrix pass (autotuned) */
    int32_t asm_batch;        /* list entries in flight per thread in the matrix assembly (autotuned) */
    double  cg_mv_ms[3];      /* ms per matrix pass of the depths 4, 8, 16 at the last tuning (0: not timed) */
    double  mean_mat;         /* mean stored charge-matrix entries per atom (the entries a matrix pass
                                 streams: those inside the charge cutoff under the mixed policy) */
    double  asm_ms[3];        /* ms per assembly of the depths 4, 8, 16 at the last tuning (0: not timed) */
    int32_t gather_batch;     /* list entries in flight per thread in the charge-force gather (autotuned) */
    int32_t fp64_atoms;       /* MIXED: atoms whose covalent terms the last evaluation redid in FP64 (see
                                 ctbop_compute) */
    int32_t fp64_bonds;       /* MIXED: bonds whose pair term the last evaluation took in FP64 */
    int32_t pad;
    double  gather_ms[3];     /* ms per charge-force gather of the depths 4, 6, 8 at the last tuning */
    int32_t cov_lanes;        /* lanes per atom in the bond-order and covalent-force passes (autotuned) */
    int32_t pad2;
    double  cov_ms[3];        /* ms of bond-order + covalent-force pass at 4, 8, 16 lanes at the last tuning */
    int32_t build_warps;      /* list build: warps per block (autotuned) */
    int32_t build_batch;      /* list build: stencil cells per batch (autotuned) */
    double  build_ms[6];      /* ms per list build of the shapes (2,64) (2,128) (4,64) (4,128) (8,64) (8,128) */
} ctbop_stats;

typedef struct ctbop_system ctbop_system;

/* Fill *o with defaults (MIXED precision, skin 0.3 A, 200 iterations). */
int ctbop_default_options(ctbop_options* o);

/* Create a system on o->device. p and o are copied. *out receives the handle.
 * Fails with INVALID_ARG on null pointers, non-positive masses or cutoffs,
 * R >= S, or a charge cutoff below the largest covalent cutoff. */
int ctbop_create(const ctbop_params* p, const ctbop_options* o, ctbop_system** out);

/* Free the system and all of its device memory. Null is accepted. */
int ctbop_destroy(ctbop_system* s);

/* Message for the last error on s (empty string if none; never null). */
const char* ctbop_last_error(const ctbop_system* s);

/* Order all later work on `cuda_stream` (a cudaStream_t; null = the
 * library's own stream, which synchronises with the legacy stream). Work
 * already enqueued on the previous stream is waited for first. Every
 * transfer the library makes, host copies included, is ordered on this
 * stream, so a non-blocking stream is safe. */
int ctbop_set_stream(ctbop_system* s, void* cuda_stream);

/* Replica layout: n_replicas >= 1, atom_offsets host int64[n_replicas+1],
 * atom_offsets[0] = 0, non-decreasing; N = atom_offsets[n_replicas].
 * Resets all per-atom state. */
int ctbop_set_layout(ctbop_system* s, int32_t n_replicas, const int64_t* atom_offsets);

/* Boxes: h host double[R*9], row-major 3x3 cell matrix per replica whose
 * rows are the cell vectors; only orthorhombic (diagonal) cells are accepted.
 * pbc host uint8[R*3], 1 = periodic axis. Along open axes the diagonal entry
 * is the extent used for binning; atoms outside [0, L) are still handled. */
int ctbop_set_box(ctbop_system* s, const double* h, const uint8_t* pbc);

/* Per-atom inputs, N entries (x and v: N*3, row-major). types: 0 or 1. */
int ctbop_set_types(ctbop_system* s, const int32_t* types, int mem);
int ctbop_set_positions(ctbop_system* s, const double* x, int mem);
int ctbop_set_velocities(ctbop_system* s, const double* v, int mem);
/* Charges: warm start for the solve, or the fixed charges for CTBOP_FIXED_CHARGES. */
int ctbop_set_charges(ctbop_system* s, const double* q, int mem);
/* frozen: uint8[N], 1 = atom never moves (its force is still computed). */
int ctbop_set_frozen(ctbop_system* s, const uint8_t* frozen, int mem);
/* Total charge per replica, host double[R] (default 0: neutral). */
int ctbop_set_total_charge(ctbop_system* s, const double* Q);

/* One evaluation: neighbour lists (rebuilt when needed), bond orders,
 * charges (unless CTBOP_FIXED_CHARGES), energy, forces, virial, per-atom
 * energies. Stream-ordered; returns before the GPU finishes. Errors found on
 * the device are reported by the next synchronising call. */
int ctbop_compute(ctbop_system* s, uint32_t flags);

/* n_steps velocity-Verlet steps of dt_fs each, charges re-minimised every
 * step. Runs as a CUDA graph replay per step; synchronises at the end to
 * check device status (neighbour overflow is repaired by growing the lists
 * and redoing the affected steps). */
int ctbop_step(ctbop_system* s, int64_t n_steps, double dt_fs);

/* Storage order of the atoms (optional; call after ctbop_set_layout and
 * before any per-atom setter). order[k] (host, N entries) is the caller's
 * index of the atom the library stores in slot k; it must permute the atoms
 * within each replica. Every later per-atom input and output (set_types,
 * set_positions, set_velocities, set_charges, set_frozen, per-atom
 * ctbop_get selectors, param_grad's F_ref, removal_energies' candidates)
 * stays in the caller's order; the library permutes on the device. A
 * spatially coherent storage order (e.g. along a Morton curve) makes the
 * charge solve's 32-atom preconditioner blocks compact and its gathers
 * local. NULL or the identity: storage order = caller order. Errors:
 * INVALID_ARG (not such a permutation), STATE (no layout, or per-atom
 * arrays already set). */
int ctbop_set_order(ctbop_system* s, const int64_t* order);

/* Copy a result out: dst (caller-owned, host or device as mem says) must
 * hold the element count the CTBOP_GET_* selector lists, in doubles; the
 * library cannot check its size. Per-atom selectors come back in the
 * caller's atom order (ctbop_set_order). mem = CTBOP_HOST synchronises the
 * system's stream; CTBOP_DEVICE is stream-ordered. Errors: INVALID_ARG
 * (null dst, unknown selector, bad mem), STATE (no layout; coordination
 * before an evaluation), CUDA. */
int ctbop_get(ctbop_system* s, int what, void* dst, int mem);

/* Synchronise and report counters and device error bits. */
int ctbop_status(ctbop_system* s, ctbop_stats* st);

/* Phases of one step, for ctbop_profile_steps. */
#define CTBOP_NPHASE 10
/* 0 kick + drift, 1 neighbour lists (flag-guarded, no-op without a rebuild),
 * 2 bond orders (Eq. 2, 7), 3 charge-system assembly, 4 CG start, 5 CG matrix
 * pass, 6 CG update, 7 charges from the CG solution, 8 covalent force slots,
 * 9 charge forces + slot gather + half kick. */

/* Run n_steps velocity-Verlet steps (same arithmetic as ctbop_step) with
 * every kernel launched directly and bracketed by CUDA events on the
 * system's stream, synchronising after each phase. Adds the GPU time of each
 * phase (ms) to ms_out[CTBOP_NPHASE] and the number of kernel launches to
 * launches_out[CTBOP_NPHASE] (host arrays, caller-owned, not cleared).
 * Slower than ctbop_step: for per-kernel timing only. */
int ctbop_profile_steps(ctbop_system* s, int64_t n_steps, double dt_fs, double* ms_out, int64_t* launches_out);

/* NVT (the paper's MD runs NVT, Sec. 3.3, naming no thermostat; read as one
 * Nose-Hoover thermostat per replica). T0[r] > 0 (K) and tau[r] > 0 (fs)
 * attach a thermostat to replica r with mass Qm = g kB T0 tau^2, g = 3 per
 * mobile atom (less 3 when the replica has no frozen atom); T0[r] <= 0 leaves
 * it NVE. Both arrays are [R], host; T0 == NULL turns every thermostat off.
 * The thermostat variables xi, eta start at 0. The extended energy
 * E + K + Qm xi^2 / 2 + g kB T0 eta is conserved by ctbop_step. Set after
 * set_layout and set_frozen. Errors: INVALID_ARG, STATE. */
int ctbop_set_thermostat(ctbop_system* s, const double* T0, const double* tau);

/* Replace the potential's parameters (copied; same validity rules as
 * ctbop_create). The next compute/step rebuilds the lists and re-captures
 * its graphs. Errors: INVALID_ARG. */
int ctbop_set_params(ctbop_system* s, const ctbop_params* p);

/* Force-matching loss and its gradient with respect to every parameter
 * (the paper fits its parameters to energies, forces and charges, Sec. 2,
 * but prints no fitting method).
 *   loss = sum_r w_E[r] (E_r - E_ref[r])^2 + sum_r w_F[r] sum_{i in r} |F_i - F_ref_i|^2
 * at the charge minimiser of the current positions. dtheta receives dloss/d
 * of every field of ctbop_params, in that struct's layout (host,
 * caller-owned; the mass fields get 0). Pair fields enter E through the
 * ordered pair (t_i, t_j): the gradient of a symmetric pair constant is the
 * sum of its two entries.
 * w_E, E_ref: [R] host or NULL (no energy term); w_F: [R] host, F_ref:
 * [N,3] host, or NULL (no force term). The energy part is the analytic
 * partial derivative at fixed charges (exact at the minimiser). The force
 * part adds the derivative of that gradient along dL/dF and the charge
 * response through one adjoint CG solve; both directional derivatives are
 * exact (forward mode). Arithmetic follows the system's policy: FP64, or FP32
 * terms with FP64 sums under CTBOP_PREC_MIXED. Leaves the system at its
 * positions with the minimiser charges, energies and forces.
 * CG_NOT_CONVERGED if the charge or adjoint solve does not converge. */
int ctbop_param_grad(ctbop_system* s, const double* w_E, const double* E_ref, const double* w_F,
                     const double* F_ref, double* loss, ctbop_params* dtheta);

/* Removal energies of the Si desorption screening (Sec. 3.3: the stability
 * of a surface Si atom is the total-energy change when it is eliminated,
 * taken every 1 ps; atoms below a threshold, 6.5 eV there, are removed).
 * For every candidate atom i (global index, cand[0..n_cand), host):
 *   dE[c] = E(replica without i) + E0_{t_i} - E(replica)
 * with every other atom in place and both energies at their charge
 * minimiser with the replica's total charge: the atom leaves as an isolated
 * neutral atom, whose energy is its self-energy constant E0 (a reading: the
 * paper does not state the reference state). Each candidate is taken alone
 * from the current state; the screening decides which to remove.
 * Evaluates the system first if it has not been (compute). The systems
 * without each candidate run as replicas of one batch, in chunks of at most
 * max_atoms atoms (0 = 4,194,304), on the system's stream; the batch system
 * is kept for the next call (its device memory grows with max_atoms).
 * dE: host, n_cand doubles, caller-owned. Errors: INVALID_ARG (an index
 * outside [0, N), null arrays), STATE (no layout, box, types or positions),
 * CG_NOT_CONVERGED (a batch solve), OOM, CUDA. */
int ctbop_removal_energies(ctbop_system* s, int64_t n_cand, const int64_t* cand, int64_t max_atoms, double* dE);

/* Energy minimisation (the paper relaxes structures and cools them to 0 K,
 * Sec. 3, naming no method): FIRE (Bitzek et al., Phys. Rev. Lett. 97,
 * 170201 (2006); N_min 5, f_inc 1.1, f_dec 0.5, alpha_start 0.1, f_alpha
 * 0.99) with the semi-implicit Euler step, on E(x) = min_q E(x, q): every
 * force evaluation solves the charges. One FIRE state per replica; over a
 * replica's mobile atoms, each iteration:
 *   stop when max_i |F_i| < fmax (eV/A);
 *   P = F . v; P >= 0: after more than N_min such iterations in a row,
 *     dt = min(f_inc dt, dt_max) and alpha *= f_alpha; then
 *     v = (1 - alpha) v + alpha |v| F / |F|;
 *   P < 0: dt *= f_dec, alpha = alpha_start, v = 0;
 *   v += dt F / m; x += dt v (dt in fs).
 * Starts from rest (velocities zeroed) at dt0 and leaves velocities zero;
 * frozen atoms never move. At most max_iter iterations per replica.
 * iters ([R] host or NULL): iterations each replica took to converge, -1 if
 * it reached max_iter first; fmax_out ([R] host or NULL): each replica's
 * max |F_i| at its last check. Returns CTBOP_OK either way.
 * Errors: INVALID_ARG (max_iter < 0, fmax <= 0, not 0 < dt0 <= dt_max),
 * STATE, CG_NOT_CONVERGED, NONFINITE, NEIGH_OVERFLOW, OOM, CUDA. */
int ctbop_minimize(ctbop_system* s, int64_t max_iter, double fmax, double dt0, double dt_max, int64_t* iters,
                   double* fmax_out);

/* One ring of the C network (ctbop_rings). */
typedef struct ctbop_ring {
    int32_t replica;      /* replica the ring's atoms belong to */
    int32_t size;         /* number of atoms, 3..8 */
    double  centre[3];    /* mean of its atoms' positions, unwrapped along the ring (A) */
    double  orientation;  /* 6-rings: in-plane angle of the vertex diagonals modulo 60 degrees (their
                             circular mean in that period), 0 when a diagonal points along x; NaN otherwise */
} ctbop_ring;

/* Ring statistics of the C network (Sec. 3.3 follows the numbers of 5-, 6-
 * and 7-membered C rings and the in-plane orientation of the 6-membered
 * ones; it gives no ring criterion). Counts primitive rings: closed paths
 * of distinct C atoms joined by C-C bonds shorter than bond_cut, whose bond
 * vectors sum to zero (a path around a periodic box is no ring), with no
 * shorter path in the bond graph between any two of their atoms (same
 * displacement) than along the ring; sizes 3..max_size (max_size <= 8).
 * bond_cut: 0 = the C-C covalent cutoff S; at most that S (the lists hold
 * every pair within it). Needs a completed compute or step (STATE).
 * Writes up to cap records to out (host, caller-owned; any order) and the
 * total number of rings to *n_rings, which may exceed cap (call again with
 * a larger cap). Errors: INVALID_ARG, STATE, OOM, CUDA. */
int ctbop_rings(ctbop_system* s, double bond_cut, int32_t max_size, int64_t cap, ctbop_ring* out, int64_t* n_rings);

/* Per-replica total energy (eV) of the last evaluation, written to
 * energy[0..R) (host array, caller-owned): the sum over each replica of the
 * per-atom energies, i.e. the value ctbop_get(CTBOP_GET_ENERGY) returns, up
 * to summation order. The paper has no counterpart: this is a library
 * utility for callers that cannot allocate device memory when they read the
 * energy. Examples: a program whose GPU memory is held by another
 * framework's caching allocator, where a new cudaMalloc can fail or force
 * that allocator to give memory back; a monitoring loop between steps, where
 * a cudaFree would synchronise the whole device and stall other streams; a
 * long run that must not fail for lack of memory once it has started. It
 * calls no allocating routine. Its scratch is a fixed file-scope device array
 * of 304 x 64 + 64 doubles plus a counter (about 156 KB, held by every GPU
 * that loads the library until the process exits), which limits it to
 * systems of at most 64 replicas (more -> CTBOP_ERR_INVALID_ARG, nothing
 * computed); there is no limit on the atom count.
 * The scratch array's address is looked up when the system is created
 * (ctbop_create, which also loads the kernel if the runtime loads modules
 * lazily), so every call, the first included, only launches one kernel on
 * the system's stream and copies R doubles back, synchronising the stream.
 * Calls must not overlap (on any stream or thread): they share the scratch.
 * Errors: INVALID_ARG (null pointer, too many replicas), STATE (no
 * evaluation yet), CUDA. */
int ctbop_energy_noalloc(ctbop_system* s, double* energy);

/* Arithmetic-pipe peaks of a GPU (a measurement utility, not part of the
 * method: the roofline of the kernels bound by arithmetic needs them, and
 * the FP32, special-function and FP64 rates are not published for every
 * part). Microkernels run independent dependent chains of one instruction
 * kind on every SM at full occupancy (FP32 fused multiply-add; the
 * special-function instructions ex2.approx and rsqrt.approx; FP64 fused
 * multiply-add), each timed by CUDA events on `cuda_stream` (a
 * cudaStream_t; null = the legacy stream) around one launch of about 40 ms
 * after a warm-up launch. Allocates and frees a small device buffer.
 * Synchronises the stream. Errors: INVALID_ARG (null out), CUDA. */
typedef struct ctbop_peaks {
    double fp32_tflops;     /* FP32 FMA rate x 2 flops (TFLOP/s) */
    double mufu_ex2_tops;   /* ex2.approx.f32 per second (1e12/s) */
    double mufu_rsq_tops;   /* rsqrt.approx.f32 per second (1e12/s) */
    double fp64_tflops;     /* FP64 FMA rate x 2 flops (TFLOP/s) */
    double ms[4];           /* timed launch of each microkernel, in that order (ms) */
    double sm_mhz;          /* median SM clock of the blocks of the FP32 launch (clock64 over globaltimer) */
    int32_t sms;            /* multiprocessors */
    int32_t pad;
} ctbop_peaks;

int ctbop_measure_peaks(int32_t device, void* cuda_stream, ctbop_peaks* out);

#ifdef __cplusplus
}
#endif

#endif /* CTBOP_H */
