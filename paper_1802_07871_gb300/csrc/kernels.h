// kernels.h — device state and kernel launchers of libctbop (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include "internal.cuh"
#include "ctbop.h"

namespace ct {

// RMS force (eV/A) below which a replica's next evaluation takes the
// accurate mode (see k_bond): outside it, with the cutoffs of taper bonds
// from FP64 positions (cutoff_fp64), the largest FP32 force error measured
// on hot slabs (2000-2500 K, after 50-400 steps) is 1.4e-5 of the RMS force
// (about 2.5e-5 eV/A), so a 1e-4 bar relative to the RMS force holds from
// about 0.25 eV/A on; the threshold keeps a margin of four.
#define ACC_RMS 1.0

// Offsets (in doubles) of the fields of ctbop_params: the layout of a
// parameter gradient.
enum ParamOffsets {
  PG_A = 0, PG_B = 4, PG_L1 = 8, PG_L2 = 12, PG_R = 16, PG_S = 20, PG_KAPPA = 24,
  PG_SIGMA = 28, PG_P = 32, PG_G = 36, PG_N = 44,
  PG_GAMMA = 52, PG_C = 68, PG_D = 84, PG_H = 100, PG_ALPHA = 116,
  PG_E0 = 132, PG_CHI = 134, PG_J = 136, PG_GAMMA_C = 138, PG_MASS = 140,
  PG_RCOUL = 142, PG_KE = 143, PG_NPARAM = 144
};

// Per-replica double accumulators, one row of RA_STRIDE per replica.
enum RepSlots {
  RA_E = 0,        // potential energy
  RA_KE = 1,       // kinetic energy
  RA_F2 = 2,       // sum of |F_i|^2 (the RMS force that selects the next evaluation's precision mode)
  RA_W = 3,        // virial, 9 components
  RA_STRIDE = 12
};

// Nose-Hoover thermostat per replica (double), see md.cu.
enum NhSlots {
  NH_XI = 0,       // xi (1/fs)
  NH_ETA = 1,      // eta (fs)
  NH_QM = 2,       // Qm (eV fs^2)
  NH_GKT = 3,      // g kB T0 (eV)
  NH_ON = 4,       // 1 when the replica has a thermostat
  NH_QINV = 5,     // 1 / Qm
  NH_XIH = 6,      // xi after this step's first half-update
  NH_STRIDE = 8
};

// CG scalars per replica (double), see cg.cu.
enum CgSlots {
  CG_DOTS = 0,     // [2 buffers][2]: r.z, w.z
  CG_UPD = 4,      // [3 buffers][4]: sum y, sum r, sum r^2, (unused)
  CG_SCAL = 16,    // [2 buffers][2]: gamma, alpha of an iteration
  CG_AB = 20,      // alpha, beta of the running iteration
  CG_C = 22,       // c = sum y / sum d of the running iteration
  CG_SD = 23,      // sum d (d = D^-1 1)
  CG_SQ0 = 24,     // sum of the extrapolated starting guess
  CG_DQ = 25,      // uniform shift putting the starting guess on sum q = Q
  CG_M = 26,       // mean of the stored (re-centred) r
  CG_SHIFT = 27,   // total subtracted from r by the re-centring
  CG_MU = 28,      // mu = -mean(r), the electronegativity
  CG_RES = 29,     // rms of r - mean(r)
  CG_RESMAX = 30,  // max |r - mean(r)|
  CG_Q = 31,       // requested total charge
  CG_NAT = 32,     // atoms in the replica
  CG_RES0 = 33,    // max |r - mean(r)| of the starting guess
  CG_SQF = 34,     // sum of q + dq after the iteration (the final neutrality shift)
  CG_STRIDE = 36
};

struct DevState {
  int N = 0, R = 0, ncells = 0;
  int cap_cov = 0, cap_all = 0;
  int ld = 0;                   // column stride of the lists: N rounded up to 32
  // per atom
  double *x = nullptr, *v = nullptr, *F = nullptr, *xref = nullptr, *q = nullptr, *e_atom = nullptr;
  int *type = nullptr, *rep = nullptr;
  uint8_t* frozen = nullptr;
  int4* cell4 = nullptr;
  void* u = nullptr;            // Real4[N]
  // per replica
  RepInfo* reps = nullptr;
  double* rep_acc = nullptr;    // [R][RA_STRIDE]
  double* cg = nullptr;         // [R][CG_STRIDE]
  double* nh = nullptr;         // [R][NH_STRIDE] thermostats
  int* cg_conv = nullptr;       // [R] converged flag
  int* cg_iters = nullptr;      // [R] iterations used
  // cells
  int *cell_count = nullptr, *cell_fill = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
  int* cell_rep = nullptr;      // [ncells] replica of each cell
  int* scan_tmp = nullptr;      // >= 1025 ints
  // lists
  int2* nl = nullptr;           // [cap_all*ld] (j, code) list entries, column-major
  int *ncov = nullptr, *nall = nullptr, *rev = nullptr;
  int* nfix = nullptr;          // [N] end of the core part of each list (covalent + core entries)
  int* nmat = nullptr;          // [N] stored charge-matrix entries per atom: the list entries inside the
                                // charge cutoff (FP32, compacted), or nall (FP64)
  int2* lst = nullptr;          // [N][cap_all] row-major build scratch (j, code)
  // stiff covalent bonds (FP32 path): a queue of bond ids i * cap_cov + e and,
  // per bond, the FP64-evaluated pair term (dE/dr, energy) as double2
  int* stiff_n = nullptr;
  int* stiff_q = nullptr;       // [N * cap_cov]
  // atoms whose covalent terms the FP32 path recomputes in FP64 (accurate
  // mode, see k_bond): a queue of atom ids, FP64 cell offsets of every atom
  // and FP64 bond orders of the queued atoms; sum |F|^2 of each replica's
  // previous evaluation (0: none yet, the accurate mode)
  int* flag_n = nullptr;
  int* flag_q = nullptr;        // [N]
  void* u64 = nullptr;          // double4 [N]
  void* bo64 = nullptr;         // double4 [N * cap_cov]
  int* acc_mode = nullptr;      // [R] 1: the replica's evaluation takes the FP32 path's accurate mode
  const PotParams<double>* Pd = nullptr;   // host copy of the FP64 parameters
  void* stiff_pe = nullptr;     // double2 [N * cap_cov]
  void* bo = nullptr;           // Real4[N*cap_cov]
  void* gslot = nullptr;        // Real4[N*cap_cov]
  void* M = nullptr;            // [cap_all*ld] charge matrix: FP32 (j, coefficient) int2 pairs, or FP64 coefficients
  void *Dg = nullptr, *dinv = nullptr;   // Real[N]: Hessian diagonal without self-images, Jacobi inverse
  // CG: the iterate is q itself (FP64); the rest in the working precision
  double *cqh1 = nullptr, *cqh2 = nullptr;  // q of the previous two solves
  void *cr = nullptr, *cp = nullptr, *cs = nullptr;  // Real[N]: r (shifted), p, s = H p
  void* cdq = nullptr;          // Real[N]: q - q0, the iteration's change (added to q at the end)
  void *cy = nullptr, *cw = nullptr, *cd = nullptr, *cv = nullptr;  // Real[N]: y = D^-1 r, w = H z, d = D^-1 1, v = H d
  unsigned long long* cg_rmax = nullptr;  // [R][3 buffers][2]: max r, max -r (order-preserving map)
  void* qr = nullptr;           // Real[N]: charges in the working precision
  int* cg_hist = nullptr;       // solutions held in q, cqh1, cqh2 (0..3)
  // control
  int* flag_rebuild = nullptr;
  int* flag_one = nullptr;      // a flag that stays 1 (list-build tuning)
  long long* rebuild_count = nullptr;
  int* maxcnt = nullptr;        // [3] at the last rebuild: max ncov, max count of the rest, max nall
  unsigned* err = nullptr;
  int* cg_it = nullptr;         // iteration counter of the running solve
  int* cg_blocks = nullptr;     // last-block counters [3]
  int* cg_active = nullptr;     // 1 while the solve runs (host-loop mirror of the graph condition)
  long long* cg_total = nullptr;
  // sizes for launches
  int nsm = 152;
  int mv_batch = 16;            // list entries in flight per thread in the CG matrix pass (tuned)
  int asm_batch = 8;            // list entries in flight per thread in the assembly (tuned)
  int gather_batch = 8;         // list entries in flight per thread in the charge-force gather (tuned)
  int cov_lanes = 8;            // lanes per atom in the covalent passes (4, 8 or 16; tuned)
  int cov_lanes_ok = 7;         // lane counts whose blocks fit shared memory (bits: 4, 8, 16)
  int build_shape = 3;          // list-build shape: index into the (warps, stencil batch) table (tuned)
  // charge-CG preconditioner: block-Jacobi on 32-atom blocks (1) or Jacobi (0)
  int precond = 1;
  void* binv = nullptr;         // [ceil(N/32)][32][32] block inverses, row by row per block: FP16 (FP32 path) or FP64
  void* bsum = nullptr;         // Real[N]: row sums of the block inverses (d = M^-1 1)
  long long* precond_epoch = nullptr;   // rebuild count the block inverses were formed at (-1: never)
  void* stage = nullptr;        // [N * 24 bytes] staging for per-atom inputs and outputs in the caller's order
};

struct SolveCfg {
  double tol;
  int max_iter;
  int use_cond;
  cudaGraphConditionalHandle cond;
};

template <class R> void launch_rebuild(const DevState& S, const PotParams<R>& P, cudaStream_t st);
template <class R> void launch_bond(const DevState& S, const PotParams<R>& P, cudaStream_t st);
template <class R> void launch_assemble(const DevState& S, const PotParams<R>& P, const TypeParams& T,
                                        cudaStream_t st);
template <class R> void launch_cg_begin(const DevState& S, const TypeParams& T, cudaStream_t st, double tol,
                                        const double* rhs = nullptr);
template <class R> void launch_cg_iter(const DevState& S, const SolveCfg& cfg, cudaStream_t st);
template <class R> void launch_cg_end(const DevState& S, cudaStream_t st);
template <class R> void launch_cg_mv(const DevState& S, cudaStream_t st);
template <class R> cudaError_t tune_cg_mv(DevState& S, cudaStream_t st, float* ms_out);
template <class R> void launch_cg_up(const DevState& S, const SolveCfg& cfg, cudaStream_t st);
template <class R> void launch_cov_force(const DevState& S, const PotParams<R>& P, const TypeParams& T,
                                         cudaStream_t st);
// virial: accumulate the virial (an evaluation) or not (an MD step: the
// library recomputes it when it is read after steps)
template <class R> void launch_coul_gather(const DevState& S, const PotParams<R>& P, const TypeParams& T,
                                           int kick, double half_dt, cudaStream_t st, bool virial);
template <class R> void launch_forces(const DevState& S, const PotParams<R>& P, const TypeParams& T,
                                      int kick, double half_dt, cudaStream_t st, bool virial);
template <class R> void launch_kick_drift(const DevState& S, const TypeParams& T, double dt, double half_skin2,
                                          cudaStream_t st);
void launch_zero_acc(const DevState& S, cudaStream_t st);
void launch_nh_end(const DevState& S, double dt, cudaStream_t st);
template <class R> cudaError_t setup_pot(int cap_cov, int* lanes_ok);
template <class R> void launch_copy_q(const DevState& S, cudaStream_t st);
// launch shape for kernels with one thread per atom: resident blocks only,
// each block a contiguous chunk of atoms (a multiple of its size)
int atom_dims(int N, int nsm, const void* kernel, int threads, int& chunk);
template <class R> void launch_block_setup(const DevState& S, cudaStream_t st);
template <class R>
cudaError_t tune_assemble(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st, float* ms_out);
template <class R>
cudaError_t tune_gather(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st, float* ms_out);
// List-build shapes (csrc/nbr.cu): warps per block x stencil cells per batch
#define BUILD_SHAPES 6
int build_shape_index(int warps, int batch);   // -1 if not a shape
void build_shape_of(int k, int* warps, int* batch);
template <class R>
cudaError_t tune_build(DevState& S, const PotParams<R>& P, const int* one, cudaStream_t st, float* ms_out);
template <class R>
cudaError_t tune_cov(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st, float* ms_out,
                     bool fast);
// Parameter gradient of the energy (csrc/grad.cu), in FP32 (fp32) or FP64
// arithmetic with FP64 sums. grad[0..143] = sum_r wval_r dE_r/dtheta at the
// current positions and charges. With a direction dir ([N,3], positions)
// and/or qdir ([N], charges), grad[144..287] = sum_r wtan_r d/de dE_r/dtheta
// along (x + e dir, q + e qdir), exact (forward mode); with dir, vout ([N])
// = d/de (H q + chi)(x + e dir) at fixed charges. Without a direction the
// tangents stay zero and vout is unused.
cudaError_t launch_param_grad(const DevState& S, const ::ctbop_params& P, bool fp32, const double* wval,
                              const double* wtan, const double* dir, const double* qdir, double* grad,
                              double* vout, cudaStream_t st);
// Energy minimisation (csrc/relax.cu): one FIRE state per replica,
// [R][FI_STRIDE] doubles; FI_P..FI_FMAX2 are the per-iteration sums.
enum FireSlots {
  FI_P = 0, FI_VV = 1, FI_FF = 2, FI_FMAX2 = 3, FI_DT = 4, FI_ALPHA = 5, FI_NPOS = 6,
  FI_DONE = 7,     // 0 moving, 1 converged, -1 stopped at the iteration limit
  FI_CV = 8, FI_CF = 9, FI_ITERS = 10, FI_LASTF2 = 11, FI_STRIDE = 12
};
struct FireCfg {
  double fmax2, dt_max, f_inc, f_dec, alpha0, f_alpha, n_min, max_iter;
};
void launch_fire_reduce(const DevState& S, double* fire, const FireCfg& cfg, int* blocks, int* active,
                        cudaStream_t st);
template <class R>
void launch_fire_move(const DevState& S, const TypeParams& T, const double* fire, double half_skin2,
                      cudaStream_t st);
// Primitive C rings (csrc/rings.cu): records appended through *count (the
// total, which may exceed cap; records past cap are dropped).
template <class R>
void launch_rings(const DevState& S, double bond_cut, int max_size, ::ctbop_ring* out, long long cap,
                  unsigned long long* count, cudaStream_t st);
// Storage order (csrc/order.cu): dst[k] = src[order[k]] (to_storage) or
// dst[order[k]] = src[k], elements of 1, 4, 8 or 24 bytes.
cudaError_t launch_permute(int N, const int* order, const void* src, void* dst, int elem_bytes, bool to_storage,
                           cudaStream_t st);
// Desorption screening (csrc/screen.cu): covalent coordination per atom
// (neighbours within S of the pair) and the leave-one-out gather, one item
// per batch replica: source replica [src_off, src_off + src_n) without its
// local atom drop, written from dst_off on.
struct LooItem {
  long long src_off;
  int src_n;
  int drop;
  long long dst_off;
};
template <class R> void launch_coordination(const DevState& S, const PotParams<R>& P, double* out, cudaStream_t st);
void launch_loo_gather(const LooItem* items, int n_items, int max_n, const DevState& S, double* ox, int* otype,
                       uint8_t* ofrozen, double* oq, cudaStream_t st);
int noalloc_setup(void** addr, std::string& why);
int energy_noalloc(const double* e_atom, const int* rep, int N, int R, void* scratch, cudaStream_t st,
                   double* host_out, std::string& why);

}  // namespace ct
