// api.cu — the C ABI of libctbop (include/ctbop.h): system state, device
// memory, parameter packing, the evaluation sequence, CUDA-graph capture
// (the charge CG loop is a conditional WHILE node) and MD stepping.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctbop.h"
#include "kernels.h"

using namespace ct;

namespace {

const double kAcc = 9.648533212e-3;   // 1 eV/(A u) in A/fs^2
const double kKB = 8.617333262e-5;    // Boltzmann constant, eV/K

struct DevBuf {
  std::vector<void*> ptrs;
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// Temporary device buffers of one call, stream-ordered, freed on every
// return path (error returns included).
// From the system's own memory pool (which keeps what it has mapped: a pool
// that returns its memory at every synchronisation made each call pay about
// 0.2 ms at 1M atoms to map it again), or the device's default pool.
struct Scratch {
  cudaStream_t st;
  cudaMemPool_t pool;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s, cudaMemPool_t p = nullptr) : st(s), pool(p) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  template <class T> cudaError_t alloc(T** out, size_t n) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, bytes, pool, st) : cudaMallocAsync(&q, bytes, st);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    *out = static_cast<T*>(q);
    return cudaSuccess;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, st);
  }
};

}  // namespace

struct ctbop_system {
  ctbop_params p;
  ctbop_options o;
  cudaStream_t stream = nullptr;       // stream all work is ordered on
  cudaStream_t own_stream = nullptr;   // used when the caller gives none
  cudaMemPool_t pool = nullptr;        // per-call scratch (Scratch)
  cudaStream_t body_stream = nullptr;
  void* noalloc_scratch = nullptr;     // the allocation-free energy's scratch array on this device
  std::string err;
  DevState S;
  PotParams<float> Pf;
  PotParams<double> Pd;
  TypeParams T;
  bool mixed = true;
  double rlist = 0.0;
  // host-side layout
  int R = 0;
  std::vector<int64_t> off;
  std::vector<double> box;      // R*3
  std::vector<uint8_t> pbc;     // R*3
  std::vector<double> Q;        // R
  bool have_layout = false, have_box = false, have_types = false, have_pos = false;
  bool have_forces = false, need_rebuild = true, reps_dirty = true, caps_known = false;
  bool virial_stale = false;   // MD steps leave the virial out of the replica sums
  // allocations
  DevBuf atom_buf, list_buf, cell_buf, rep_buf;
  int alloc_N = -1, alloc_R = -1, alloc_cells = -1, alloc_cov = -1, alloc_all = -1;
  // graphs
  cudaGraphExec_t g_eval = nullptr, g_step = nullptr;
  bool nvt = false;             // some replica has a Nose-Hoover thermostat
  // matrix-pass autotuning: the lists it was tuned on, and the timings
  int tuned_N = -1, tuned_cap = -1;
  float mv_ms[3] = {0.f, 0.f, 0.f};
  float asm_ms[3] = {0.f, 0.f, 0.f};
  float gather_ms[3] = {0.f, 0.f, 0.f};
  bool gather_forced = false;
  float cov_ms[3] = {0.f, 0.f, 0.f};
  // a step chunk's starting state, for redoing it after a list overflow
  double *snap_x = nullptr, *snap_v = nullptr, *snap_F = nullptr, *snap_q = nullptr;
  bool cov_forced = false;
  float build_ms[BUILD_SHAPES] = {};
  bool tune_pending = false;
  double g_step_dt = -1.0;
  bool use_graph = true;
  // pinned host scratch
  int* h_int = nullptr;
  // counters
  int64_t steps = 0, solves = 0;
  // leave-one-out batches of the desorption screening (created on first use)
  ctbop_system* loo = nullptr;
  // storage order (ctbop_set_order): slot k holds the caller's atom order[k]
  bool ordered = false;
  std::vector<int64_t> order, slot;
  int* d_order = nullptr;
};

static int fail(ctbop_system* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(s, e_ == cudaErrorMemoryAllocation ? CTBOP_ERR_OOM : CTBOP_ERR_CUDA,    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

template <class T>
static cudaError_t dalloc(DevBuf& b, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  b.ptrs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// ------------------------------------------------------------- parameters
template <class Rr>
static void pack_params(const ctbop_params& p, double skin, PotParams<Rr>& P) {
  for (int k = 0; k < 4; ++k) {
    P.A[k] = (Rr)p.A[k];
    P.B[k] = (Rr)p.B[k];
    P.lam1[k] = (Rr)p.lambda1[k];
    P.lam2[k] = (Rr)p.lambda2[k];
    P.Rin[k] = (Rr)p.R[k];
    P.Sout[k] = (Rr)p.S[k];
    P.kappa[k] = (Rr)p.kappa[k];
    P.pi_SR[k] = (Rr)(M_PI / (p.S[k] - p.R[k]));
    P.A64[k] = p.A[k];
    P.B64[k] = p.B[k];
    P.lam1_64[k] = p.lambda1[k];
    P.lam2_64[k] = p.lambda2[k];
    P.Rin64[k] = p.R[k];
    P.Sout64[k] = p.S[k];
    P.kappa64[k] = p.kappa[k];
    P.rcov_list2[k] = (Rr)((p.S[k] + skin) * (p.S[k] + skin));
    double sg = p.sigma[k], pp = p.p[k];
    P.sigma[k] = (Rr)sg;
    P.p[k] = (Rr)pp;
    P.g1[k] = (Rr)p.g[k][0];
    P.g2[k] = (Rr)p.g[k][1];
    P.n1[k] = (Rr)p.n[k][0];
    P.n2[k] = (Rr)p.n[k][1];
    // G normalises b to 1 at zeta = 0 (Sec. 2, after Eq. 5 and Eq. 7)
    P.G[k] = (Rr)std::pow(std::pow(p.g[k][0], -pp) + std::pow(p.g[k][1], -pp), -1.0 / (2.0 * sg * pp));
    P.inv2s[k] = (Rr)(1.0 / (2.0 * sg));
    P.inv2sp[k] = (Rr)(1.0 / (2.0 * sg * pp));
    int a = k / 2, b = k % 2;
    P.gshield3[k] = (Rr)std::pow(p.gamma_c[a] * p.gamma_c[b], -1.5);
  }
  for (int t = 0; t < 8; ++t)
    for (int l = 0; l < 2; ++l) {
      P.gam[t][l] = (Rr)p.gamma[t][l];
      P.c2[t][l] = (Rr)(p.c[t][l] * p.c[t][l]);
      P.d2[t][l] = (Rr)(p.d[t][l] * p.d[t][l]);
      P.h[t][l] = (Rr)p.h[t][l];
      P.alpha[t][l] = (Rr)p.alpha[t][l];
      P.c2d2[t][l] = (Rr)(p.c[t][l] * p.c[t][l] / (p.d[t][l] * p.d[t][l]));
    }
  P.rcoul = (Rr)p.r_coul;
  P.inv_rcoul = (Rr)(1.0 / p.r_coul);
  P.ke = (Rr)p.k_e;
  P.rall_list2 = (Rr)((p.r_coul + skin) * (p.r_coul + skin));
  P.rcore_list2 = p.r_coul > skin ? (Rr)((p.r_coul - skin) * (p.r_coul - skin)) : (Rr)0;
}

static bool params_valid(const ctbop_params* p, std::string& why) {
  for (int k = 0; k < 4; ++k) {
    if (!(p->R[k] > 0 && p->S[k] > p->R[k])) { why = "need 0 < R < S for every pair"; return false; }
    if (!(p->sigma[k] > 0 && p->p[k] > 0 && p->g[k][0] > 0 && p->g[k][1] > 0 && p->n[k][0] > 0 && p->n[k][1] > 0)) {
      why = "sigma, p, g_l, n_l must be positive (Sec. 2)";
      return false;
    }
  }
  for (int t = 0; t < 2; ++t) {
    if (!(p->mass[t] > 0)) { why = "masses must be positive"; return false; }
    if (!(p->gamma_c[t] > 0)) { why = "charge shielding gamma_c must be positive"; return false; }
    if (!(p->J[t] > 0)) { why = "J must be positive"; return false; }
  }
  double smax = 0;
  for (int k = 0; k < 4; ++k) smax = std::max(smax, p->S[k]);
  if (!(p->r_coul >= smax)) { why = "charge cutoff must be at least the largest covalent cutoff"; return false; }
  return true;
}

// ------------------------------------------------------------- helpers
// Stream-ordered transfers. The library's kernels run on s->stream, which
// may be a non-blocking stream (the usual kind from a framework's stream
// pool); the legacy default stream, where a plain cudaMemcpy or cudaMemset
// runs, is not ordered with such a stream in either direction.
static cudaError_t sync_copy(ctbop_system* s, void* dst, const void* src, size_t n, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n, kind, s->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(s->stream);
}
static cudaError_t zero_async(ctbop_system* s, void* p, size_t n) { return cudaMemsetAsync(p, 0, n, s->stream); }

static void destroy_graphs(ctbop_system* s) {
  if (s->g_eval) cudaGraphExecDestroy(s->g_eval);
  if (s->g_step) cudaGraphExecDestroy(s->g_step);
  s->g_eval = s->g_step = nullptr;
  s->g_step_dt = -1.0;
}

static int setup_reps(ctbop_system* s) {
  std::vector<RepInfo> info(s->R);
  int cells = 0;
  for (int r = 0; r < s->R; ++r) {
    RepInfo& ri = info[r];
    memset(&ri, 0, sizeof(ri));
    for (int d = 0; d < 3; ++d) {
      double L = s->box[3 * r + d];
      ri.L[d] = L;
      ri.pbc[d] = s->pbc[3 * r + d] ? 1 : 0;
      int n = (int)std::floor(L / (0.5 * s->rlist));
      if (n < 1) n = 1;
      if (n > 4096) n = 4096;
      ri.n[d] = n;
      ri.hc[d] = L / n;
      ri.hcf[d] = (float)ri.hc[d];
      int m = (int)std::ceil(s->rlist / ri.hc[d] - 1e-12);
      if (m < 1) m = 1;
      if (!ri.pbc[d] && m > n - 1) m = std::max(1, n - 1);
      if (m > 8) return fail(s, CTBOP_ERR_INVALID_ARG, "box edge too small for the cutoff (more than 8 cells of stencil)");
      ri.m[d] = m;
    }
    long long nc = (long long)ri.n[0] * ri.n[1] * ri.n[2];
    if (cells + nc > 4 * 1024 * 1024) return fail(s, CTBOP_ERR_INVALID_ARG, "too many cells (more than 4M)");
    ri.cell_off = cells;
    cells += (int)nc;
    ri.atom_off = (int)s->off[r];
    ri.natoms = (int)(s->off[r + 1] - s->off[r]);
  }
  if (s->alloc_cells < cells) {
    s->cell_buf.release();
    DevState& S = s->S;
    CK(dalloc(s->cell_buf, &S.cell_count, cells));
    CK(dalloc(s->cell_buf, &S.cell_fill, cells));
    CK(dalloc(s->cell_buf, &S.cell_start, cells));
    CK(dalloc(s->cell_buf, &S.cell_rep, cells));
    s->alloc_cells = cells;
    destroy_graphs(s);
  }
  s->S.ncells = cells;
  CK(sync_copy(s, s->S.reps, info.data(), sizeof(RepInfo) * s->R, cudaMemcpyHostToDevice));
  {
    std::vector<int> crep(cells);
    for (int r = 0; r < s->R; ++r) {
      int end = r + 1 < s->R ? info[r + 1].cell_off : cells;
      for (int c = info[r].cell_off; c < end; ++c) crep[c] = r;
    }
    CK(sync_copy(s, s->S.cell_rep, crep.data(), sizeof(int) * cells, cudaMemcpyHostToDevice));
  }
  // per-replica CG constants
  std::vector<double> cg((size_t)s->R * CG_STRIDE, 0.0);
  for (int r = 0; r < s->R; ++r) {
    cg[(size_t)r * CG_STRIDE + CG_Q] = s->Q[r];
    cg[(size_t)r * CG_STRIDE + CG_NAT] = (double)(s->off[r + 1] - s->off[r]);
  }
  CK(sync_copy(s, s->S.cg, cg.data(), sizeof(double) * cg.size(), cudaMemcpyHostToDevice));
  s->reps_dirty = false;
  return CTBOP_OK;
}

static int alloc_atoms(ctbop_system* s) {
  DevState& S = s->S;
  int N = (int)s->off[s->R];
  if (s->alloc_N == N && s->alloc_R == s->R) return CTBOP_OK;
  destroy_graphs(s);
  s->atom_buf.release();
  s->rep_buf.release();
  s->list_buf.release();
  s->alloc_cov = s->alloc_all = -1;
  S.N = N;
  S.R = s->R;
  size_t rs = s->mixed ? 4 : 8;
  CK(dalloc(s->atom_buf, &S.x, 3 * (size_t)N));
  CK(dalloc(s->atom_buf, &S.v, 3 * (size_t)N));
  CK(dalloc(s->atom_buf, &S.F, 3 * (size_t)N));
  CK(dalloc(s->atom_buf, &S.xref, 3 * (size_t)N));
  CK(dalloc(s->atom_buf, &S.q, (size_t)N));
  CK(dalloc(s->atom_buf, &S.e_atom, (size_t)N));
  CK(dalloc(s->atom_buf, &S.type, (size_t)N));
  CK(dalloc(s->atom_buf, &S.rep, (size_t)N));
  CK(dalloc(s->atom_buf, &S.frozen, (size_t)N));
  CK(dalloc(s->atom_buf, &S.cell4, (size_t)N));
  unsigned char* u = nullptr;
  CK(dalloc(s->atom_buf, &u, (size_t)N * 4 * rs));
  S.u = u;
  CK(dalloc(s->atom_buf, &S.cell_atoms, (size_t)N));
  {
    void** rv[] = {&S.Dg, &S.dinv, &S.cy, &S.cw, &S.cd, &S.cv, &S.qr, &S.cr, &S.cp, &S.cs, &S.cdq};
    for (void** pp : rv) {
      unsigned char* b = nullptr;
      CK(dalloc(s->atom_buf, &b, (size_t)N * rs));
      *pp = b;
    }
  }
  {
    unsigned char *bi = nullptr, *bs = nullptr;
    CK(dalloc(s->atom_buf, &bi, (size_t)((N + 31) / 32) * 1024 * rs));
    CK(dalloc(s->atom_buf, &bs, (size_t)N * rs));
    S.binv = bi;
    S.bsum = bs;
  }
  {
    unsigned char* sg = nullptr;
    CK(dalloc(s->atom_buf, &sg, (size_t)N * 24));
    S.stage = sg;
  }
  // kept allocated: a stream-ordered allocation per ctbop_step call returned
  // its memory to the pool's owner at every synchronisation and cost about
  // 0.2 ms per call at 1M atoms
  CK(dalloc(s->atom_buf, &s->snap_x, 3 * (size_t)N + 1));
  CK(dalloc(s->atom_buf, &s->snap_v, 3 * (size_t)N + 1));
  CK(dalloc(s->atom_buf, &s->snap_F, 3 * (size_t)N + 1));
  CK(dalloc(s->atom_buf, &s->snap_q, (size_t)N + 1));
  CK(dalloc(s->atom_buf, &S.cqh1, (size_t)N));
  CK(dalloc(s->atom_buf, &S.cqh2, (size_t)N));
  CK(dalloc(s->atom_buf, &S.ncov, (size_t)N));
  CK(dalloc(s->atom_buf, &S.nall, (size_t)N));
  CK(dalloc(s->atom_buf, &S.nfix, (size_t)N));
  if (s->mixed) {
    CK(dalloc(s->atom_buf, &S.nmat, (size_t)N));
    CK(zero_async(s, S.nmat, sizeof(int) * (size_t)N));
  } else {
    S.nmat = S.nall;   // FP64 keeps the coefficients aligned with the list
  }
  CK(zero_async(s, S.v, sizeof(double) * 3 * (size_t)N));
  CK(zero_async(s, S.F, sizeof(double) * 3 * (size_t)N));
  CK(zero_async(s, S.q, sizeof(double) * (size_t)N));
  CK(zero_async(s, S.frozen, (size_t)N));
  CK(zero_async(s, S.cqh1, sizeof(double) * (size_t)N));
  CK(zero_async(s, S.cqh2, sizeof(double) * (size_t)N));
  CK(zero_async(s, S.cp, (size_t)N * rs));
  CK(zero_async(s, S.cs, (size_t)N * rs));
  CK(zero_async(s, S.qr, (size_t)N * rs));
  // replica ids
  std::vector<int> rep(N);
  for (int r = 0; r < s->R; ++r)
    for (int64_t i = s->off[r]; i < s->off[r + 1]; ++i) rep[i] = r;
  CK(sync_copy(s, S.rep, rep.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
  // per-replica and control
  CK(dalloc(s->rep_buf, &S.reps, (size_t)s->R));
  CK(dalloc(s->rep_buf, &S.rep_acc, (size_t)s->R * RA_STRIDE));
  CK(dalloc(s->rep_buf, &S.cg, (size_t)s->R * CG_STRIDE));
  CK(dalloc(s->rep_buf, &S.nh, (size_t)s->R * NH_STRIDE));
  CK(zero_async(s, S.nh, sizeof(double) * s->R * NH_STRIDE));
  s->nvt = false;
  CK(dalloc(s->rep_buf, &S.cg_rmax, (size_t)s->R * 6));
  CK(dalloc(s->rep_buf, &S.cg_conv, (size_t)s->R));
  CK(dalloc(s->rep_buf, &S.cg_iters, (size_t)s->R));
  CK(dalloc(s->rep_buf, &S.scan_tmp, 1040));
  CK(dalloc(s->rep_buf, &S.flag_rebuild, 1));
  CK(dalloc(s->rep_buf, &S.flag_one, 1));
  {
    int one = 1;
    CK(cudaMemcpyAsync(S.flag_one, &one, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  CK(dalloc(s->rep_buf, &S.rebuild_count, 1));
  CK(dalloc(s->rep_buf, &S.precond_epoch, 1));
  CK(cudaMemsetAsync(S.precond_epoch, 0xff, sizeof(long long), s->stream));   // -1: form at the first solve
  CK(dalloc(s->rep_buf, &S.maxcnt, 3));
  CK(dalloc(s->rep_buf, &S.stiff_n, 1));
  CK(zero_async(s, S.stiff_n, sizeof(int)));
  CK(dalloc(s->rep_buf, &S.acc_mode, (size_t)s->R));
  CK(cudaMemsetAsync(S.acc_mode, 0, sizeof(int) * s->R, s->stream));
  if (s->mixed) {
    CK(dalloc(s->rep_buf, &S.flag_n, 1));
    CK(zero_async(s, S.flag_n, sizeof(int)));
    CK(dalloc(s->atom_buf, &S.flag_q, (size_t)std::max(N, 1)));
    unsigned char* u64 = nullptr;
    CK(dalloc(s->atom_buf, &u64, (size_t)std::max(N, 1) * 32));
    S.u64 = u64;
  }
  CK(dalloc(s->rep_buf, &S.err, 1));
  CK(dalloc(s->rep_buf, &S.cg_it, 1));
  CK(dalloc(s->rep_buf, &S.cg_blocks, 3));
  CK(dalloc(s->rep_buf, &S.cg_hist, 1));
  CK(dalloc(s->rep_buf, &S.cg_active, 1));
  CK(dalloc(s->rep_buf, &S.cg_total, 1));
  CK(zero_async(s, S.rep_acc, sizeof(double) * s->R * RA_STRIDE));
  CK(zero_async(s, S.rebuild_count, sizeof(long long)));
  CK(zero_async(s, S.err, sizeof(unsigned)));
  CK(zero_async(s, S.cg_total, sizeof(long long)));
  CK(zero_async(s, S.cg_blocks, 3 * sizeof(int)));
  CK(zero_async(s, S.cg_hist, sizeof(int)));
  CK(zero_async(s, S.maxcnt, 3 * sizeof(int)));
  CK(zero_async(s, S.cg_it, sizeof(int)));
  s->alloc_N = N;
  s->alloc_R = s->R;
  s->reps_dirty = true;
  s->caps_known = false;
  s->have_forces = false;
  return CTBOP_OK;
}

static int alloc_lists(ctbop_system* s, int cap_cov, int cap_all) {
  DevState& S = s->S;
  // capacities rounded to multiples of 8 (all entries) and 4 (covalent)
  cap_all = (std::max(cap_all, cap_cov) + 7) & ~7;
  cap_cov = (cap_cov + 3) & ~3;
  if (s->alloc_cov == cap_cov && s->alloc_all == cap_all) return CTBOP_OK;
  destroy_graphs(s);
  s->list_buf.release();
  int N = S.N;
  size_t rs = s->mixed ? 4 : 8;
  S.cap_cov = cap_cov;
  S.cap_all = cap_all;
  S.ld = ((N + 31) / 32) * 32;
  if (S.ld == 0) S.ld = 32;
  size_t ncol = (size_t)S.ld * cap_all;
  CK(dalloc(s->list_buf, &S.nl, ncol));
  CK(dalloc(s->list_buf, &S.lst, (size_t)std::max(N, 1) * cap_all));
  CK(dalloc(s->list_buf, &S.rev, (size_t)N * cap_cov));
  CK(dalloc(s->list_buf, &S.stiff_q, (size_t)std::max(N, 1) * cap_cov));
  if (s->mixed) {
    unsigned char* b64 = nullptr;
    CK(dalloc(s->list_buf, &b64, (size_t)std::max(N, 1) * cap_cov * 32));
    S.bo64 = b64;
  }
  {
    double2* pe = nullptr;
    CK(dalloc(s->list_buf, &pe, (size_t)std::max(N, 1) * cap_cov));
    S.stiff_pe = pe;
  }
  unsigned char *bo = nullptr, *gs = nullptr, *M = nullptr;
  CK(dalloc(s->list_buf, &bo, (size_t)N * cap_cov * 4 * rs));
  CK(dalloc(s->list_buf, &gs, (size_t)N * cap_cov * 4 * rs));
  // 8 bytes per entry: (j, FP32 coefficient) pairs, or FP64 coefficients
  CK(dalloc(s->list_buf, &M, ncol * 8));
  CK(zero_async(s, M, ncol * 8));    // defined values for the first tuning run
  S.bo = bo;
  S.gslot = gs;
  S.M = M;
  if (cap_cov > 512) return fail(s, CTBOP_ERR_NEIGH_OVERFLOW, "covalent entries per atom beyond 512");
  CK(s->mixed ? setup_pot<float>(cap_cov, &S.cov_lanes_ok) : setup_pot<double>(cap_cov, &S.cov_lanes_ok));
  if (!(S.cov_lanes_ok & (S.cov_lanes == 4 ? 1 : S.cov_lanes == 8 ? 2 : 4))) {
    S.cov_lanes = (S.cov_lanes_ok & 2) ? 8 : 16;
    destroy_graphs(s);
  }
  s->alloc_cov = cap_cov;
  s->alloc_all = cap_all;
  return CTBOP_OK;
}

// The next evaluation of every replica in the accurate mode of the FP32
// path (see k_bond): no previous RMS force counts for new positions, box,
// types or parameters.
static int reset_precision_mode(ctbop_system* s) {
  if (s->alloc_N < 0 || !s->S.rep_acc) return CTBOP_OK;
  CK(cudaMemset2DAsync(s->S.rep_acc + RA_F2, RA_STRIDE * sizeof(double), 0, sizeof(double), s->R, s->stream));
  return CTBOP_OK;
}

// ------------------------------------------------------------- evaluation
static double cg_tol(const ctbop_system* s) {
  if (s->o.cg_tol > 0) return s->o.cg_tol;
  return s->mixed ? 1e-5 : 1e-11;
}

template <class Rr>
static void enqueue_front(ctbop_system* s, const PotParams<Rr>& P, cudaStream_t st, bool md, double dt) {
  DevState& S = s->S;
  if (md) launch_kick_drift<Rr>(S, s->T, dt, 0.25 * s->o.skin * s->o.skin, st);
  launch_zero_acc(S, st);
  launch_rebuild<Rr>(S, P, st);
}

template <class Rr>
static void enqueue_middle(ctbop_system* s, const PotParams<Rr>& P, cudaStream_t st) {
  DevState& S = s->S;
  launch_bond<Rr>(S, P, st);
  launch_assemble<Rr>(S, P, s->T, st);
  if (S.precond) launch_block_setup<Rr>(S, st);
  launch_cg_begin<Rr>(S, s->T, st, cg_tol(s));
}

template <class Rr>
static void enqueue_back(ctbop_system* s, const PotParams<Rr>& P, cudaStream_t st, bool md, double dt,
                         bool solve) {
  DevState& S = s->S;
  if (solve) launch_cg_end<Rr>(S, st);
  launch_forces<Rr>(S, P, s->T, md ? 1 : 0, 0.5 * dt, st, !md);
  if (md && s->nvt) launch_nh_end(S, dt, st);
}

template <class Rr>
static int capture_graph(ctbop_system* s, const PotParams<Rr>& P, bool md, double dt, cudaGraphExec_t* out) {
  cudaStream_t cs = s->stream;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  enqueue_front<Rr>(s, P, cs, md, dt);
  enqueue_middle<Rr>(s, P, cs);
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg_graph;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg_graph, &deps, nullptr, &ndeps);
  cudaGraphConditionalHandle handle;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, cg_graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, cg_graph, deps, nullptr, ndeps, &cp);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      SolveCfg cfg{cg_tol(s), s->o.cg_max_iter, 1, handle};
      launch_cg_iter<Rr>(s->S, cfg, s->body_stream);
      e = cudaStreamEndCapture(s->body_stream, &body);
    }
  }
  enqueue_back<Rr>(s, P, cs, md, dt, true);
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(s, CTBOP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  if (e2 != cudaSuccess) return fail(s, CTBOP_ERR_CUDA, std::string("graph capture end: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(s, CTBOP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return CTBOP_OK;
}

// Host-driven variant of the same sequence (no graph): the CG loop polls the
// device's active flag every few iterations.
template <class Rr>
static int run_direct(ctbop_system* s, const PotParams<Rr>& P, bool md, double dt, bool solve) {
  cudaStream_t st = s->stream;
  enqueue_front<Rr>(s, P, st, md, dt);
  if (solve) {
    enqueue_middle<Rr>(s, P, st);
    SolveCfg cfg{cg_tol(s), s->o.cg_max_iter, 0, 0};
    for (int it = 0; it < s->o.cg_max_iter + 4; it += 4) {
      for (int k = 0; k < 4; ++k) launch_cg_iter<Rr>(s->S, cfg, st);
      CK(cudaMemcpyAsync(s->h_int, s->S.cg_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*s->h_int == 0) break;
    }
  } else {
    launch_bond<Rr>(s->S, P, st);
  }
  enqueue_back<Rr>(s, P, st, md, dt, solve);
  CK(cudaGetLastError());
  return CTBOP_OK;
}

static int read_err(ctbop_system* s, unsigned& bits) {
  CK(cudaStreamSynchronize(s->stream));
  CK(sync_copy(s, &bits, s->S.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  return CTBOP_OK;
}

// Build the lists for the current positions. The first build of a layout
// measures the entry counts and sizes the lists from them; an overflow grows
// them and builds again.
static int ensure_lists(ctbop_system* s) {
  DevState& S = s->S;
  int one = 1;
  if (!s->caps_known) {
    int cc = s->o.cap_cov > 0 ? s->o.cap_cov : 32;
    int ca = s->o.cap_all > 0 ? s->o.cap_all : 64;
    int rc = alloc_lists(s, cc, std::max(ca, cc));
    if (rc) return rc;
  }
  for (int attempt = 0;; ++attempt) {
    if (attempt > 4) return fail(s, CTBOP_ERR_NEIGH_OVERFLOW, "could not size the neighbour lists");
    CK(cudaMemcpyAsync(S.flag_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemsetAsync(S.err, 0, sizeof(unsigned), s->stream));
    if (s->mixed) launch_rebuild<float>(S, s->Pf, s->stream);
    else launch_rebuild<double>(S, s->Pd, s->stream);
    CK(cudaGetLastError());
    unsigned bits = 0;
    int rc = read_err(s, bits);
    if (rc) return rc;
    int mc[3];
    CK(sync_copy(s, mc, S.maxcnt, sizeof(mc), cudaMemcpyDeviceToHost));
    if (bits & CT_ERR_NONFINITE) return fail(s, CTBOP_ERR_NONFINITE, "non-finite position");
    bool over = (bits & (CT_ERR_NBR_OVERFLOW | CT_ERR_COV_OVERFLOW)) != 0;
    if (!over && (bits & CT_ERR_REV_MISSING)) return fail(s, CTBOP_ERR_CUDA, "internal: asymmetric covalent list");
    if (!over && s->caps_known) break;
    // size from the measured maxima with headroom for motion (a list holds
    // cap_cov covalent slots, then the rest)
    int cc = std::max(mc[0] + mc[0] / 4 + 4, 8);
    cc = (cc + 3) & ~3;
    int ca = cc + mc[1] + mc[1] / 8 + 16;
    cc = (cc + 3) & ~3;
    ca = (ca + 7) & ~7;
    if (s->o.cap_cov > 0) cc = std::max(cc, s->o.cap_cov);
    if (s->o.cap_all > 0) ca = std::max(ca, s->o.cap_all);
    if (over) {
      cc = std::max(cc, S.cap_cov);
      ca = std::max(ca, S.cap_all);
    }
    cc = (cc + 3) & ~3;
    ca = (std::max(ca, cc) + 7) & ~7;
    bool same = (cc == S.cap_cov && ca == S.cap_all);
    s->caps_known = true;
    if (same && !over) break;
    rc = alloc_lists(s, cc, ca);   // fresh buffers: build again
    if (rc) return rc;
  }
  s->need_rebuild = false;
  CK(cudaMemsetAsync(S.err, 0, sizeof(unsigned), s->stream));
  // the matrix pass's depth for these lists (CTBOP_MV_BATCH = 4, 8 or 16
  // forces one): chosen by timing on the first solve's assembled matrix
  if (S.N > 0 && (s->tuned_N != S.N || s->tuned_cap != S.cap_all)) {
    int before = S.mv_batch;
    const char* fb = getenv("CTBOP_MV_BATCH");
    int forced = fb ? atoi(fb) : 0;
    if (forced == 4 || forced == 8 || forced == 16) S.mv_batch = forced;
    else s->tune_pending = true;
    // the gather's depth likewise (CTBOP_GATHER_BATCH = 4, 6 or 8 forces one)
    const char* gbv = getenv("CTBOP_GATHER_BATCH");
    int gforced = gbv ? atoi(gbv) : 0;
    s->gather_forced = gforced == 4 || gforced == 6 || gforced == 8;
    if (s->gather_forced && S.gather_batch != gforced) {
      S.gather_batch = gforced;
      destroy_graphs(s);
    }
    // and the covalent passes' lanes per atom (CTBOP_COV_LANES = 4, 8 or 16)
    const char* clv = getenv("CTBOP_COV_LANES");
    int cforced = clv ? atoi(clv) : 0;
    s->cov_forced = (cforced == 4 && (S.cov_lanes_ok & 1)) || (cforced == 8 && (S.cov_lanes_ok & 2)) || cforced == 16;
    if (s->cov_forced && S.cov_lanes != cforced) {
      S.cov_lanes = cforced;
      destroy_graphs(s);
    }
    // the list build's shape (CTBOP_BUILD_SHAPE = "warps,batch" forces one),
    // timed here on the lists just built
    const char* bsv = getenv("CTBOP_BUILD_SHAPE");
    int bw = 0, bb = 0, bforced = -1;
    if (bsv && sscanf(bsv, "%d,%d", &bw, &bb) == 2) bforced = build_shape_index(bw, bb);
    int before_b = S.build_shape;
    if (bforced >= 0) {
      S.build_shape = bforced;
    } else {
      cudaError_t e = s->mixed ? tune_build<float>(S, s->Pf, S.flag_one, s->stream, s->build_ms)
                               : tune_build<double>(S, s->Pd, S.flag_one, s->stream, s->build_ms);
      if (e != cudaSuccess) return fail(s, CTBOP_ERR_CUDA, std::string("list-build tuning: ") + cudaGetErrorString(e));
    }
    s->tuned_N = S.N;
    s->tuned_cap = S.cap_all;
    if (S.mv_batch != before || S.build_shape != before_b) destroy_graphs(s);
  }
  return CTBOP_OK;
}

static int prepare(ctbop_system* s) {
  if (!s->have_layout || !s->have_box || !s->have_types || !s->have_pos)
    return fail(s, CTBOP_ERR_STATE, "layout, box, types and positions must be set first");
  int rc = alloc_atoms(s);
  if (rc) return rc;
  if (s->reps_dirty) {
    rc = setup_reps(s);
    if (rc) return rc;
  }
  if (s->need_rebuild || !s->caps_known) {
    rc = ensure_lists(s);
    if (rc) return rc;
  }
  return CTBOP_OK;
}

template <class Rr>
static int eval_t(ctbop_system* s, const PotParams<Rr>& P, uint32_t flags) {
  bool solve = !(flags & CTBOP_FIXED_CHARGES);
  if (solve && s->tune_pending) {
    // this evaluation runs directly; its assembled matrix then times the
    // matrix pass's depths (the solver state is kept across the timing)
    int rc = run_direct<Rr>(s, P, false, 0.0, true);
    if (rc) return rc;
    int before = s->S.mv_batch, before_asm = s->S.asm_batch, before_g = s->S.gather_batch;
    int before_c = s->S.cov_lanes;
    cudaError_t e = tune_cg_mv<Rr>(s->S, s->stream, s->mv_ms);
    if (e == cudaSuccess) e = tune_assemble<Rr>(s->S, P, s->T, s->stream, s->asm_ms);
    if (e == cudaSuccess && !s->cov_forced) e = tune_cov<Rr>(s->S, P, s->T, s->stream, s->cov_ms, true);
    if (e == cudaSuccess && !s->gather_forced) e = tune_gather<Rr>(s->S, P, s->T, s->stream, s->gather_ms);
    if (e != cudaSuccess) return fail(s, CTBOP_ERR_CUDA, std::string("pass tuning: ") + cudaGetErrorString(e));
    s->tune_pending = false;
    if (s->S.mv_batch != before || s->S.asm_batch != before_asm || s->S.gather_batch != before_g ||
        s->S.cov_lanes != before_c)
      destroy_graphs(s);
    s->solves++;
    s->have_forces = true;
    s->virial_stale = false;
    return CTBOP_OK;
  }
  if (s->use_graph && solve) {
    if (!s->g_eval) {
      int rc = capture_graph<Rr>(s, P, false, 0.0, &s->g_eval);
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(s->g_eval, s->stream));
  } else {
    int rc = run_direct<Rr>(s, P, false, 0.0, solve);
    if (rc) return rc;
  }
  if (solve) s->solves++;
  s->have_forces = true;
  s->virial_stale = false;
  return CTBOP_OK;
}

// The virial of the current state, after MD steps (whose force gather leaves
// it out: 15% of that pass at 1M atoms): the covalent slots and per-atom
// energies again, then the gather with the virial and no kick, which
// recomputes every replica sum from the same positions, charges and
// velocities.
template <class Rr>
static int refresh_virial(ctbop_system* s, const PotParams<Rr>& P) {
  DevState& S = s->S;
  launch_cov_force<Rr>(S, P, s->T, s->stream);
  CK(cudaMemsetAsync(S.rep_acc, 0, sizeof(double) * (size_t)s->R * RA_STRIDE, s->stream));
  launch_coul_gather<Rr>(S, P, s->T, 0, 0.0, s->stream, true);
  CK(cudaGetLastError());
  s->virial_stale = false;
  return CTBOP_OK;
}

namespace {
// A pair of timing events, destroyed on every return path.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    return e != cudaSuccess ? e : cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

template <class Rr>
static int profile_t(ctbop_system* s, const PotParams<Rr>& P, int64_t n, double dt, double* ms, int64_t* cnt) {
  cudaStream_t st = s->stream;
  DevState& S = s->S;
  EventPair ev;
  CK(ev.create());
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  auto timed = [&](int ph, int launches, auto&& fn) -> int {
    CK(cudaEventRecord(e0, st));
    fn();
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    ms[ph] += t;
    cnt[ph] += launches;
    return CTBOP_OK;
  };
  int rc = CTBOP_OK;
  SolveCfg cfg{cg_tol(s), s->o.cg_max_iter, 0, 0};
  for (int64_t k = 0; k < n && !rc; ++k) {
    CK(cudaMemsetAsync(S.err, 0, sizeof(unsigned), st));
    rc = timed(0, 1, [&] { launch_kick_drift<Rr>(S, s->T, dt, 0.25 * s->o.skin * s->o.skin, st); });
    if (!rc) rc = timed(1, 12, [&] { launch_zero_acc(S, st); launch_rebuild<Rr>(S, P, st); });
    if (!rc) rc = timed(2, sizeof(Rr) == 4 ? 3 : 1, [&] { launch_bond<Rr>(S, P, st); });
    if (!rc) rc = timed(3, 1, [&] { launch_assemble<Rr>(S, P, s->T, st); });
    if (!rc) rc = timed(4, S.precond ? 5 : 3, [&] {
      if (S.precond) launch_block_setup<Rr>(S, st);
      launch_cg_begin<Rr>(S, s->T, st, cg_tol(s));
    });
    for (int it = 0; it < s->o.cg_max_iter && !rc; ++it) {
      CK(cudaMemcpyAsync(s->h_int, S.cg_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*s->h_int == 0) break;
      rc = timed(5, 1, [&] { launch_cg_mv<Rr>(S, st); });
      if (!rc) rc = timed(6, 1, [&] { launch_cg_up<Rr>(S, cfg, st); });
    }
    if (!rc) rc = timed(7, 2, [&] { launch_cg_end<Rr>(S, st); });
    if (!rc) rc = timed(8, sizeof(Rr) == 4 ? 3 : 1, [&] { launch_cov_force<Rr>(S, P, s->T, st); });
    if (!rc) rc = timed(9, s->nvt ? 2 : 1, [&] {
      launch_coul_gather<Rr>(S, P, s->T, 1, 0.5 * dt, st, false);
      if (s->nvt) launch_nh_end(S, dt, st);
    });
    if (!rc) {
      unsigned bits = 0;
      rc = read_err(s, bits);
      if (!rc && (bits & (CT_ERR_NBR_OVERFLOW | CT_ERR_COV_OVERFLOW)))
        rc = fail(s, CTBOP_ERR_NEIGH_OVERFLOW, "neighbour lists overflowed during profiling; run ctbop_step first");
      if (!rc && (bits & CT_ERR_NONFINITE)) rc = fail(s, CTBOP_ERR_NONFINITE, "non-finite energy, force or position");
    }
    s->steps++;
    s->solves++;
    s->virial_stale = true;
  }
  return rc;
}

// ------------------------------------------------------------- C ABI
extern "C" {

int ctbop_default_options(ctbop_options* o) {
  if (!o) return CTBOP_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->precision = CTBOP_PREC_MIXED;
  o->cg_max_iter = 200;
  o->cg_tol = 0.0;
  o->skin = 0.3;
  o->device = 0;
  return CTBOP_OK;
}

int ctbop_create(const ctbop_params* p, const ctbop_options* o, ctbop_system** out) {
  if (!p || !o || !out) return CTBOP_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  if (!params_valid(p, why)) return CTBOP_ERR_INVALID_ARG;
  if (o->precision != CTBOP_PREC_FP64 && o->precision != CTBOP_PREC_MIXED) return CTBOP_ERR_INVALID_ARG;
  if (o->precond != CTBOP_PRECOND_BLOCK && o->precond != CTBOP_PRECOND_JACOBI) return CTBOP_ERR_INVALID_ARG;
  if (!(o->skin >= 0) || o->cg_max_iter < 1) return CTBOP_ERR_INVALID_ARG;
  if (cudaSetDevice(o->device) != cudaSuccess) return CTBOP_ERR_CUDA;
  ctbop_system* s = new ctbop_system();
  s->p = *p;
  s->o = *o;
  s->mixed = o->precision == CTBOP_PREC_MIXED;
  s->S.precond = o->precond == CTBOP_PRECOND_BLOCK ? 1 : 0;
  pack_params<float>(*p, o->skin, s->Pf);
  pack_params<double>(*p, o->skin, s->Pd);
  s->S.Pd = &s->Pd;
  for (int t = 0; t < 2; ++t) {
    s->T.E0[t] = p->E0[t];
    s->T.chi[t] = p->chi[t];
    s->T.J[t] = p->J[t];
    s->T.mass[t] = p->mass[t] / kAcc;          // KE = 1/2 m v^2 in eV with v in A/fs
    s->T.inv_mass_acc[t] = kAcc / p->mass[t];
  }
  double smax = 0;
  for (int k = 0; k < 4; ++k) smax = std::max(smax, p->S[k]);
  s->rlist = std::max(p->r_coul, smax) + o->skin;
  const char* ng = getenv("CTBOP_NO_GRAPH");
  s->use_graph = !(ng && ng[0] == '1');
  int dev = 0;
  cudaDeviceProp prop;
  cudaGetDevice(&dev);
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) s->S.nsm = prop.multiProcessorCount;
  if (cudaStreamCreate(&s->own_stream) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->body_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&s->h_int, 64) != cudaSuccess) {
    if (s->body_stream) cudaStreamDestroy(s->body_stream);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
    return CTBOP_ERR_CUDA;
  }
  s->stream = s->own_stream;
  {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    if (cudaMemPoolCreate(&s->pool, &pp) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      s->pool = nullptr;   // the default pool then
      cudaGetLastError();
    }
  }
  {
    std::string why;
    if (noalloc_setup(&s->noalloc_scratch, why)) {
      if (s->pool) cudaMemPoolDestroy(s->pool);
      cudaFreeHost(s->h_int);
      cudaStreamDestroy(s->body_stream);
      cudaStreamDestroy(s->own_stream);
      delete s;
      return CTBOP_ERR_CUDA;
    }
  }
  *out = s;
  return CTBOP_OK;
}

int ctbop_set_thermostat(ctbop_system* s, const double* T0, const double* tau) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  if (T0 && !tau) return fail(s, CTBOP_ERR_INVALID_ARG, "tau needed with T0");
  cudaSetDevice(s->o.device);
  DevState& S = s->S;
  const int R = s->R;
  std::vector<uint8_t> fr(S.N);
  if (S.N) CK(sync_copy(s, fr.data(), S.frozen, S.N, cudaMemcpyDeviceToHost));
  std::vector<double> h((size_t)R * NH_STRIDE, 0.0);
  bool any = false;
  for (int r = 0; r < R; ++r) {
    if (!T0 || !(T0[r] > 0)) continue;
    if (!(tau[r] > 0) || !std::isfinite(tau[r]) || !std::isfinite(T0[r]))
      return fail(s, CTBOP_ERR_INVALID_ARG, "thermostat needs T0 > 0 and tau > 0");
    int64_t mobile = 0;
    bool any_frozen = false;
    for (int64_t i = s->off[r]; i < s->off[r + 1]; ++i) {
      if (fr[i]) any_frozen = true; else ++mobile;
    }
    double g = 3.0 * mobile - (any_frozen ? 0.0 : 3.0);
    if (g <= 0) continue;   // nothing to thermostat
    double gkT = g * kKB * T0[r], Qm = gkT * tau[r] * tau[r];
    double* row = h.data() + (size_t)r * NH_STRIDE;
    row[NH_ON] = 1.0;
    row[NH_GKT] = gkT;
    row[NH_QM] = Qm;
    row[NH_QINV] = 1.0 / Qm;
    any = true;
  }
  CK(sync_copy(s, S.nh, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
  if (any != s->nvt) destroy_graphs(s);   // the step graph holds the end-of-step update or not
  s->nvt = any;
  return CTBOP_OK;
}

int ctbop_set_params(ctbop_system* s, const ctbop_params* p) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!p) return fail(s, CTBOP_ERR_INVALID_ARG, "null params");
  std::string why;
  if (!params_valid(p, why)) return fail(s, CTBOP_ERR_INVALID_ARG, why);
  cudaSetDevice(s->o.device);
  CK(cudaStreamSynchronize(s->stream));
  s->p = *p;
  pack_params<float>(*p, s->o.skin, s->Pf);
  pack_params<double>(*p, s->o.skin, s->Pd);
  for (int t = 0; t < 2; ++t) {
    s->T.E0[t] = p->E0[t];
    s->T.chi[t] = p->chi[t];
    s->T.J[t] = p->J[t];
    s->T.mass[t] = p->mass[t] / kAcc;
    s->T.inv_mass_acc[t] = kAcc / p->mass[t];
  }
  double smax = 0;
  for (int k = 0; k < 4; ++k) smax = std::max(smax, p->S[k]);
  double rl = std::max(p->r_coul, smax) + s->o.skin;
  if (rl != s->rlist) {
    s->rlist = rl;
    s->reps_dirty = true;   // cell grids depend on the list radius
  }
  destroy_graphs(s);        // the graphs hold the old parameters
  if (s->loo) {             // so does the screening's batch system
    ctbop_destroy(s->loo);
    s->loo = nullptr;
  }
  s->need_rebuild = true;
  s->have_forces = false;
  return reset_precision_mode(s);
}

int ctbop_destroy(ctbop_system* s) {
  if (!s) return CTBOP_OK;
  cudaSetDevice(s->o.device);
  cudaStreamSynchronize(s->stream);
  if (s->loo) ctbop_destroy(s->loo);
  if (s->d_order) cudaFree(s->d_order);
  destroy_graphs(s);
  s->atom_buf.release();
  s->list_buf.release();
  s->cell_buf.release();
  s->rep_buf.release();
  if (s->body_stream) cudaStreamDestroy(s->body_stream);
  if (s->own_stream) cudaStreamDestroy(s->own_stream);
  if (s->h_int) cudaFreeHost(s->h_int);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return CTBOP_OK;
}

const char* ctbop_last_error(const ctbop_system* s) { return s ? s->err.c_str() : "null system"; }

int ctbop_set_stream(ctbop_system* s, void* stream) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  // a graph cannot be captured on the legacy default stream: null selects
  // the library's own stream, which synchronises with the legacy stream
  cudaSetDevice(s->o.device);
  CK(cudaStreamSynchronize(s->stream));
  s->stream = stream ? (cudaStream_t)stream : s->own_stream;
  return CTBOP_OK;
}

int ctbop_set_layout(ctbop_system* s, int32_t n_replicas, const int64_t* atom_offsets) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (n_replicas < 1 || !atom_offsets) return fail(s, CTBOP_ERR_INVALID_ARG, "need n_replicas >= 1 and offsets");
  if (atom_offsets[0] != 0) return fail(s, CTBOP_ERR_INVALID_ARG, "atom_offsets[0] must be 0");
  for (int r = 0; r < n_replicas; ++r)
    if (atom_offsets[r + 1] < atom_offsets[r]) return fail(s, CTBOP_ERR_INVALID_ARG, "atom_offsets must not decrease");
  if (atom_offsets[n_replicas] > (int64_t)INT32_MAX / 64) return fail(s, CTBOP_ERR_INVALID_ARG, "too many atoms");
  cudaSetDevice(s->o.device);
  s->R = n_replicas;
  s->off.assign(atom_offsets, atom_offsets + n_replicas + 1);
  s->Q.assign(n_replicas, 0.0);
  s->box.assign(3 * n_replicas, 0.0);
  s->pbc.assign(3 * n_replicas, 0);
  s->have_layout = true;
  s->have_box = s->have_types = s->have_pos = false;
  s->ordered = false;
  s->order.clear();
  s->slot.clear();
  s->need_rebuild = true;
  s->reps_dirty = true;
  s->alloc_N = -1;
  return alloc_atoms(s);
}

int ctbop_set_box(ctbop_system* s, const double* h, const uint8_t* pbc) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  if (!h || !pbc) return fail(s, CTBOP_ERR_INVALID_ARG, "null box or pbc");
  for (int r = 0; r < s->R; ++r) {
    const double* m = h + 9 * r;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (a != b && m[3 * a + b] != 0.0)
          return fail(s, CTBOP_ERR_INVALID_ARG, "only orthorhombic (diagonal) cells are supported");
    for (int d = 0; d < 3; ++d) {
      double L = m[4 * d];
      if (!(L > 0) || !std::isfinite(L)) return fail(s, CTBOP_ERR_INVALID_ARG, "box edges must be positive");
      s->box[3 * r + d] = L;
      s->pbc[3 * r + d] = pbc[3 * r + d] ? 1 : 0;
    }
  }
  destroy_graphs(s);
  s->have_box = true;
  s->reps_dirty = true;
  s->need_rebuild = true;
  return reset_precision_mode(s);
}

static int copy_in(ctbop_system* s, void* dst, const void* src, size_t bytes, int mem) {
  if (!src && bytes) return fail(s, CTBOP_ERR_INVALID_ARG, "null input pointer");
  if (mem != CTBOP_HOST && mem != CTBOP_DEVICE) return fail(s, CTBOP_ERR_INVALID_ARG, "mem must be CTBOP_HOST or CTBOP_DEVICE");
  cudaSetDevice(s->o.device);
  if (mem == CTBOP_HOST) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s->stream));
  }
  return CTBOP_OK;
}

// A per-atom input (caller order) into a storage-order device array.
static int copy_in_atoms(ctbop_system* s, void* dst, const void* src, int elem_bytes, int mem) {
  size_t bytes = (size_t)elem_bytes * s->S.N;
  if (!s->ordered) return copy_in(s, dst, src, bytes, mem);
  if (!src && bytes) return fail(s, CTBOP_ERR_INVALID_ARG, "null input pointer");
  if (mem != CTBOP_HOST && mem != CTBOP_DEVICE) return fail(s, CTBOP_ERR_INVALID_ARG, "mem must be CTBOP_HOST or CTBOP_DEVICE");
  cudaSetDevice(s->o.device);
  void* tmp = s->S.stage;   // N x 24 bytes: the largest element
  CK(cudaMemcpyAsync(tmp, src, bytes, mem == CTBOP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     s->stream));
  CK(launch_permute(s->S.N, s->d_order, tmp, dst, elem_bytes, true, s->stream));
  if (mem == CTBOP_HOST) CK(cudaStreamSynchronize(s->stream));
  return CTBOP_OK;
}

int ctbop_set_order(ctbop_system* s, const int64_t* order) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  if (s->have_types || s->have_pos) return fail(s, CTBOP_ERR_STATE, "set the order before the per-atom arrays");
  cudaSetDevice(s->o.device);
  const int64_t N = s->S.N;
  if (!order) {
    s->ordered = false;
    s->order.clear();
    s->slot.clear();
    return CTBOP_OK;
  }
  std::vector<int64_t> slot(N, -1);
  bool ident = true;
  for (int r = 0; r < s->R; ++r)
    for (int64_t k = s->off[r]; k < s->off[r + 1]; ++k) {
      int64_t a = order[k];
      if (a < s->off[r] || a >= s->off[r + 1] || slot[a] >= 0)
        return fail(s, CTBOP_ERR_INVALID_ARG, "order must permute the atoms within each replica");
      slot[a] = k;
      ident = ident && a == k;
    }
  if (ident) {
    s->ordered = false;
    s->order.clear();
    s->slot.clear();
    return CTBOP_OK;
  }
  std::vector<int> o32(order, order + N);
  if (s->d_order) cudaFree(s->d_order);
  s->d_order = nullptr;
  CK(cudaMalloc(&s->d_order, sizeof(int) * std::max<int64_t>(N, 1)));
  CK(sync_copy(s, s->d_order, o32.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
  s->order.assign(order, order + N);
  s->slot = std::move(slot);
  s->ordered = true;
  return CTBOP_OK;
}

int ctbop_set_types(ctbop_system* s, const int32_t* types, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  size_t N = s->S.N;
  if (mem == CTBOP_HOST && types)
    for (size_t i = 0; i < N; ++i)
      if (types[i] != 0 && types[i] != 1) return fail(s, CTBOP_ERR_INVALID_ARG, "types must be 0 (Si) or 1 (C)");
  int rc = copy_in_atoms(s, s->S.type, types, sizeof(int), mem);
  if (rc) return rc;
  s->have_types = true;
  s->need_rebuild = true;
  return reset_precision_mode(s);
}

int ctbop_set_positions(ctbop_system* s, const double* x, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  int rc = copy_in_atoms(s, s->S.x, x, 3 * sizeof(double), mem);
  if (rc) return rc;
  // new positions break the time series the CG start extrapolates: keep
  // only the last solution as the starting guess
  *s->h_int = s->solves > 0 ? 1 : 0;
  CK(cudaMemcpyAsync(s->S.cg_hist, s->h_int, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->have_pos = true;
  s->need_rebuild = true;
  s->have_forces = false;
  return reset_precision_mode(s);
}

int ctbop_set_velocities(ctbop_system* s, const double* v, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  return copy_in_atoms(s, s->S.v, v, 3 * sizeof(double), mem);
}

int ctbop_set_charges(ctbop_system* s, const double* q, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  int rc = copy_in_atoms(s, s->S.q, q, sizeof(double), mem);
  if (rc) return rc;
  if (s->mixed) launch_copy_q<float>(s->S, s->stream);
  else launch_copy_q<double>(s->S, s->stream);
  CK(cudaGetLastError());
  return CTBOP_OK;
}

int ctbop_set_frozen(ctbop_system* s, const uint8_t* frozen, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  return copy_in_atoms(s, s->S.frozen, frozen, 1, mem);
}

int ctbop_set_total_charge(ctbop_system* s, const double* Q) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "set_layout first");
  if (!Q) return fail(s, CTBOP_ERR_INVALID_ARG, "null Q");
  for (int r = 0; r < s->R; ++r) {
    if (!std::isfinite(Q[r])) return fail(s, CTBOP_ERR_INVALID_ARG, "Q must be finite");
    s->Q[r] = Q[r];
  }
  s->reps_dirty = true;
  return CTBOP_OK;
}

int ctbop_compute(ctbop_system* s, uint32_t flags) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  cudaSetDevice(s->o.device);
  int rc = prepare(s);
  if (rc) return rc;
  rc = s->mixed ? eval_t<float>(s, s->Pf, flags) : eval_t<double>(s, s->Pd, flags);
  if (rc) return rc;
  CK(cudaGetLastError());
  return CTBOP_OK;
}

int ctbop_step(ctbop_system* s, int64_t n_steps, double dt_fs) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (n_steps < 0 || !(dt_fs > 0) || !std::isfinite(dt_fs)) return fail(s, CTBOP_ERR_INVALID_ARG, "need n_steps >= 0, dt > 0");
  cudaSetDevice(s->o.device);
  int rc = prepare(s);
  if (rc) return rc;
  if (!s->have_forces) {
    rc = ctbop_compute(s, 0);
    if (rc) return rc;
  }
  DevState& S = s->S;
  const int64_t chunk = 100;
  // snapshot buffers for redoing a chunk after a list overflow
  double *sx = s->snap_x, *sv = s->snap_v, *sF = s->snap_F, *sq = s->snap_q;
  size_t N = S.N;
  int result = CTBOP_OK;
  int64_t done = 0;
  int redo = 0;
  while (done < n_steps) {
    int64_t n = std::min(chunk, n_steps - done);
    cudaMemcpyAsync(sx, S.x, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(sv, S.v, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(sF, S.F, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(sq, S.q, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemsetAsync(S.err, 0, sizeof(unsigned), s->stream);
    if (s->use_graph) {
      if (!s->g_step || s->g_step_dt != dt_fs) {
        if (s->g_step) cudaGraphExecDestroy(s->g_step);
        s->g_step = nullptr;
        result = s->mixed ? capture_graph<float>(s, s->Pf, true, dt_fs, &s->g_step)
                          : capture_graph<double>(s, s->Pd, true, dt_fs, &s->g_step);
        if (result) break;
        s->g_step_dt = dt_fs;
      }
      for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = cudaGraphLaunch(s->g_step, s->stream);
        if (e != cudaSuccess) { result = fail(s, CTBOP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e)); break; }
      }
      if (result) break;
    } else {
      for (int64_t k = 0; k < n && !result; ++k)
        result = s->mixed ? run_direct<float>(s, s->Pf, true, dt_fs, true)
                          : run_direct<double>(s, s->Pd, true, dt_fs, true);
      if (result) break;
    }
    unsigned bits = 0;
    result = read_err(s, bits);
    if (result) break;
    if (bits & (CT_ERR_NBR_OVERFLOW | CT_ERR_COV_OVERFLOW)) {
      if (++redo > 3) { result = fail(s, CTBOP_ERR_NEIGH_OVERFLOW, "neighbour lists kept overflowing"); break; }
      // restore the chunk's starting state, grow the lists, redo the chunk
      cudaMemcpyAsync(S.x, sx, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
      cudaMemcpyAsync(S.v, sv, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
      cudaMemcpyAsync(S.F, sF, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s->stream);
      cudaMemcpyAsync(S.q, sq, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->stream);
      // the restored q is the next starting guess; its time history is gone
      *s->h_int = 1;
      cudaMemcpyAsync(S.cg_hist, s->h_int, sizeof(int), cudaMemcpyHostToDevice, s->stream);
      int mc[3];
      sync_copy(s, mc, S.maxcnt, sizeof(mc), cudaMemcpyDeviceToHost);
      int cc = (std::max(S.cap_cov, mc[0] + mc[0] / 4 + 4) + 3) & ~3;
      int ca = std::max(S.cap_all, cc + mc[1] + mc[1] / 8 + 16);
      result = alloc_lists(s, cc, (ca + 7) & ~7);
      if (result) break;
      s->need_rebuild = true;
      result = ensure_lists(s);
      if (result) break;
      // recompute forces at the restored positions with the new lists
      result = ctbop_compute(s, 0);
      if (result) break;
      continue;
    }
    if (bits & CT_ERR_NONFINITE) { result = fail(s, CTBOP_ERR_NONFINITE, "non-finite energy, force or position"); done += n; break; }
    if (bits & CT_ERR_REV_MISSING) { result = fail(s, CTBOP_ERR_CUDA, "internal: asymmetric covalent list"); break; }
    done += n;
    s->steps += n;
    s->solves += n;
    if (n > 0) s->virial_stale = true;
    if (bits & CT_ERR_CG_MAXITER) { result = fail(s, CTBOP_ERR_CG_NOT_CONVERGED, "charge CG reached max_iter"); break; }
  }
  cudaStreamSynchronize(s->stream);
  return result;
}

int ctbop_get(ctbop_system* s, int what, void* dst, int mem) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!dst) return fail(s, CTBOP_ERR_INVALID_ARG, "null destination");
  if (mem != CTBOP_HOST && mem != CTBOP_DEVICE) return fail(s, CTBOP_ERR_INVALID_ARG, "mem must be CTBOP_HOST or CTBOP_DEVICE");
  if (!s->have_layout) return fail(s, CTBOP_ERR_STATE, "nothing computed");
  cudaSetDevice(s->o.device);
  DevState& S = s->S;
  cudaMemcpyKind kind = mem == CTBOP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  size_t N = S.N, R = s->R;
  if (what == CTBOP_GET_VIRIAL && s->virial_stale && s->have_forces) {
    int rc = s->mixed ? refresh_virial<float>(s, s->Pf) : refresh_virial<double>(s, s->Pd);
    if (rc) return rc;
  }
  if (what == CTBOP_GET_COORDINATION) {
    // computed from the current lists, which an evaluation leaves valid
    if (!s->have_forces) return fail(s, CTBOP_ERR_STATE, "coordination: compute or step first");
    if (N == 0) return CTBOP_OK;
    Scratch scr(s->stream, s->pool);
    double* tmp = nullptr;
    CK(scr.alloc(&tmp, N));
    if (s->mixed) launch_coordination<float>(S, s->Pf, tmp, s->stream);
    else launch_coordination<double>(S, s->Pd, tmp, s->stream);
    CK(cudaGetLastError());
    if (s->ordered) {
      double* tmp2 = nullptr;
      CK(scr.alloc(&tmp2, N));
      CK(launch_permute((int)N, s->d_order, tmp, tmp2, 8, false, s->stream));
      tmp = tmp2;
    }
    CK(cudaMemcpyAsync(dst, tmp, sizeof(double) * N, kind, s->stream));
    if (mem == CTBOP_HOST) CK(cudaStreamSynchronize(s->stream));
    return CTBOP_OK;
  }
  const void* src = nullptr;
  size_t width = 0, pitch = 0, rows = 1;
  switch (what) {
    case CTBOP_GET_ENERGY: src = S.rep_acc + RA_E; width = 8; pitch = RA_STRIDE * 8; rows = R; break;
    case CTBOP_GET_VIRIAL: src = S.rep_acc + RA_W; width = 72; pitch = RA_STRIDE * 8; rows = R; break;
    case CTBOP_GET_KINETIC: src = S.rep_acc + RA_KE; width = 8; pitch = RA_STRIDE * 8; rows = R; break;
    case CTBOP_GET_MU: src = S.cg + CG_MU; width = 8; pitch = CG_STRIDE * 8; rows = R; break;
    case CTBOP_GET_FORCES: src = S.F; width = pitch = 24 * N; break;
    case CTBOP_GET_POSITIONS: src = S.x; width = pitch = 24 * N; break;
    case CTBOP_GET_VELOCITIES: src = S.v; width = pitch = 24 * N; break;
    case CTBOP_GET_CHARGES: src = S.q; width = pitch = 8 * N; break;
    case CTBOP_GET_E_ATOM: src = S.e_atom; width = pitch = 8 * N; break;
    case CTBOP_GET_THERMOSTAT: src = S.nh + NH_XI; width = 32; pitch = NH_STRIDE * 8; rows = R; break;
    default: return fail(s, CTBOP_ERR_INVALID_ARG, "unknown selector");
  }
  if (width == 0) return CTBOP_OK;
  const bool per_atom = what == CTBOP_GET_FORCES || what == CTBOP_GET_POSITIONS || what == CTBOP_GET_VELOCITIES ||
                        what == CTBOP_GET_CHARGES || what == CTBOP_GET_E_ATOM;
  if (per_atom && s->ordered) {
    // back to the caller's order, through the staging buffer
    void* tmp = S.stage;
    CK(launch_permute((int)N, s->d_order, src, tmp, (int)(width / N), false, s->stream));
    CK(cudaMemcpyAsync(dst, tmp, width, kind, s->stream));
  } else if (rows == 1 || pitch == width) {
    CK(cudaMemcpyAsync(dst, src, width * rows, kind, s->stream));
  } else if (mem == CTBOP_HOST && width * rows <= 24 * N) {
    // strided per-replica sums: packed on the device first (a strided copy
    // straight to host memory took 0.2 ms for a few bytes), then one copy
    CK(cudaMemcpy2DAsync(S.stage, width, src, pitch, width, rows, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(dst, S.stage, width * rows, kind, s->stream));
  } else {
    CK(cudaMemcpy2DAsync(dst, width, src, pitch, width, rows, kind, s->stream));
  }
  if (mem == CTBOP_HOST) CK(cudaStreamSynchronize(s->stream));
  return CTBOP_OK;
}

int ctbop_profile_steps(ctbop_system* s, int64_t n_steps, double dt_fs, double* ms_out, int64_t* launches_out) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!ms_out || !launches_out || n_steps < 0 || !(dt_fs > 0)) return fail(s, CTBOP_ERR_INVALID_ARG, "bad profile arguments");
  cudaSetDevice(s->o.device);
  int rc = prepare(s);
  if (rc) return rc;
  if (!s->have_forces) {
    rc = ctbop_compute(s, 0);
    if (rc) return rc;
  }
  return s->mixed ? profile_t<float>(s, s->Pf, n_steps, dt_fs, ms_out, launches_out)
                  : profile_t<double>(s, s->Pd, n_steps, dt_fs, ms_out, launches_out);
}

int ctbop_status(ctbop_system* s, ctbop_stats* st) {
  if (!s || !st) return CTBOP_ERR_INVALID_ARG;
  cudaSetDevice(s->o.device);
  memset(st, 0, sizeof(*st));
  st->steps = s->steps;
  st->solves = s->solves;
  if (s->alloc_N < 0) return CTBOP_OK;
  DevState& S = s->S;
  CK(cudaStreamSynchronize(s->stream));
  unsigned bits = 0;
  long long rb = 0, tot = 0;
  int it = 0, mc[3] = {0, 0, 0};
  CK(sync_copy(s, &bits, S.err, sizeof(bits), cudaMemcpyDeviceToHost));
  CK(sync_copy(s, &rb, S.rebuild_count, sizeof(rb), cudaMemcpyDeviceToHost));
  CK(sync_copy(s, &tot, S.cg_total, sizeof(tot), cudaMemcpyDeviceToHost));
  CK(sync_copy(s, &it, S.cg_it, sizeof(it), cudaMemcpyDeviceToHost));
  CK(sync_copy(s, mc, S.maxcnt, sizeof(mc), cudaMemcpyDeviceToHost));
  double res = 0, res0 = 0;
  CK(sync_copy(s, &res, S.cg + CG_RESMAX, sizeof(double), cudaMemcpyDeviceToHost));
  CK(sync_copy(s, &res0, S.cg + CG_RES0, sizeof(double), cudaMemcpyDeviceToHost));
  st->cg_residual_start = res0;
  st->cg_mv_batch = S.mv_batch;
  for (int k = 0; k < 3; ++k) st->cg_mv_ms[k] = s->mv_ms[k];
  for (int k = 0; k < 3; ++k) st->asm_ms[k] = s->asm_ms[k];
  st->asm_batch = S.asm_batch;
  for (int k = 0; k < 3; ++k) st->gather_ms[k] = s->gather_ms[k];
  st->gather_batch = S.gather_batch;
  for (int k = 0; k < 3; ++k) st->cov_ms[k] = s->cov_ms[k];
  st->cov_lanes = S.cov_lanes;
  build_shape_of(S.build_shape, &st->build_warps, &st->build_batch);
  for (int k = 0; k < BUILD_SHAPES; ++k) st->build_ms[k] = s->build_ms[k];
  if (S.flag_n) CK(sync_copy(s, &st->fp64_atoms, S.flag_n, sizeof(int), cudaMemcpyDeviceToHost));
  if (S.stiff_n) CK(sync_copy(s, &st->fp64_bonds, S.stiff_n, sizeof(int), cudaMemcpyDeviceToHost));
  st->error_bits = bits;
  st->rebuilds = rb;
  st->cg_iters_total = tot;
  st->cg_iters_last = it;
  st->cg_residual_last = res;
  st->max_cov = mc[0];
  st->max_all = mc[2];
  if (S.N > 0 && S.ncov) {
    std::vector<int> a(S.N), b(S.N), c(S.N);
    CK(sync_copy(s, a.data(), S.ncov, sizeof(int) * S.N, cudaMemcpyDeviceToHost));
    CK(sync_copy(s, b.data(), S.nall, sizeof(int) * S.N, cudaMemcpyDeviceToHost));
    CK(sync_copy(s, c.data(), S.nmat, sizeof(int) * S.N, cudaMemcpyDeviceToHost));
    double sa = 0, sb = 0, sc = 0;
    for (int i = 0; i < S.N; ++i) { sa += a[i]; sb += b[i]; sc += c[i]; }
    st->mean_cov = sa / S.N;
    st->mean_all = sb / S.N;
    st->mean_mat = sc / S.N;
  }
  if (bits & CT_ERR_NONFINITE) return fail(s, CTBOP_ERR_NONFINITE, "non-finite energy, force or position");
  if (bits & CT_ERR_CG_MAXITER) return fail(s, CTBOP_ERR_CG_NOT_CONVERGED, "charge CG reached max_iter");
  return CTBOP_OK;
}

}  // extern "C"

// Force-matching gradient, in the system's precision policy. With g =
// dL/dF, the force part of dL/dtheta is -T1 + lambda . d(Hq + chi)/dtheta:
//   T1 = d/de dE/dtheta (x + e g) at the fixed minimiser charges, and
//   v  = d/de (H q + chi)(x + e g), both from one forward-mode pass of the
//        parameter-gradient kernels along g;
//   lambda solves the projected adjoint system H lambda = v (sum lambda = 0
//        per replica) with the charge solver;
//   lambda . d(Hq + chi)/dtheta = d/ds dE/dtheta (q + s lambda), a second
//        forward-mode pass, along the charges.
// No step sizes: both passes carry exact directional derivatives.
template <class Rr>
static int param_grad_impl(ctbop_system* s, const double* w_E, const double* E_ref, const double* w_F,
                           const double* F_ref, double* loss_out, double* dth) {
  DevState& S = s->S;
  cudaStream_t st = s->stream;
  const int N = S.N, R = s->R;
  const bool fp32 = sizeof(Rr) == 4;
  int rc = ctbop_compute(s, 0);
  if (rc) return rc;
  std::vector<double> E(R), F((size_t)3 * N);
  CK(cudaMemcpy2DAsync(E.data(), 8, S.rep_acc + RA_E, RA_STRIDE * 8, 8, R, cudaMemcpyDeviceToHost, st));
  CK(sync_copy(s, F.data(), S.F, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
  // loss and its derivatives with respect to E_r and F_i
  double loss = 0.0;
  std::vector<double> a(R, 0.0), g((size_t)3 * N, 0.0), one(R, 1.0);
  double gmax = 0.0;
  for (int r = 0; r < R; ++r) {
    if (w_E && E_ref) {
      double d = E[r] - E_ref[r];
      loss += w_E[r] * d * d;
      a[r] = 2.0 * w_E[r] * d;
    }
    if (w_F && F_ref)
      for (int64_t i = s->off[r]; i < s->off[r + 1]; ++i)
        for (int k = 0; k < 3; ++k) {
          double d = F[3 * i + k] - F_ref[3 * i + k];
          loss += w_F[r] * d * d;
          g[3 * i + k] = 2.0 * w_F[r] * d;
          gmax = std::max(gmax, std::fabs(g[3 * i + k]));
        }
  }
  *loss_out = loss;
  double *d_w = nullptr, *d_one = nullptr, *d_g = nullptr, *d_dir = nullptr, *d_v = nullptr, *d_cg = nullptr;
  double *d_h1 = nullptr, *d_h2 = nullptr, *d_q0 = nullptr, *d_lam = nullptr;
  Scratch scr(st, s->pool);
  if (scr.alloc(&d_w, R) || scr.alloc(&d_one, R) || scr.alloc(&d_g, 2 * PG_NPARAM) ||
      scr.alloc(&d_dir, (size_t)3 * N) || scr.alloc(&d_v, N) || scr.alloc(&d_cg, (size_t)R * CG_STRIDE) ||
      scr.alloc(&d_h1, N) || scr.alloc(&d_h2, N) || scr.alloc(&d_q0, N) || scr.alloc(&d_lam, N))
    return fail(s, CTBOP_ERR_OOM, "param_grad: temporary buffers");
  const ctbop_params& P = s->p;
  std::vector<double> G(2 * PG_NPARAM, 0.0), L(2 * PG_NPARAM, 0.0);
  CK(cudaMemcpyAsync(d_w, a.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_one, one.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  if (gmax == 0.0) {
    // energy part only: sum_r a_r dE_r/dtheta at the minimiser
    CK(launch_param_grad(S, P, fp32, d_w, nullptr, nullptr, nullptr, d_g, nullptr, st));
    CK(cudaMemcpyAsync(G.data(), d_g, sizeof(double) * 2 * PG_NPARAM, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else {
    // energy part, T1 and v in one forward-mode pass along g
    std::vector<double> v(N);
    CK(cudaMemcpyAsync(d_dir, g.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
    CK(launch_param_grad(S, P, fp32, d_w, d_one, d_dir, nullptr, d_g, d_v, st));
    CK(cudaMemcpyAsync(G.data(), d_g, sizeof(double) * 2 * PG_NPARAM, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(v.data(), d_v, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < PG_NPARAM; ++k) G[k] -= G[PG_NPARAM + k];
    // rhs of the solver's H q + chi = mu 1 form: chi := -v (the matrix at x
    // is the one the charge solve above assembled)
    double vmax = 0.0;
    for (int i = 0; i < N; ++i) {
      v[i] = -v[i];
      vmax = std::max(vmax, std::fabs(v[i]));
    }
    CK(cudaMemcpyAsync(d_v, v.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
    // keep the charges and the solver state: per-replica scalars, history
    CK(cudaMemcpyAsync(d_q0, S.q, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d_cg, S.cg, sizeof(double) * R * CG_STRIDE, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d_h1, S.cqh1, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d_h2, S.cqh2, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    int hist_saved = 0;
    CK(sync_copy(s, &hist_saved, S.cg_hist, sizeof(int), cudaMemcpyDeviceToHost));
    // the adjoint: zero total per replica, cold start
    std::vector<double> cgh((size_t)R * CG_STRIDE);
    CK(sync_copy(s, cgh.data(), S.cg, sizeof(double) * cgh.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < R; ++r) cgh[(size_t)r * CG_STRIDE + CG_Q] = 0.0;
    CK(sync_copy(s, S.cg, cgh.data(), sizeof(double) * cgh.size(), cudaMemcpyHostToDevice));
    int zero = 0;
    CK(sync_copy(s, S.cg_hist, &zero, sizeof(int), cudaMemcpyHostToDevice));
    // FP64: the charge solve's absolute tolerance. FP32: the charge solve's
    // relative reach (its tolerance over the electronegativity scale, about
    // 2e-6) applied to the size of this right-hand side.
    double tol = cg_tol(s);
    if (fp32 && s->o.cg_tol <= 0) tol = std::max(tol, 2e-6 * vmax);
    SolveCfg cfg{tol, s->o.cg_max_iter, 0, 0};
    launch_cg_begin<Rr>(S, s->T, st, cfg.tol, d_v);
    for (int it = 0; it < s->o.cg_max_iter + 4; it += 4) {
      for (int k = 0; k < 4; ++k) launch_cg_iter<Rr>(S, cfg, st);
      CK(cudaMemcpyAsync(s->h_int, S.cg_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*s->h_int == 0) break;
    }
    launch_cg_end<Rr>(S, st);
    unsigned bits = 0;
    rc = read_err(s, bits);
    if (!rc && (bits & CT_ERR_CG_MAXITER)) rc = fail(s, CTBOP_ERR_CG_NOT_CONVERGED, "param_grad: adjoint CG reached max_iter");
    // lambda out, the charges and the solver state back
    CK(cudaMemcpyAsync(d_lam, S.q, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(S.q, d_q0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    launch_copy_q<Rr>(S, st);
    CK(cudaMemcpyAsync(S.cg, d_cg, sizeof(double) * R * CG_STRIDE, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(S.cqh1, d_h1, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(S.cqh2, d_h2, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(S.cg_hist, &hist_saved, sizeof(int), cudaMemcpyHostToDevice, st));
    if (!rc) {
      // lambda . d(Hq + chi)/dtheta: forward mode along the charges
      CK(launch_param_grad(S, P, fp32, d_one, d_one, nullptr, d_lam, d_g, nullptr, st));
      CK(cudaMemcpyAsync(L.data(), d_g, sizeof(double) * 2 * PG_NPARAM, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    if (!rc)
      for (int k = 0; k < PG_NPARAM; ++k) G[k] += L[PG_NPARAM + k];
  }
  if (rc) return rc;
  G[PG_MASS] = G[PG_MASS + 1] = 0.0;   // the mass is not in E
  for (int k = 0; k < PG_NPARAM; ++k) dth[k] = G[k];
  return CTBOP_OK;
}

extern "C" {

int ctbop_param_grad(ctbop_system* s, const double* w_E, const double* E_ref, const double* w_F,
                     const double* F_ref, double* loss, ctbop_params* dtheta) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!loss || !dtheta) return fail(s, CTBOP_ERR_INVALID_ARG, "null loss or dtheta");
  if (!s->have_layout || !s->have_pos || !s->have_types)
    return fail(s, CTBOP_ERR_STATE, "set layout, box, types and positions first");
  cudaSetDevice(s->o.device);
  static_assert(sizeof(ctbop_params) == PG_NPARAM * sizeof(double), "ctbop_params is 144 doubles");
  static_assert(offsetof(ctbop_params, sigma) == PG_SIGMA * sizeof(double), "layout");
  static_assert(offsetof(ctbop_params, gamma) == PG_GAMMA * sizeof(double), "layout");
  static_assert(offsetof(ctbop_params, E0) == PG_E0 * sizeof(double), "layout");
  static_assert(offsetof(ctbop_params, k_e) == PG_KE * sizeof(double), "layout");
  double* out = reinterpret_cast<double*>(dtheta);
  std::vector<double> Fs;
  if (F_ref && s->ordered) {   // the targets in storage order
    Fs.resize((size_t)3 * s->S.N);
    for (int64_t k = 0; k < s->S.N; ++k)
      for (int d = 0; d < 3; ++d) Fs[3 * k + d] = F_ref[3 * s->order[k] + d];
    F_ref = Fs.data();
  }
  return s->mixed ? param_grad_impl<float>(s, w_E, E_ref, w_F, F_ref, loss, out)
                  : param_grad_impl<double>(s, w_E, E_ref, w_F, F_ref, loss, out);
}

int ctbop_energy_noalloc(ctbop_system* s, double* energy) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (!energy) return fail(s, CTBOP_ERR_INVALID_ARG, "null energy pointer");
  if (!s->have_forces || s->alloc_N < 0) return fail(s, CTBOP_ERR_STATE, "compute or step first");
  cudaSetDevice(s->o.device);
  std::string why;
  int rc = energy_noalloc(s->S.e_atom, s->S.rep, s->S.N, s->R, s->noalloc_scratch, s->stream, energy, why);
  if (rc == -1) return fail(s, CTBOP_ERR_INVALID_ARG, why);
  if (rc) return fail(s, CTBOP_ERR_CUDA, why);
  return CTBOP_OK;
}

// Removal energies of the desorption screening (Sec. 3.3). The systems
// without each candidate are evaluated as replicas of one batch system
// (s->loo, kept between calls): candidates are grouped by source replica, a
// chunk holds as many as fit in max_atoms, and a device gather builds each
// chunk from the current state. The batch's starting charges are the
// source's (the solver shifts them onto the replica total).
int ctbop_removal_energies(ctbop_system* s, int64_t n_cand, const int64_t* cand, int64_t max_atoms, double* dE) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (n_cand < 0 || (n_cand > 0 && (!cand || !dE))) return fail(s, CTBOP_ERR_INVALID_ARG, "bad candidate arrays");
  if (!s->have_layout || !s->have_box || !s->have_types || !s->have_pos)
    return fail(s, CTBOP_ERR_STATE, "layout, box, types and positions must be set first");
  cudaSetDevice(s->o.device);
  DevState& S = s->S;
  const int64_t N = S.N;
  for (int64_t c = 0; c < n_cand; ++c)
    if (cand[c] < 0 || cand[c] >= N) return fail(s, CTBOP_ERR_INVALID_ARG, "candidate index out of range");
  if (n_cand == 0) return CTBOP_OK;
  int rc = CTBOP_OK;
  if (!s->have_forces) {
    rc = ctbop_compute(s, 0);
    if (rc) return rc;
  }
  const int R = s->R;
  std::vector<double> E(R);
  std::vector<int> types(N);
  CK(cudaMemcpy2DAsync(E.data(), 8, S.rep_acc + RA_E, RA_STRIDE * 8, 8, R, cudaMemcpyDeviceToHost, s->stream));
  CK(sync_copy(s, types.data(), S.type, sizeof(int) * N, cudaMemcpyDeviceToHost));
  struct Job { int64_t c; int r; int n; int drop; };
  std::vector<Job> jobs;
  for (int64_t c = 0; c < n_cand; ++c) {
    int64_t k = s->ordered ? s->slot[cand[c]] : cand[c];   // storage slot
    int r = (int)(std::upper_bound(s->off.begin(), s->off.end(), k) - s->off.begin()) - 1;
    int n = (int)(s->off[r + 1] - s->off[r]);
    if (n == 1) dE[c] = s->T.E0[types[k]] - E[r];   // nothing remains: E = 0
    else jobs.push_back({c, r, n, (int)(k - s->off[r])});
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& b) { return a.r < b.r; });
  const int64_t budget = max_atoms > 0 ? max_atoms : ((int64_t)1 << 22);
  bool one_source = true;
  for (const Job& j : jobs) one_source = one_source && j.r == jobs[0].r;
  if (!s->loo && !jobs.empty()) {
    ctbop_options o2 = s->o;
    o2.cap_cov = o2.cap_all = 0;
    rc = ctbop_create(&s->p, &o2, &s->loo);
    if (rc) return fail(s, rc, "removal energies: batch system");
  }
  if (s->loo) {
    rc = ctbop_set_stream(s->loo, s->stream);
    if (rc) return fail(s, rc, "removal energies: " + s->loo->err);
  }
  ctbop_system* L = s->loo;
  double *d_x = nullptr, *d_q = nullptr;
  int* d_t = nullptr;
  uint8_t* d_f = nullptr;
  LooItem* d_items = nullptr;
  size_t cap_atoms = 0, cap_items = 0;
  std::unique_ptr<Scratch> scr;   // the chunk buffers; replaced when a chunk needs more
  size_t first_chunk = 0;
  for (size_t j0 = 0; j0 < jobs.size() && !rc;) {
    // the chunk: jobs [j0, j1), padded (single source) to the first chunk's size
    size_t j1 = j0;
    int64_t atoms = 0;
    while (j1 < jobs.size() && j1 - j0 < 65535 && (j1 == j0 || atoms + jobs[j1].n - 1 <= budget)) {
      atoms += jobs[j1].n - 1;
      ++j1;
    }
    if (j0 == 0) first_chunk = j1 - j0;
    std::vector<Job> chunk(jobs.begin() + j0, jobs.begin() + j1);
    while (one_source && chunk.size() < first_chunk) chunk.push_back(chunk.back());
    const int C = (int)chunk.size();
    std::vector<int64_t> off(C + 1, 0);
    std::vector<LooItem> items(C);
    std::vector<double> h((size_t)9 * C, 0.0), Q(C);
    std::vector<uint8_t> pbc((size_t)3 * C);
    int max_n = 0;
    for (int k = 0; k < C; ++k) {
      const Job& jb = chunk[k];
      off[k + 1] = off[k] + jb.n - 1;
      items[k] = {s->off[jb.r], jb.n, jb.drop, off[k]};
      for (int d = 0; d < 3; ++d) {
        h[9 * k + 4 * d] = s->box[3 * jb.r + d];
        pbc[3 * k + d] = s->pbc[3 * jb.r + d];
      }
      Q[k] = s->Q[jb.r];
      max_n = std::max(max_n, jb.n);
    }
    const size_t na = (size_t)off[C];
    if (na > cap_atoms || (size_t)C > cap_items) {
      cap_atoms = std::max(na, cap_atoms);
      cap_items = std::max((size_t)C, cap_items);
      scr.reset(new Scratch(s->stream));
      CK(scr->alloc(&d_x, 3 * cap_atoms));
      CK(scr->alloc(&d_q, cap_atoms));
      CK(scr->alloc(&d_t, cap_atoms));
      CK(scr->alloc(&d_f, cap_atoms));
      CK(scr->alloc(&d_items, cap_items));
    }
    // layout, box and total charge only when they change (a new layout
    // reallocates the batch system)
    bool relayout = !L->have_layout || L->R != C || L->off != off;
    if (relayout) rc = ctbop_set_layout(L, C, off.data());
    bool rebox = relayout || L->box.size() != (size_t)3 * C;
    for (int k = 0; !rebox && k < C; ++k)
      for (int d = 0; d < 3; ++d)
        rebox = rebox || L->box[3 * k + d] != h[9 * k + 4 * d] || L->pbc[3 * k + d] != pbc[3 * k + d];
    if (!rc && rebox) rc = ctbop_set_box(L, h.data(), pbc.data());
    if (!rc && (relayout || L->Q != Q)) rc = ctbop_set_total_charge(L, Q.data());
    if (!rc) {
      CK(cudaMemcpyAsync(d_items, items.data(), sizeof(LooItem) * C, cudaMemcpyHostToDevice, s->stream));
      launch_loo_gather(d_items, C, max_n, S, d_x, d_t, d_f, d_q, s->stream);
      CK(cudaGetLastError());
      rc = ctbop_set_types(L, d_t, CTBOP_DEVICE);
      if (!rc) rc = ctbop_set_frozen(L, d_f, CTBOP_DEVICE);
      if (!rc) rc = ctbop_set_positions(L, d_x, CTBOP_DEVICE);
      if (!rc) rc = ctbop_set_charges(L, d_q, CTBOP_DEVICE);
    }
    if (!rc) {
      // start from the given charges, not an extrapolation of another chunk's
      *L->h_int = 1;
      CK(cudaMemcpyAsync(L->S.cg_hist, L->h_int, sizeof(int), cudaMemcpyHostToDevice, s->stream));
      rc = ctbop_compute(L, 0);
    }
    if (rc) {
      std::string why = L->err;
      CK(cudaStreamSynchronize(s->stream));
      return fail(s, rc, "removal energies: " + why);
    }
    std::vector<double> El(C);
    CK(cudaMemcpy2DAsync(El.data(), 8, L->S.rep_acc + RA_E, RA_STRIDE * 8, 8, C, cudaMemcpyDeviceToHost,
                         s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (size_t k = 0; k < j1 - j0; ++k) {
      const Job& jb = chunk[k];
      dE[jb.c] = El[k] + s->T.E0[types[s->off[jb.r] + jb.drop]] - E[jb.r];
    }
    j0 = j1;
  }
  CK(cudaStreamSynchronize(s->stream));
  return CTBOP_OK;
}

// Grow the lists after an overflow (from the counts the last build
// measured) and evaluate again at the current positions.
static int regrow_and_recompute(ctbop_system* s) {
  DevState& S = s->S;
  int mc[3];
  CK(sync_copy(s, mc, S.maxcnt, sizeof(mc), cudaMemcpyDeviceToHost));
  int cc = (std::max(S.cap_cov, mc[0] + mc[0] / 4 + 4) + 3) & ~3;
  int ca = std::max(S.cap_all, cc + mc[1] + mc[1] / 8 + 16);
  int rc = alloc_lists(s, cc, (ca + 7) & ~7);
  if (rc) return rc;
  s->need_rebuild = true;
  rc = ensure_lists(s);
  if (rc) return rc;
  CK(zero_async(s, S.err, sizeof(unsigned)));
  return ctbop_compute(s, 0);
}

// FIRE minimisation, one state per replica (csrc/relax.cu). Each iteration
// reads back the number of replicas still moving and the error word.
int ctbop_minimize(ctbop_system* s, int64_t max_iter, double fmax, double dt0, double dt_max, int64_t* iters,
                   double* fmax_out) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  if (max_iter < 0 || !(fmax > 0) || !std::isfinite(fmax) || !(dt0 > 0) || !std::isfinite(dt_max) || dt_max < dt0)
    return fail(s, CTBOP_ERR_INVALID_ARG, "need max_iter >= 0, fmax > 0, 0 < dt0 <= dt_max");
  if (!s->have_layout || !s->have_box || !s->have_types || !s->have_pos)
    return fail(s, CTBOP_ERR_STATE, "layout, box, types and positions must be set first");
  cudaSetDevice(s->o.device);
  int rc = CTBOP_OK;
  DevState& S = s->S;
  if (!s->have_forces) {
    rc = ctbop_compute(s, 0);
    if (rc) return rc;
  }
  const int R = s->R;
  double* fire = nullptr;
  int* ctl = nullptr;
  Scratch scr(s->stream, s->pool);
  CK(scr.alloc(&fire, (size_t)R * FI_STRIDE));
  CK(scr.alloc(&ctl, 2));
  std::vector<double> fh((size_t)R * FI_STRIDE, 0.0);
  const FireCfg cfg{fmax * fmax, dt_max, 1.1, 0.5, 0.1, 0.99, 5.0, (double)max_iter};
  for (int r = 0; r < R; ++r) {
    fh[(size_t)r * FI_STRIDE + FI_DT] = dt0;
    fh[(size_t)r * FI_STRIDE + FI_ALPHA] = cfg.alpha0;
  }
  CK(sync_copy(s, fire, fh.data(), sizeof(double) * fh.size(), cudaMemcpyHostToDevice));
  CK(zero_async(s, ctl, 2 * sizeof(int)));
  CK(zero_async(s, S.v, sizeof(double) * 3 * (size_t)S.N));   // from rest
  const double half_skin2 = 0.25 * s->o.skin * s->o.skin;
  int redo = 0;
  for (;;) {
    launch_fire_reduce(S, fire, cfg, ctl, ctl + 1, s->stream);
    CK(cudaGetLastError());
    CK(sync_copy(s, s->h_int, ctl + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (*s->h_int == 0) break;
    if (s->mixed) launch_fire_move<float>(S, s->T, fire, half_skin2, s->stream);
    else launch_fire_move<double>(S, s->T, fire, half_skin2, s->stream);
    CK(cudaGetLastError());
    CK(zero_async(s, S.err, sizeof(unsigned)));
    rc = ctbop_compute(s, 0);
    unsigned bits = 0;
    if (!rc) rc = read_err(s, bits);
    while (!rc && (bits & (CT_ERR_NBR_OVERFLOW | CT_ERR_COV_OVERFLOW))) {
      if (++redo > 3) {
        rc = fail(s, CTBOP_ERR_NEIGH_OVERFLOW, "neighbour lists kept overflowing");
        break;
      }
      rc = regrow_and_recompute(s);
      if (!rc) rc = read_err(s, bits);
    }
    if (!rc && (bits & CT_ERR_NONFINITE)) rc = fail(s, CTBOP_ERR_NONFINITE, "non-finite energy, force or position");
    if (!rc && (bits & CT_ERR_CG_MAXITER)) rc = fail(s, CTBOP_ERR_CG_NOT_CONVERGED, "charge CG reached max_iter");
    if (rc) break;
  }
  if (!rc) {
    CK(sync_copy(s, fh.data(), fire, sizeof(double) * fh.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < R; ++r) {
      const double* f = fh.data() + (size_t)r * FI_STRIDE;
      if (iters) iters[r] = f[FI_DONE] == 1.0 ? (int64_t)f[FI_ITERS] : -1;
      if (fmax_out) fmax_out[r] = std::sqrt(f[FI_LASTF2]);
    }
  }
  CK(zero_async(s, S.v, sizeof(double) * 3 * (size_t)S.N));   // left at rest
  CK(cudaStreamSynchronize(s->stream));
  return rc;
}

int ctbop_rings(ctbop_system* s, double bond_cut, int32_t max_size, int64_t cap, ctbop_ring* out, int64_t* n_rings) {
  if (!s) return CTBOP_ERR_INVALID_ARG;
  const double scc = s->p.S[3];   // C-C pair
  if (!n_rings || cap < 0 || (cap > 0 && !out) || max_size < 3 || max_size > 8 || !(bond_cut >= 0) ||
      bond_cut > scc)
    return fail(s, CTBOP_ERR_INVALID_ARG, "rings: need n_rings, cap >= 0 (out if cap > 0), 3 <= max_size <= 8, "
                                          "0 <= bond_cut <= the C-C cutoff S");
  if (!s->have_forces) return fail(s, CTBOP_ERR_STATE, "rings: compute or step first");
  cudaSetDevice(s->o.device);
  if (bond_cut == 0) bond_cut = scc;
  ctbop_ring* d_out = nullptr;
  unsigned long long* d_cnt = nullptr;
  Scratch scr(s->stream, s->pool);
  CK(scr.alloc(&d_out, (size_t)std::max<int64_t>(cap, 1)));
  CK(scr.alloc(&d_cnt, 1));
  CK(zero_async(s, d_cnt, sizeof(unsigned long long)));
  if (s->mixed) launch_rings<float>(s->S, bond_cut, max_size, d_out, cap, d_cnt, s->stream);
  else launch_rings<double>(s->S, bond_cut, max_size, d_out, cap, d_cnt, s->stream);
  CK(cudaGetLastError());
  unsigned long long n = 0;
  CK(sync_copy(s, &n, d_cnt, sizeof(n), cudaMemcpyDeviceToHost));
  int64_t m = std::min<int64_t>((int64_t)n, cap);
  if (m > 0) CK(sync_copy(s, out, d_out, sizeof(ctbop_ring) * m, cudaMemcpyDeviceToHost));
  *n_rings = (int64_t)n;
  CK(cudaStreamSynchronize(s->stream));
  return CTBOP_OK;
}

}  // extern "C"
