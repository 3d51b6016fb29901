// cg.cu — charge minimisation (Sec. 2: charges minimise E_tot at every
// step, by conjugate gradients).
//
// E is quadratic in q, so the constrained minimum (sum_r q = Q_r per
// replica) solves H q + chi = mu 1. Two Jacobi-preconditioned CG solves share
// every pass over the matrix: H s = -chi and H t = 1, after which
// q = s + mu t with mu = (Q - sum s) / sum t. Vectors are stored (s, t)
// interleaved as double2. The iteration is the one-reduction (Chronopoulos-
// Gear) form of PCG: per iteration one matrix pass that also forms the two
// dot products (r.z, w.z) and, in its last block, the step lengths; and one
// element-wise update that forms the sums for the convergence test. Dot
// products, residual sums and the vectors are FP64; the matrix entries and
// the gathered z_j are in the working precision.
//
// The matrix passes run one thread per atom over its column of the list
// (entry e of atom i at e * ld + i), so every warp load of entry e of 32
// consecutive atoms is one 128-byte line, four entries are in flight per
// thread, and the FP64 epilogue (which on this GPU issues at a small fraction
// of the FP32 rate) is lane-parallel rather than once per atom.
//
// Starting guess: the previous solutions extrapolated in time (quadratic
// from three, linear from two, the last one alone otherwise).
//
// Convergence (per replica): max|r_s| + |mu| max|r_t| below tol, a bound on
// the max-norm of the stationarity residual mu 1 - H q - chi (an rms test
// lets a few weakly coupled atoms, such as adatoms, keep large errors). The
// last block of each update launch decides, marks converged replicas, and
// ends the loop through the CUDA-graph condition (or a device flag the host
// polls).
#include "internal.cuh"
#include "kernels.h"

namespace ct {

__device__ inline double ldcg(const double* p) { return __ldcg(p); }

// Grid-wide "am I the last block" after this block's atomics.
__device__ inline bool last_block(int* counter) {
  __shared__ bool am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int t = atomicAdd(counter, 1);
    am_last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Convergence test for every unconverged replica from the sums at upd_off
// and the residual maxima of buffer mbuf.
__device__ inline int check_replicas(int R, double* cg, const float* rmax, int* conv, int* iters, int upd_off,
                                     int mbuf, int it_done, double tol, int first) {
  int all = 1;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (conv[r]) continue;
    double* c = cg + (size_t)r * CG_STRIDE;
    const double* u5 = c + upd_off;
    double rss = ldcg(u5 + 0), rtt = ldcg(u5 + 1), rst = ldcg(u5 + 2), xs = ldcg(u5 + 3), xt = ldcg(u5 + 4);
    float ms = __ldcg(rmax + (size_t)r * 6 + mbuf * 2), mt = __ldcg(rmax + (size_t)r * 6 + mbuf * 2 + 1);
    double nat = c[CG_NAT];
    // mu is undefined before t has any weight (cold start: x = 0)
    double mu = (c[CG_Q] - xs) / xt;
    bool mu_ok = (xt != 0.0) && isfinite(mu);
    double res2 = (rss + 2.0 * mu * rst + mu * mu * rtt) / (nat > 0 ? nat : 1.0);
    double rms = (mu_ok && isfinite(res2)) ? sqrt(res2 > 0.0 ? res2 : 0.0) : INFINITY;
    double bound = mu_ok ? (double)ms + fabs(mu) * (double)mt : INFINITY;
    if (!isfinite(bound)) bound = INFINITY;
    c[CG_MU] = mu_ok ? mu : 0.0;
    c[CG_RES] = rms;
    c[CG_RESMAX] = bound;
    if (first) c[CG_RES0] = bound;
    if (nat == 0 || bound <= tol) {
      conv[r] = 1;
      iters[r] = it_done;
    } else {
      all = 0;
    }
  }
  return __syncthreads_and(all);
}

// Per-lane running maxima of |r_s|, |r_t| for one replica, merged per warp
// and flushed with atomics (float bit patterns order like non-negative values).
struct LaneMax {
  int rep = -1;
  float s = 0.f, t = 0.f;
  __device__ inline void flush(float* base) {
    if (rep >= 0) {
      atomic_max_nonneg(base + (size_t)rep * 6, s);
      atomic_max_nonneg(base + (size_t)rep * 6 + 1, t);
    }
    s = t = 0.f;
  }
  __device__ inline void add(int r, float as, float at, float* base) {
    if (r != rep) { flush(base); rep = r; }
    s = fmaxf(s, as);
    t = fmaxf(t, at);
  }
  __device__ inline void finish(float* base) {
    int r0 = __shfl_sync(CT_FULL, rep, 0);
    if (__all_sync(CT_FULL, rep == r0)) {
      for (int o = 16; o > 0; o >>= 1) {
        s = fmaxf(s, __shfl_xor_sync(CT_FULL, s, o));
        t = fmaxf(t, __shfl_xor_sync(CT_FULL, t, o));
      }
      if ((threadIdx.x & 31) != 0) rep = -1;
    }
    flush(base);
  }
};

// --------------------------------------------------------------- prepare
__global__ void k_cg_prep(int R, double* __restrict__ cg, float* __restrict__ rmax, int* __restrict__ conv,
                          int* __restrict__ iters, int* __restrict__ it, int* __restrict__ blocks,
                          int* __restrict__ active) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double* c = cg + (size_t)r * CG_STRIDE;
    for (int k = 0; k < CG_MU; ++k) c[k] = 0.0;
    for (int k = 0; k < 6; ++k) rmax[(size_t)r * 6 + k] = 0.f;
    conv[r] = 0;
    iters[r] = 0;
  }
  if (threadIdx.x == 0) {
    *it = 0;
    blocks[0] = 0;
    blocks[1] = 0;
    blocks[2] = 0;
    *active = 1;
  }
}

// Starting guess extrapolated from the stored solutions and its copy in the
// matvec precision; shifts the history (h2 <- h1, h1 <- the last solution).
template <class R>
__global__ void k_cg_extrap(int N, double2* __restrict__ x, double2* __restrict__ h1, double2* __restrict__ h2,
                            typename Vec2<R>::T* __restrict__ xr, const int* __restrict__ hist) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int nh = *hist;
  double2 xo = x[i], a = h1[i], b = h2[i], x0;
  if (nh >= 3) {
    x0.x = 3.0 * xo.x - 3.0 * a.x + b.x;
    x0.y = 3.0 * xo.y - 3.0 * a.y + b.y;
  } else if (nh == 2) {
    x0.x = 2.0 * xo.x - a.x;
    x0.y = 2.0 * xo.y - a.y;
  } else {
    x0 = xo;
  }
  h2[i] = a;
  h1[i] = xo;
  x[i] = x0;
  typename Vec2<R>::T v;
  v.x = (R)x0.x;
  v.y = (R)x0.y;
  xr[i] = v;
}

// Row sums sum_e M_e v_j(e) of atom i over its column of the list.
template <class R>
__device__ inline void row_sum(int i, int na, int ld, const int* __restrict__ nbr, const R* __restrict__ M,
                               const typename Vec2<R>::T* __restrict__ v, R& hs, R& ht) {
  using V2 = typename Vec2<R>::T;
  const int* pn = nbr + i;
  const R* pm = M + i;
  hs = R(0);
  ht = R(0);
  int e = 0;
  for (; e + 4 <= na; e += 4) {
    size_t o = (size_t)e * ld;
    int j0 = __ldg(pn + o), j1 = __ldg(pn + o + ld), j2 = __ldg(pn + o + 2 * (size_t)ld),
        j3 = __ldg(pn + o + 3 * (size_t)ld);
    R m0 = __ldg(pm + o), m1 = __ldg(pm + o + ld), m2 = __ldg(pm + o + 2 * (size_t)ld),
      m3 = __ldg(pm + o + 3 * (size_t)ld);
    V2 z0 = v[j0], z1 = v[j1], z2 = v[j2], z3 = v[j3];
    hs += m0 * z0.x + m1 * z1.x + m2 * z2.x + m3 * z3.x;
    ht += m0 * z0.y + m1 * z1.y + m2 * z2.y + m3 * z3.y;
  }
  for (; e < na; ++e) {
    size_t o = (size_t)e * ld;
    int j0 = __ldg(pn + o);
    R m0 = __ldg(pm + o);
    V2 z0 = v[j0];
    hs += m0 * z0.x;
    ht += m0 * z0.y;
  }
}

// r = b - H x0, z = D^-1 r with b = (-chi, 1); sums and maxima for the
// initial test (kept in update buffer 2).
template <class R>
__global__ void k_cg_init(int N, int ld, int chunk, const int* __restrict__ nbr,
                          const int* __restrict__ nall, const R* __restrict__ M, const double* __restrict__ Dg,
                          const double* __restrict__ dinv, const int* __restrict__ type, const int* __restrict__ rep,
                          TypeParams T, const double2* __restrict__ x, const typename Vec2<R>::T* __restrict__ xr,
                          double2* __restrict__ r, double2* __restrict__ z, typename Vec2<R>::T* __restrict__ zr,
                          double* __restrict__ cg, float* __restrict__ rmax, int Rn, int* __restrict__ conv,
                          int* __restrict__ iters, int* __restrict__ blocks, int* __restrict__ active, double tol) {
  const int ub = CG_UPD + 2 * 5;
  RepAcc<5> acc;
  acc.init();
  LaneMax lm;
  int a0 = blockIdx.x * chunk, a1 = min(N, a0 + chunk);
  for (int i = a0 + (int)threadIdx.x; i < a1; i += blockDim.x) {
    R hs, ht;
    row_sum<R>(i, nall[i], ld, nbr, M, xr, hs, ht);
    double2 xi = x[i];
    double D = Dg[i];
    double2 ri;
    ri.x = -T.chi[type[i]] - (D * xi.x + (double)hs);
    ri.y = 1.0 - (D * xi.y + (double)ht);
    double di = dinv[i];
    double2 zi;
    zi.x = ri.x * di;
    zi.y = ri.y * di;
    r[i] = ri;
    z[i] = zi;
    typename Vec2<R>::T zz;
    zz.x = (R)zi.x;
    zz.y = (R)zi.y;
    zr[i] = zz;
    int rid = rep[i];
    acc.to(rid, cg + ub, CG_STRIDE);
    acc.v[0] += ri.x * ri.x;
    acc.v[1] += ri.y * ri.y;
    acc.v[2] += ri.x * ri.y;
    acc.v[3] += xi.x;
    acc.v[4] += xi.y;
    lm.add(rid, fabsf((float)ri.x), fabsf((float)ri.y), rmax + 2 * 2);
  }
  lane_flush<5>(acc, cg + ub, CG_STRIDE);
  lm.finish(rmax + 2 * 2);
  if (last_block(blocks)) {
    int all = check_replicas(Rn, cg, rmax, conv, iters, ub, 2, 0, tol, 1);
    if (threadIdx.x == 0) {
      blocks[0] = 0;
      if (all) *active = 0;
    }
  }
}

// w = H z and the dots (r.z, w.z) for both solves; the last block turns the
// dots into the step lengths alpha, beta of this iteration.
template <class R>
__global__ void k_cg_mv(int N, int ld, int chunk, const int* __restrict__ nbr, const int* __restrict__ nall,
                        const R* __restrict__ M, const double* __restrict__ Dg, const int* __restrict__ rep,
                        const int* __restrict__ conv, const int* __restrict__ itp,
                        const typename Vec2<R>::T* __restrict__ zr, const double2* __restrict__ z,
                        const double2* __restrict__ r, double2* __restrict__ w, double* __restrict__ cg, int Rn,
                        int* __restrict__ blocks, const int* __restrict__ active) {
  if (*active == 0) return;
  int it = *itp;
  int buf = CG_DOTS + (it & 1) * 4;
  RepAcc<4> acc;
  acc.init();
  int a0 = blockIdx.x * chunk, a1 = min(N, a0 + chunk);
  for (int i = a0 + (int)threadIdx.x; i < a1; i += blockDim.x) {
    int rid = rep[i];
    if (conv[rid]) continue;
    R hs, ht;
    row_sum<R>(i, nall[i], ld, nbr, M, zr, hs, ht);
    double2 zi = z[i], rri = r[i];
    double D = Dg[i];
    double2 wi;
    wi.x = D * zi.x + (double)hs;
    wi.y = D * zi.y + (double)ht;
    w[i] = wi;
    acc.to(rid, cg + buf, CG_STRIDE);
    acc.v[0] += rri.x * zi.x;
    acc.v[1] += wi.x * zi.x;
    acc.v[2] += rri.y * zi.y;
    acc.v[3] += wi.y * zi.y;
  }
  lane_flush<4>(acc, cg + buf, CG_STRIDE);
  if (last_block(blocks + 2)) {
    int sprev = CG_SCAL + ((it + 1) & 1) * 4;
    int scur = CG_SCAL + (it & 1) * 4;
    for (int rr = threadIdx.x; rr < Rn; rr += blockDim.x) {
      if (conv[rr]) continue;
      double* c = cg + (size_t)rr * CG_STRIDE;
      double g[2] = {ldcg(c + buf + 0), ldcg(c + buf + 2)};
      double d[2] = {ldcg(c + buf + 1), ldcg(c + buf + 3)};
      for (int k = 0; k < 2; ++k) {
        double a = 0.0, b = 0.0;
        if (it == 0) {
          a = d[k] != 0.0 ? g[k] / d[k] : 0.0;
        } else {
          double gp = c[sprev + 2 * k], ap = c[sprev + 2 * k + 1];
          b = gp != 0.0 ? g[k] / gp : 0.0;
          double den = d[k] - (ap != 0.0 ? b * g[k] / ap : 0.0);
          a = den != 0.0 ? g[k] / den : 0.0;
        }
        c[CG_AB + 2 * k] = a;
        c[CG_AB + 2 * k + 1] = b;
        c[scur + 2 * k] = g[k];
        c[scur + 2 * k + 1] = a;
      }
    }
    if (threadIdx.x == 0) blocks[2] = 0;
  }
}

// Element-wise update, the sums and maxima for the convergence test.
template <class R>
__global__ void k_cg_up(int N, int chunk, const int* __restrict__ rep, const double* __restrict__ dinv,
                        int* __restrict__ conv, int* __restrict__ iters, int* __restrict__ itp,
                        const double2* __restrict__ w, double2* __restrict__ x, double2* __restrict__ r,
                        double2* __restrict__ p, double2* __restrict__ s, double2* __restrict__ z,
                        typename Vec2<R>::T* __restrict__ zr, double* __restrict__ cg, float* __restrict__ rmax,
                        int Rn, int* __restrict__ blocks, int* __restrict__ active, unsigned* __restrict__ err,
                        double tol, int max_iter, int use_cond, cudaGraphConditionalHandle cond) {
  if (*active == 0) {
    // nothing left to do (converged at the start): end the loop
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  int it = *itp;
  int mb = it % 3;
  int ubuf = CG_UPD + mb * 5;
  // zero the buffers the next iteration accumulates into
  if (blockIdx.x == 0) {
    int dn = CG_DOTS + ((it + 1) & 1) * 4, un = CG_UPD + ((it + 1) % 3) * 5, mn = (it + 1) % 3;
    for (int q = threadIdx.x; q < Rn * 11; q += blockDim.x) {
      int rr = q / 11, k = q % 11;
      double* c = cg + (size_t)rr * CG_STRIDE;
      if (k < 4) c[dn + k] = 0.0;
      else if (k < 9) c[un + k - 4] = 0.0;
      else rmax[(size_t)rr * 6 + mn * 2 + (k - 9)] = 0.f;
    }
  }
  RepAcc<5> acc;
  acc.init();
  LaneMax lm;
  int a0 = blockIdx.x * chunk, a1 = min(N, a0 + chunk);
  int crid = -1;
  double as = 0, bs = 0, at = 0, bt = 0;
  for (int i = a0 + (int)threadIdx.x; i < a1; i += blockDim.x) {
    int rid = rep[i];
    if (conv[rid]) continue;
    if (rid != crid) {
      const double* c = cg + (size_t)rid * CG_STRIDE;
      as = ldcg(c + CG_AB + 0); bs = ldcg(c + CG_AB + 1);
      at = ldcg(c + CG_AB + 2); bt = ldcg(c + CG_AB + 3);
      crid = rid;
    }
    double2 zi = z[i], wi = w[i], pi = p[i], si = s[i], xi = x[i], ri = r[i];
    pi.x = zi.x + bs * pi.x; pi.y = zi.y + bt * pi.y;
    si.x = wi.x + bs * si.x; si.y = wi.y + bt * si.y;
    xi.x += as * pi.x; xi.y += at * pi.y;
    ri.x -= as * si.x; ri.y -= at * si.y;
    double di = dinv[i];
    zi.x = ri.x * di; zi.y = ri.y * di;
    p[i] = pi; s[i] = si; x[i] = xi; r[i] = ri; z[i] = zi;
    typename Vec2<R>::T zz;
    zz.x = (R)zi.x; zz.y = (R)zi.y;
    zr[i] = zz;
    acc.to(rid, cg + ubuf, CG_STRIDE);
    acc.v[0] += ri.x * ri.x; acc.v[1] += ri.y * ri.y; acc.v[2] += ri.x * ri.y;
    acc.v[3] += xi.x; acc.v[4] += xi.y;
    lm.add(rid, fabsf((float)ri.x), fabsf((float)ri.y), rmax + mb * 2);
  }
  lane_flush<5>(acc, cg + ubuf, CG_STRIDE);
  lm.finish(rmax + mb * 2);
  if (last_block(blocks + 1)) {
    int all = check_replicas(Rn, cg, rmax, conv, iters, ubuf, mb, it + 1, tol, 0);
    if (threadIdx.x == 0) {
      blocks[1] = 0;
      *itp = it + 1;
      bool stop = all || (it + 1 >= max_iter);
      if (stop) {
        if (!all) atomicOr(err, CT_ERR_CG_MAXITER);
        *active = 0;
      }
      if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
    }
  }
}

// q = s + mu t per replica (and its copy in the working precision); count
// the solve's iterations and its history.
template <class R>
__global__ void k_cg_final(int N, const int* __restrict__ rep, const double2* __restrict__ x,
                           const double* __restrict__ cg, double* __restrict__ q, R* __restrict__ qr,
                           const int* __restrict__ itp, long long* __restrict__ total, int* __restrict__ hist) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *total += *itp;
    int h = *hist;
    *hist = h < 3 ? h + 1 : 3;
  }
  if (i >= N) return;
  double mu = cg[(size_t)rep[i] * CG_STRIDE + CG_MU];
  double2 xi = x[i];
  double qi = xi.x + mu * xi.y;
  q[i] = qi;
  qr[i] = (R)qi;
}

// Working-precision copy of charges set from outside the solve.
template <class R>
__global__ void k_copy_q(int N, const double* __restrict__ q, R* __restrict__ qr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) qr[i] = (R)q[i];
}

// --------------------------------------------------------------- launchers
static inline int chunk_grid(int N, int per_block_min, int gmax, int& chunk) {
  int grid = (N + per_block_min - 1) / per_block_min;
  if (grid > gmax) grid = gmax;
  if (grid < 1) grid = 1;
  chunk = (N + grid - 1) / grid;
  return (N + chunk - 1) / chunk;
}

template <class R>
void launch_cg_begin(const DevState& S, const TypeParams& T, cudaStream_t st, double tol) {
  k_cg_prep<<<1, 256, 0, st>>>(S.R, S.cg, S.cg_rmax, S.cg_conv, S.cg_iters, S.cg_it, S.cg_blocks, S.cg_active);
  if (S.N == 0) return;
  k_cg_extrap<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.cx, S.cxh1, S.cxh2, (typename Vec2<R>::T*)S.cxr,
                                                    S.cg_hist);
  int chunk;
  int grid = atom_dims(S.N, S.nsm, (const void*)k_cg_init<R>, 256, chunk);
  k_cg_init<R><<<grid, 256, 0, st>>>(S.N, S.ld, chunk, S.nbr, S.nall, (const R*)S.M, S.Dg, S.dinv, S.type,
                                     S.rep, T, S.cx, (const typename Vec2<R>::T*)S.cxr, S.cr, S.cz,
                                     (typename Vec2<R>::T*)S.czr, S.cg, S.cg_rmax, S.R, S.cg_conv, S.cg_iters,
                                     S.cg_blocks, S.cg_active, tol);
}

template <class R>
void launch_cg_mv(const DevState& S, cudaStream_t st) {
  if (S.N == 0) return;
  int chunk;
  int grid = atom_dims(S.N, S.nsm, (const void*)k_cg_mv<R>, 256, chunk);
  k_cg_mv<R><<<grid, 256, 0, st>>>(S.N, S.ld, chunk, S.nbr, S.nall, (const R*)S.M, S.Dg, S.rep, S.cg_conv,
                                   S.cg_it, (const typename Vec2<R>::T*)S.czr, S.cz, S.cr, S.cw, S.cg, S.R,
                                   S.cg_blocks, S.cg_active);
}

template <class R>
void launch_cg_up(const DevState& S, const SolveCfg& cfg, cudaStream_t st) {
  if (S.N == 0) return;
  int chunk2;
  int grid2 = chunk_grid(S.N, 256, S.nsm * 4, chunk2);
  k_cg_up<R><<<grid2, 256, 0, st>>>(S.N, chunk2, S.rep, S.dinv, S.cg_conv, S.cg_iters, S.cg_it, S.cw, S.cx, S.cr,
                                    S.cp, S.cs, S.cz, (typename Vec2<R>::T*)S.czr, S.cg, S.cg_rmax, S.R,
                                    S.cg_blocks, S.cg_active, S.err, cfg.tol, cfg.max_iter, cfg.use_cond, cfg.cond);
}

template <class R>
void launch_cg_iter(const DevState& S, const SolveCfg& cfg, cudaStream_t st) {
  launch_cg_mv<R>(S, st);
  launch_cg_up<R>(S, cfg, st);
}

template <class R>
void launch_cg_end(const DevState& S, cudaStream_t st) {
  int n = S.N > 0 ? S.N : 1;
  k_cg_final<R><<<(n + 255) / 256, 256, 0, st>>>(S.N, S.rep, S.cx, S.cg, S.q, (R*)S.qr, S.cg_it, S.cg_total,
                                                 S.cg_hist);
}

template <class R>
void launch_copy_q(const DevState& S, cudaStream_t st) {
  if (S.N == 0) return;
  k_copy_q<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.q, (R*)S.qr);
}

template void launch_cg_begin<float>(const DevState&, const TypeParams&, cudaStream_t, double);
template void launch_cg_begin<double>(const DevState&, const TypeParams&, cudaStream_t, double);
template void launch_cg_mv<float>(const DevState&, cudaStream_t);
template void launch_cg_mv<double>(const DevState&, cudaStream_t);
template void launch_cg_up<float>(const DevState&, const SolveCfg&, cudaStream_t);
template void launch_cg_up<double>(const DevState&, const SolveCfg&, cudaStream_t);
template void launch_cg_iter<float>(const DevState&, const SolveCfg&, cudaStream_t);
template void launch_cg_iter<double>(const DevState&, const SolveCfg&, cudaStream_t);
template void launch_cg_end<float>(const DevState&, cudaStream_t);
template void launch_cg_end<double>(const DevState&, cudaStream_t);
template void launch_copy_q<float>(const DevState&, cudaStream_t);
template void launch_copy_q<double>(const DevState&, cudaStream_t);

}  // namespace ct
