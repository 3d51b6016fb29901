// cg.cu — charge minimisation (Sec. 2: charges minimise E_tot at every
// step, by conjugate gradients).
//
// E is quadratic in q, so the constrained minimum (sum_r q = Q_r per
// replica) solves H q + chi = mu 1 on the set sum q = Q. The solve is a
// projected, preconditioned CG that keeps the iterate feasible (M^-1 the
// block-Jacobi inverse below, or D^-1):
//   r = -(H q + chi)                       (negative gradient)
//   y = M^-1 r,  z = y - (sum y / sum d) d  with d = M^-1 1 (sum z = 0)
//   w = H z = H y - c H d                   (c = sum y / sum d)
// so every direction keeps the total charge and q never leaves the
// constraint. The iteration is the one-reduction (Chronopoulos-Gear) form:
// per iteration one matrix pass (w and the dots r.z, w.z; its last block
// forms alpha, beta) and one element-wise update (p, s, q, r, y and the sums
// that give the next c and the convergence test). H d is formed once per
// solve, in the starting pass.
//
// Re-centring: r carries a large constant part (-mu 1) that the projection
// removes only in exact arithmetic; once the residual is small, rounding of
// that part pollutes r.z and the iteration diverges. The projection and every
// CG scalar are unchanged by adding a constant to r, so each update subtracts
// the previous mean of r and accumulates the shift (mu = -(mean r + shift)).
//
// Precision: the iterate q and every reduction (dots, sums, maxima, the
// scalars alpha, beta, c, mu) are FP64. The recursion vectors r, p, s = H p,
// the iteration's change dq = q - q0, y = M^-1 r, w = H z, d, v, the matrix
// entries and the gathered y_j are in the working precision (FP32 in the
// mixed policy, FP64 in the FP64 policy); the mixed policy stores the
// block-Jacobi inverses in FP16 (see BlockStore). FP32 recursion vectors keep
// conjugacy only because r.z is formed from the centred residual (below);
// dq is folded into the FP64 q once per solve. Rounding of y and d keeps
// sum z from being exactly zero, so after the solve q is shifted uniformly
// onto sum q = Q.
//
// The matrix passes run one thread per atom over its column of the list
// (entry e of atom i at e * ld + i): a warp load of entry e of 32 consecutive
// atoms is one 128-byte line. The number of entries in flight per thread
// (the batch depth B of k_cg_mv: 4, 8 or 16) is a template parameter, timed
// on the live matrix after every list allocation and the fastest kept. The
// FP64 epilogue (issued at a small fraction of the FP32 rate on this GPU) is
// lane-parallel.
//
// Starting guess: the previous solutions extrapolated in time (quadratic
// from three, linear from two, the last one alone, zero with no history),
// then shifted uniformly onto sum q = Q.
//
// Convergence (per replica): max_i |r_i - mean(r)| below tol, i.e. the
// max-norm of the stationarity residual H q + chi - mu 1 with mu = -mean(r)
// (an rms test lets a few weakly coupled atoms, such as adatoms, keep large
// errors). The last block of each update launch decides, marks converged
// replicas, and ends the loop through the CUDA-graph condition (or a device
// flag the host polls).
#include "internal.cuh"
#include <cuda_fp16.h>
#include "kernels.h"

namespace ct {

__device__ inline double ldcg(const double* p) { return __ldcg(p); }


// Order-preserving map of doubles to unsigned 64-bit ints (max of the map =
// map of the max), for atomicMax on signed values.
__device__ inline unsigned long long dmap(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double dunmap(unsigned long long u) {
  unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double((long long)b);
}

// Per-thread running max of r and of -r for one replica. finish() merges
// them over the warp and the block (one atomicMax per block and replica, on
// the order-preserving map); every thread of the block must call it.
template <class R>
struct LaneMax {
  int rep = -1;
  R hi = -R(INFINITY), lo = -R(INFINITY);   // max r, max -r
  __device__ inline void flush(unsigned long long* base) {
    if (rep >= 0) {
      atomicMax(base + (size_t)rep * 6, dmap((double)hi));
      atomicMax(base + (size_t)rep * 6 + 1, dmap((double)lo));
    }
    hi = lo = -R(INFINITY);
  }
  __device__ inline void add(int r, R v, unsigned long long* base) {
    if (r != rep) { flush(base); rep = r; }
    hi = fmax(hi, v);
    lo = fmax(lo, -v);
  }
  __device__ inline void finish(unsigned long long* base) {
    __shared__ int s_rep[32];
    __shared__ R s_hi[32], s_lo[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int r0 = __shfl_sync(CT_FULL, rep, 0);
    bool same = __all_sync(CT_FULL, rep == r0);
    if (same) {
      for (int o = 16; o > 0; o >>= 1) {
        hi = fmax(hi, __shfl_xor_sync(CT_FULL, hi, o));
        lo = fmax(lo, __shfl_xor_sync(CT_FULL, lo, o));
      }
    } else {
      flush(base);   // a replica boundary inside the warp: per-lane atomics
    }
    if (lane == 0) {
      s_rep[warp] = same ? r0 : -1;
      s_hi[warp] = hi;
      s_lo[warp] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int nw = blockDim.x >> 5;
      rep = -1;
      hi = lo = -R(INFINITY);
      for (int w = 0; w < nw; ++w) {
        if (s_rep[w] < 0) continue;
        if (s_rep[w] != rep) { flush(base); rep = s_rep[w]; }
        hi = fmax(hi, s_hi[w]);
        lo = fmax(lo, s_lo[w]);
      }
      flush(base);
    }
    __syncthreads();
  }
};

// Sums of one value set per thread (rid < 0: none) into out[rid * stride +
// k]: a warp sum in the working precision when the warp holds one replica
// (the common case), per-lane atomics otherwise, then one FP64 atomic per
// block and replica. Every thread of the block must call it.
template <class R, int NV>
__device__ inline void flush_values(int rid, const R (&v)[NV], double* out, int stride) {
  int lane = threadIdx.x & 31;
  int r0 = __shfl_sync(CT_FULL, rid, 0);
  bool same = __all_sync(CT_FULL, rid == r0);
  RepAcc<NV> w;
  w.init();
  if (same) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      R t = warp_sum(v[k]);
      if (lane == 0) w.v[k] = (double)t;
    }
    if (lane == 0) w.rep = r0;
  } else if (rid >= 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) atomicAdd(out + (size_t)rid * stride + k, (double)v[k]);
  }
  block_flush<NV>(w, out, stride);
}

// Blocks for an element-wise pass over 256-atom tiles: at most what fits on
// the device at once, so each thread takes several atoms and the reductions
// are paid once per thread, not once per atom.
static int stride_grid(int N, int nsm, const void* kernel) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess || occ < 1) occ = 1;
  long long tiles = ((long long)N + 255) / 256, slots = (long long)nsm * occ;
  long long g = tiles < slots ? tiles : slots;
  return (int)(g < 1 ? 1 : g);
}

// Convergence test for every unconverged replica from the sums (sum y,
// sum r, sum r^2) at upd_off and the maxima of buffer mbuf; records the mean
// of r for the next re-centring and c for the next matrix pass.
__device__ inline int check_replicas(int R, double* cg, const unsigned long long* rmax, int* conv, int* iters,
                                     int upd_off,
                                     int mbuf, int it_done, double tol, int first) {
  int all = 1;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (conv[r]) continue;
    double* c = cg + (size_t)r * CG_STRIDE;
    const double* u4 = c + upd_off;
    double sy = ldcg(u4 + 0), sr = ldcg(u4 + 1), srr = ldcg(u4 + 2);
    double hi = dunmap(__ldcg(rmax + (size_t)r * 6 + mbuf * 2));
    double lo = dunmap(__ldcg(rmax + (size_t)r * 6 + mbuf * 2 + 1));
    double nat = c[CG_NAT];
    double m = nat > 0 ? sr / nat : 0.0;
    double bound = fmax(hi - m, lo + m);       // max_i |r_i - m|
    double var = nat > 0 ? srr / nat - m * m : 0.0;
    double rms = sqrt(var > 0.0 ? var : 0.0);
    if (!isfinite(bound)) bound = INFINITY;
    c[CG_M] = m;
    c[CG_MU] = -(m + c[CG_SHIFT]);
    c[CG_RES] = rms;
    c[CG_RESMAX] = bound;
    if (first) c[CG_RES0] = bound;
    double sd = c[CG_SD];
    c[CG_C] = sd != 0.0 ? sy / sd : 0.0;
    if (nat == 0 || bound <= tol) {
      conv[r] = 1;
      iters[r] = it_done;
    } else {
      all = 0;
    }
  }
  return __syncthreads_and(all);
}

// --------------------------------------------------------------- prepare
__global__ void k_cg_prep(int N, int R, double* __restrict__ cg, unsigned long long* __restrict__ rmax,
                          int* __restrict__ conv, int* __restrict__ iters, int* __restrict__ it, int* __restrict__ blocks,
                          int* __restrict__ active) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double* c = cg + (size_t)r * CG_STRIDE;
    for (int k = 0; k < CG_MU; ++k) c[k] = 0.0;
    c[CG_SQF] = 0.0;
    for (int k = 0; k < 6; ++k) rmax[(size_t)r * 6 + k] = 0ull;
    conv[r] = 0;
    iters[r] = 0;
  }
  if (threadIdx.x == 0) {
    *it = 0;
    blocks[0] = 0;
    blocks[1] = 0;
    blocks[2] = 0;
    *active = N > 0 ? 1 : 0;   // no atoms: nothing to solve, the loop ends at once
  }
}

// Block-Jacobi preconditioner: M^-1 is the exact inverse of each 32 x 32
// diagonal block of H (atoms 32b .. 32b+31 in storage order; in Jacobi
// order the blocks hold the strong local couplings, the covalent w terms and
// the near charge-kernel entries). One warp per block assembles the block
// from the stored rows (diagonal, self-images, entries whose atom is in the
// block), symmetrises it, factorises it (Cholesky), inverts the factor and
// forms M_b^-1 = W^T W with W = L^-1 (exactly symmetric: both triangles are
// the same sums in the same order). Lanes past N get an identity row. Atoms
// of different replicas in one block have exactly zero coupling, which the
// factorisation keeps. A block that is not numerically positive definite
// falls back to its Jacobi inverse. Also writes d = M^-1 1 (row sums).
//
// The inverses are formed again only after a list rebuild (the rebuild count
// differs from the one they were formed at; k_precond_mark records it once
// every block is done): between rebuilds no atom moves more than half the
// skin, H drifts by a few per cent, and a slightly stale M^-1 is still a
// fixed symmetric positive definite preconditioner for the whole solve, so
// only the iteration count can change, never the converged result.
// Storage of the block inverses: FP16 on the FP32 path (a fixed symmetric
// preconditioner steers only the iteration count; FP16 halves the largest
// stream of the update pass, 128 of its 176 bytes per atom), FP64 on the
// FP64 path. The stored values are exactly symmetric (see k_block_setup), so
// their FP16 roundings are too, and d = M^-1 1 is summed from the stored
// values.
template <class R> struct BlockStore { using T = R; };
// largest block-inverse entry kept (FP16's largest finite value is 65504)
constexpr double kBlockMax = 6.0e4;
template <> struct BlockStore<float> { using T = __half; };
__device__ inline __half blk_pack(float v) { return __float2half_rn(v); }
__device__ inline double blk_pack(double v) { return v; }
__device__ inline float blk_unpack(__half h) { return __half2float(h); }
__device__ inline double blk_unpack(double v) { return v; }
// Row `lane` of a block inverse, 32 values, with 16-byte stores.
template <class R>
__device__ inline void store_block_row(typename BlockStore<R>::T* out, int lane,
                                       const typename BlockStore<R>::T (&row)[32]) {
  constexpr int NV = 32 * (int)sizeof(typename BlockStore<R>::T) / 16;
  uint4* dst = reinterpret_cast<uint4*>(out + (size_t)lane * 32);
  const uint4* src = reinterpret_cast<const uint4*>(row);
#pragma unroll
  for (int k = 0; k < NV; ++k) dst[k] = src[k];
}

template <class R>
__global__ void __launch_bounds__(128)
    k_block_setup(int N, int ld, const int2* __restrict__ nl, const int* __restrict__ nmat,
                  const void* __restrict__ M, const R* __restrict__ Dg, typename BlockStore<R>::T* __restrict__ binv,
                  R* __restrict__ bsum, const long long* __restrict__ rebuilds,
                  const long long* __restrict__ epoch) {
  if (*rebuilds == *epoch) return;
  __shared__ R sh[4][32][33];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int base = (blockIdx.x * 4 + warp) * 32;
  if (base >= N) return;   // whole warps only
  R(*A)[33] = sh[warp];
  for (int j = 0; j < 32; ++j) A[lane][j] = R(0);
  __syncwarp();
  int i = base + lane;
  if (i < N) {
    MatView<R> mv(nl, M);
    int na = nmat[i];
    int e = 0;
    for (; e + 8 <= na; e += 8) {   // eight entries in flight
      int jj[8];
      R vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) mv.get((size_t)(e + u) * ld + i, jj[u], vv[u]);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        unsigned dj = (unsigned)(jj[u] - base);
        if (dj < 32u) A[lane][dj] += vv[u];
      }
    }
    for (; e < na; ++e) {
      int j;
      R v;
      mv.get((size_t)e * ld + i, j, v);
      unsigned dj = (unsigned)(j - base);
      if (dj < 32u) A[lane][dj] += v;
    }
    A[lane][lane] += Dg[i];
  } else {
    A[lane][lane] = R(1);
  }
  __syncwarp();
  for (int j = lane + 1; j < 32; ++j) {
    R m = R(0.5) * (A[lane][j] + A[j][lane]);
    A[lane][j] = m;
    A[j][lane] = m;
  }
  __syncwarp();
  R hii = A[lane][lane];
  bool ok = true;
  for (int k = 0; k < 32; ++k) {   // Cholesky, lower triangle in place
    R piv = A[k][k];
    if (!(piv > R(0))) { ok = false; break; }   // the same value in every lane
    R lk = sqrt(piv);
    __syncwarp();
    if (lane == k) A[k][k] = lk;
    if (lane > k) A[lane][k] /= lk;
    __syncwarp();
    if (lane > k)
      for (int j = k + 1; j <= lane; ++j) A[lane][j] -= A[lane][k] * A[j][k];
    __syncwarp();
  }
  typename BlockStore<R>::T* out = binv + (size_t)(base >> 5) * 1024;
  // the diagonal (Jacobi) block instead, where the factorisation fails or
  // the inverse leaves the stored type's range (FP16: a block with an
  // eigenvalue below 2e-5, never met with physical parameters); the
  // preconditioner only has to stay fixed and positive definite
  auto jacobi_block = [&]() {
    __syncwarp();
    const bool half = sizeof(typename BlockStore<R>::T) == 2;
    const R di = half ? min(R(1) / hii, (R)kBlockMax) : R(1) / hii;
    __align__(16) typename BlockStore<R>::T row[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) row[j] = blk_pack(j == lane ? di : R(0));
    store_block_row<R>(out, lane, row);
    if (i < N) bsum[i] = (R)blk_unpack(blk_pack(di));
  };
  if (!ok) {
    jacobi_block();
    return;
  }
  // column `lane` of W = L^-1 by forward substitution (registers)
  R w[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    R t = r == lane ? R(1) : R(0);
#pragma unroll
    for (int m = 0; m < r; ++m) t -= A[r][m] * w[m];
    w[r] = r < lane ? R(0) : t / A[r][r];
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) A[r][lane] = w[r];   // A now holds W (A[r][c] = W_rc)
  __syncwarp();
  R rs = R(0), tmax = R(0);
  __align__(16) typename BlockStore<R>::T row[32];   // row `lane` of the block
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    R t = R(0);
    for (int k = max(lane, j); k < 32; ++k) t += A[k][lane] * A[k][j];
    tmax = max(tmax, fabs(t));
    row[j] = blk_pack(t);   // element (lane, j)
    rs += (R)blk_unpack(row[j]);
  }
  if (sizeof(typename BlockStore<R>::T) == 2 && __any_sync(CT_FULL, !(tmax <= (R)kBlockMax))) {
    jacobi_block();
    return;
  }
  store_block_row<R>(out, lane, row);
  if (i < N) bsum[i] = rs;
}

__global__ void k_precond_mark(const long long* __restrict__ rebuilds, long long* __restrict__ epoch) {
  *epoch = *rebuilds;
}

template <class R>
void launch_block_setup(const DevState& S, cudaStream_t st) {
  if (S.N == 0) return;
  int nb = (S.N + 31) / 32;
  k_block_setup<R><<<(nb + 3) / 4, 128, 0, st>>>(S.N, S.ld, S.nl, S.nmat, S.M, (const R*)S.Dg,
                                                 (typename BlockStore<R>::T*)S.binv,
                                                 (R*)S.bsum, S.rebuild_count, S.precond_epoch);
  k_precond_mark<<<1, 1, 0, st>>>(S.rebuild_count, S.precond_epoch);
}

// y = M_b^-1 r for the warp's block: every lane of a full warp, i = 32b +
// lane, r_i of this lane (zero where no atom).
// The block is stored row by row (row a = element (a, j) for j = 0..31,
// contiguous), so a lane reads its row with 16-byte loads (4 in FP16, 16 in
// FP64; the inverse is symmetric, so the row is also the column).
template <class R>
__device__ inline R block_apply(const typename BlockStore<R>::T* __restrict__ binv, int i, R ri) {
  using BT = typename BlockStore<R>::T;
  constexpr int NV = 32 * (int)sizeof(BT) / 16;
  const uint4* rp = reinterpret_cast<const uint4*>(binv + (size_t)(i >> 5) * 1024 + (size_t)(i & 31) * 32);
  union {
    uint4 v[NV];
    BT b[32];
  } row;
#pragma unroll
  for (int k = 0; k < NV; ++k) row.v[k] = __ldg(rp + k);   // all in flight
  R y = R(0);
#pragma unroll
  for (int j = 0; j < 32; ++j) y += (R)blk_unpack(row.b[j]) * __shfl_sync(CT_FULL, ri, j);
  return y;
}

// Starting guess (extrapolated from the stored solutions, zero without
// history), its working-precision copy for the gathers, d = D^-1 1 and the
// guess's total per replica; shifts the history (h2 <- h1, h1 <- the last
// solution). The last block turns the totals into the uniform shift that
// puts the guess on sum q = Q.
template <class R>
__global__ void k_cg_extrap(int N, double* __restrict__ q, double* __restrict__ h1, double* __restrict__ h2,
                            R* __restrict__ qr, const R* __restrict__ dinv, R* __restrict__ d,
                            const int* __restrict__ rep, double* __restrict__ cg, int Rn,
                            const int* __restrict__ hist, int* __restrict__ blocks) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  RepAcc<1> acc;
  acc.init();
  if (i < N) {
    int nh = *hist;
    double qo = q[i], a = h1[i], b = h2[i], q0;
    if (nh >= 3) q0 = 3.0 * qo - 3.0 * a + b;
    else if (nh == 2) q0 = 2.0 * qo - a;
    else if (nh == 1) q0 = qo;
    else q0 = 0.0;
    h2[i] = a;
    h1[i] = qo;
    q[i] = q0;
    qr[i] = (R)q0;
    d[i] = dinv[i];
    acc.to(rep[i], cg + CG_SQ0, CG_STRIDE);
    acc.v[0] += q0;
  }
  lane_flush<1>(acc, cg + CG_SQ0, CG_STRIDE);
  if (last_block(blocks)) {
    for (int r = threadIdx.x; r < Rn; r += blockDim.x) {
      double* c = cg + (size_t)r * CG_STRIDE;
      double nat = c[CG_NAT];
      c[CG_DQ] = nat > 0 ? (c[CG_Q] - ldcg(c + CG_SQ0)) / nat : 0.0;
    }
    if (threadIdx.x == 0) blocks[0] = 0;
  }
}

// Row sums sum_e M_e v_j(e) of atom i over its column of the list, for one
// or two gathered vectors (NV = 1, 2), plus sum_e M_e (NV = 3). In FP32 the
// products are summed with compensation: a plain FP32 sum of ~230 terms
// whose partial sums are much larger than the result limits the reachable
// residual of the charge solve (about 1e-4 eV/e); compensated, the limit is
// the rounding of the stored entries.
template <class R>
struct RowAcc {
  R s = R(0), c = R(0);
  __device__ inline void add(R x) {
    if (sizeof(R) == 4) {
      R t = s + x;
      c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
      s = t;
    } else {
      s += x;
    }
  }
  __device__ inline R value() const { return s + c; }
};

// Row sum sum_e M_e x_j(e) of atom i for the matrix pass, software-pipelined:
// the list indices and entries of the next B entries are loaded before the
// current batch's x_j are gathered, so the streamed list (the bound of this
// pass) always has loads in flight. Each batch is summed as a small tree and
// only the running sum is compensated: the error that limits the solve
// comes from adding small terms to a large running sum, not from the few
// terms of a batch. B (entries in flight per thread) is chosen at run time
// by tune_cg_mv among the instantiated depths.
template <class R, int B>
__device__ inline R row_sum_stream(int i, int na, int ld, const int2* __restrict__ nl, const void* __restrict__ M,
                                   const R* __restrict__ x) {
  const MatView<R> mat(nl, M);
  int jn[B];
  R mn[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    jn[k] = i;
    mn[k] = R(0);
    if (k < na) mat.get((size_t)k * ld + i, jn[k], mn[k]);
  }
  RowAcc<R> acc;
  for (int e = 0; e < na; e += B) {
    int jc[B];
    R mc[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      jc[k] = jn[k];
      mc[k] = mn[k];
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      int en = e + B + k;
      jn[k] = i;
      mn[k] = R(0);
      if (en < na) mat.get((size_t)en * ld + i, jn[k], mn[k]);
    }
    R t[B];
#pragma unroll
    for (int k = 0; k < B; ++k) t[k] = mc[k] * __ldg(x + jc[k]);
#pragma unroll
    for (int w = 1; w < B; w <<= 1)
#pragma unroll
      for (int k = 0; k + w < B; k += 2 * w) t[k] += t[k + w];
    acc.add(t[0]);
  }
  return acc.value();
}

// The start of a solve needs three row sums at once: sum M q0_j, sum M d_j
// and sum M (for the uniform shift of the guess), streamed like the matrix
// pass (the next B entries loaded ahead), compensated running sums.
template <class R, int B>
__device__ inline void row_sum_stream3(int i, int na, int ld, const int2* __restrict__ nl, const void* __restrict__ M,
                                       const R* __restrict__ x0, const R* __restrict__ x1, R& h0, R& h1, R& hm) {
  const MatView<R> mat(nl, M);
  int jn[B];
  R mn[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    jn[k] = i;
    mn[k] = R(0);
    if (k < na) mat.get((size_t)k * ld + i, jn[k], mn[k]);
  }
  RowAcc<R> a0, a1, am;
  for (int e = 0; e < na; e += B) {
    int jc[B];
    R mc[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      jc[k] = jn[k];
      mc[k] = mn[k];
      int en = e + B + k;
      jn[k] = i;
      mn[k] = R(0);
      if (en < na) mat.get((size_t)en * ld + i, jn[k], mn[k]);
    }
    R t0[B], t1[B], tm[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      t0[k] = mc[k] * __ldg(x0 + jc[k]);
      t1[k] = mc[k] * __ldg(x1 + jc[k]);
      tm[k] = mc[k];
    }
#pragma unroll
    for (int w = 1; w < B; w <<= 1)
#pragma unroll
      for (int k = 0; k + w < B; k += 2 * w) {
        t0[k] += t0[k + w];
        t1[k] += t1[k + w];
        tm[k] += tm[k + w];
      }
    a0.add(t0[0]);
    a1.add(t1[0]);
    am.add(tm[0]);
  }
  h0 = a0.value();
  h1 = a1.value();
  hm = am.value();
}

// r = -(H q0 + chi), y = D^-1 r, v = H d, dq = 0; sums (sum y, sum r,
// sum r^2, sum d) and the maxima of r, -r for the initial test (update buffer
// 2). r is stored shifted by the previous solve's mean (-mu of that solve),
// which keeps the stored values small: in FP32 the whole mean of r (several
// eV/e) would otherwise cost about 1e-7 of it in every element. The shift
// starts the accumulated one, so mu = -(mean of stored r + shift) holds.
template <class R>
__global__ void __launch_bounds__(256)
    k_cg_init(int N, int ld, const int2* __restrict__ nl, const int* __restrict__ nmat,
                          const void* __restrict__ M, const R* __restrict__ Dg, const R* __restrict__ dinv,
                          const typename BlockStore<R>::T* __restrict__ binv,
                          const int* __restrict__ type, const int* __restrict__ rep, TypeParams T,
                          double* __restrict__ q, const R* __restrict__ qr, const R* __restrict__ d,
                          R* __restrict__ r, R* __restrict__ y, R* __restrict__ v, R* __restrict__ dqv,
                          double* __restrict__ cg,
                          unsigned long long* __restrict__ rmax, int Rn, int* __restrict__ conv, int* __restrict__ iters,
                          int* __restrict__ blocks, int* __restrict__ active, double tol,
                          const double* __restrict__ rhs) {
  const int ub = CG_UPD + 2 * 4;
  LaneMax<R> lm;
  R part[3] = {R(0), R(0), R(0)};   // sum y, sum r, sum r^2
  R pd[1] = {R(0)};                 // sum d
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int rid = i < N ? rep[i] : -1;
  if (rid >= 0) {
    const double* cc = cg + (size_t)rid * CG_STRIDE;
    double dq = ldcg(cc + CG_DQ);
    double mp = ldcg(cc + CG_MU);
    double s0 = isfinite(mp) ? -mp : 0.0;
    R hq, hd, hm;
    row_sum_stream3<R, 8>(i, nmat[i], ld, nl, M, qr, d, hq, hd, hm);
    R Di = Dg[i], di = d[i];
    // the guess shifted by dq: H (q0 + dq 1) = D (q0 + dq) + sum M q0_j + dq sum M
    double qi = q[i] + dq;
    q[i] = qi;
    double chi_i = rhs ? rhs[i] : by_type(T.chi, type[i]);   // rhs: a per-atom chi (adjoint solves)
    R ri = (R)(-chi_i - ((double)Di * qi + (double)hq + dq * (double)hm) - s0);
    r[i] = ri;
    v[i] = Di * di + hd;
    dqv[i] = R(0);
    part[1] = ri;
    part[2] = ri * ri;
    pd[0] = di;
    lm.add(rid, ri, rmax + 2 * 2);
  }
  {
    // y = M^-1 r (the block product takes every lane of the warp)
    R ri = rid >= 0 ? r[i] : R(0);
    R yi = binv ? block_apply(binv, i, ri) : (rid >= 0 ? dinv[i] * ri : R(0));
    if (rid >= 0) {
      y[i] = yi;
      part[0] = yi;
    }
  }
  flush_values<R, 3>(rid, part, cg + ub, CG_STRIDE);
  flush_values<R, 1>(rid, pd, cg + CG_SD, CG_STRIDE);
  lm.finish(rmax + 2 * 2);
  if (last_block(blocks)) {
    for (int rr = threadIdx.x; rr < Rn; rr += blockDim.x) {
      double* cc = cg + (size_t)rr * CG_STRIDE;
      double mp = cc[CG_MU];
      cc[CG_SHIFT] = isfinite(mp) ? -mp : 0.0;   // the shift every thread applied
    }
    __syncthreads();
    int all = check_replicas(Rn, cg, rmax, conv, iters, ub, 2, 0, tol, 1);
    if (threadIdx.x == 0) {
      blocks[0] = 0;
      if (all) *active = 0;
    }
  }
}

// w = H z = H y - c v with z = y - c d, and the dots (r.z, w.z); the last
// block turns them into the step lengths alpha, beta of this iteration.
// r.z is formed from r - mean(r): rounding leaves sum z slightly off zero,
// and before the first re-centring r carries its whole mean (-mu), whose
// product with that sum would swamp r.z once the residual is small (warm
// starts near the tolerance then diverge).
template <class R, int B>
__global__ void __launch_bounds__(256)
    k_cg_mv(int N, int ld, const int2* __restrict__ nl, const int* __restrict__ nmat, const void* __restrict__ M,
            const R* __restrict__ Dg, const int* __restrict__ rep, const int* __restrict__ conv,
            const int* __restrict__ itp, const R* __restrict__ y, const R* __restrict__ d, const R* __restrict__ v,
            const R* __restrict__ r, R* __restrict__ w, double* __restrict__ cg, int Rn,
            int* __restrict__ blocks, const int* __restrict__ active) {
  if (*active == 0) return;
  int it = *itp;
  int buf = CG_DOTS + (it & 1) * 2;
  R dots[2] = {R(0), R(0)};
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int rid = i < N ? rep[i] : -1;
  if (rid >= 0 && !conv[rid]) {
    const double* cc = cg + (size_t)rid * CG_STRIDE;
    R c = (R)ldcg(cc + CG_C);
    R m = (R)ldcg(cc + CG_M);   // mean of the stored r
    R hy = row_sum_stream<R, B>(i, nmat[i], ld, nl, M, y);
    R yi = y[i];
    R zi = yi - c * d[i];
    R wi = Dg[i] * yi + hy - c * v[i];
    w[i] = wi;
    dots[0] = (r[i] - m) * zi;   // r.z
    dots[1] = wi * zi;           // w.z
  } else {
    rid = -1;
  }
  flush_values<R, 2>(rid, dots, cg + buf, CG_STRIDE);
  if (last_block(blocks + 2)) {
    int sprev = CG_SCAL + ((it + 1) & 1) * 2;
    int scur = CG_SCAL + (it & 1) * 2;
    for (int rr = threadIdx.x; rr < Rn; rr += blockDim.x) {
      if (conv[rr]) continue;
      double* cc = cg + (size_t)rr * CG_STRIDE;
      double g = ldcg(cc + buf + 0), dd = ldcg(cc + buf + 1);
      double a = 0.0, b = 0.0;
      if (it == 0) {
        a = dd != 0.0 ? g / dd : 0.0;
      } else {
        double gp = cc[sprev], ap = cc[sprev + 1];
        b = gp != 0.0 ? g / gp : 0.0;
        double den = dd - (ap != 0.0 ? b * g / ap : 0.0);
        a = den != 0.0 ? g / den : 0.0;
      }
      cc[CG_AB] = a;
      cc[CG_AB + 1] = b;
      cc[scur] = g;
      cc[scur + 1] = a;
    }
    if (threadIdx.x == 0) blocks[2] = 0;
  }
}

// Element-wise update; the sums and maxima for the next c and the test.
// Threads take 256-atom tiles strided over the grid; per-thread partial sums
// in the working precision (a few atoms each), FP64 across warps and blocks.
// The iterate's change dq = q - q0 is accumulated in the working precision
// (it is small next to q) and added to the FP64 q once, after the loop, so
// the loop issues no FP64 arithmetic per atom.
template <class R>
__global__ void __launch_bounds__(256)
    k_cg_up(int N, const int* __restrict__ rep, const R* __restrict__ dinv,
            const typename BlockStore<R>::T* __restrict__ binv,
            int* __restrict__ conv,
            int* __restrict__ iters, int* __restrict__ itp, const R* __restrict__ w, const R* __restrict__ d,
            R* __restrict__ dqv, R* __restrict__ r, R* __restrict__ p, R* __restrict__ s,
            R* __restrict__ y, double* __restrict__ cg, unsigned long long* __restrict__ rmax, int Rn,
            int* __restrict__ blocks, int* __restrict__ active, unsigned* __restrict__ err, double tol,
            int max_iter, int use_cond, cudaGraphConditionalHandle cond) {
  if (*active == 0) {
    // nothing left to do (converged at the start): end the loop
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  int it = *itp;
  int mb = it % 3;
  int ubuf = CG_UPD + mb * 4;
  // zero the buffers the next iteration accumulates into
  if (blockIdx.x == 0) {
    int dn = CG_DOTS + ((it + 1) & 1) * 2, un = CG_UPD + ((it + 1) % 3) * 4, mn = (it + 1) % 3;
    for (int k = threadIdx.x; k < Rn * 8; k += blockDim.x) {
      int rr = k / 8, kk = k % 8;
      double* c = cg + (size_t)rr * CG_STRIDE;
      if (kk < 2) c[dn + kk] = 0.0;
      else if (kk < 6) c[un + kk - 2] = 0.0;
      else rmax[(size_t)rr * 6 + mn * 2 + (kk - 6)] = 0ull;
    }
  }
  LaneMax<R> lm;
  int crid = -1;
  R a = R(0), b = R(0), c = R(0), mprev = R(0);
  R part[3] = {R(0), R(0), R(0)};   // sum y, sum r, sum r^2
  for (int t = blockIdx.x; (long long)t * 256 < N; t += gridDim.x) {
    int i = t * 256 + (int)threadIdx.x;
    int rid = i < N ? rep[i] : -1;
    bool act = rid >= 0 && !conv[rid];
    R ri = R(0);
    if (act && rid != crid) {
      if (crid >= 0) {   // a replica boundary in this thread's atoms
        double* o = cg + (size_t)crid * CG_STRIDE + ubuf;
        for (int k = 0; k < 3; ++k) atomicAdd(o + k, (double)part[k]);
        part[0] = part[1] = part[2] = R(0);
      }
      const double* cc = cg + (size_t)rid * CG_STRIDE;
      a = (R)ldcg(cc + CG_AB);
      b = (R)ldcg(cc + CG_AB + 1);
      c = (R)ldcg(cc + CG_C);
      mprev = (R)ldcg(cc + CG_M);
      crid = rid;
    }
    if (act) {
      R zi = y[i] - c * d[i];   // the same z as the matrix pass formed
      R pi = zi + b * p[i];
      R si = w[i] + b * s[i];
      ri = (r[i] - a * si) - mprev;
      p[i] = pi;
      s[i] = si;
      dqv[i] += a * pi;
      r[i] = ri;
    }
    // y = M^-1 r: the block product takes every lane of the warp (blocks do
    // not couple replicas, so a converged replica's lanes enter with r = 0)
    R yi = binv ? block_apply(binv, i, ri) : (act ? dinv[i] * ri : R(0));
    if (act) {
      y[i] = yi;
      part[0] += yi;
      part[1] += ri;
      part[2] += ri * ri;
      lm.add(rid, ri, rmax + mb * 2);
    }
  }
  flush_values<R, 3>(crid, part, cg + ubuf, CG_STRIDE);
  lm.finish(rmax + mb * 2);
  if (last_block(blocks + 1)) {
    // the mean this launch subtracted joins the accumulated shift (the value
    // every thread used is still in CG_M)
    for (int rr = threadIdx.x; rr < Rn; rr += blockDim.x)
      if (!conv[rr]) {
        double* cc = cg + (size_t)rr * CG_STRIDE;
        cc[CG_SHIFT] += (double)(R)cc[CG_M];
      }
    __syncthreads();
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

// sum_i (q_i + dq_i) per replica: the iterate's total before the final
// shift.
template <class R>
__global__ void __launch_bounds__(256) k_cg_qsum(int N, const int* __restrict__ rep, const double* __restrict__ q,
                                                 const R* __restrict__ dqv, double* __restrict__ cg) {
  RepAcc<1> acc;
  acc.init();
  for (int t = blockIdx.x; (long long)t * 256 < N; t += gridDim.x) {
    int i = t * 256 + (int)threadIdx.x;
    if (i >= N) break;
    acc.to(rep[i], cg + CG_SQF, CG_STRIDE);
    acc.v[0] += q[i] + (double)dqv[i];
  }
  lane_flush<1>(acc, cg + CG_SQF, CG_STRIDE);
}

// q <- q + dq, shifted uniformly onto sum q = Q exactly (rounding of y and d
// keeps sum z, and so the iterate's total, from being exact); the
// working-precision copy for the force passes; the solve's iteration count
// and its history.
template <class R>
__global__ void k_cg_final(int N, const int* __restrict__ rep, const double* __restrict__ cg,
                           double* __restrict__ q, const R* __restrict__ dqv, R* __restrict__ qr,
                           const int* __restrict__ itp, long long* __restrict__ total, int* __restrict__ hist) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *total += *itp;
    int h = *hist;
    *hist = h < 3 ? h + 1 : 3;
  }
  if (i < N) {
    const double* c = cg + (size_t)rep[i] * CG_STRIDE;
    double nat = c[CG_NAT];
    double shift = nat > 0 ? (c[CG_Q] - c[CG_SQF]) / nat : 0.0;
    double qi = q[i] + (double)dqv[i] + shift;
    q[i] = qi;
    qr[i] = (R)qi;
  }
}

// Working-precision copy of charges set from outside the solve.
template <class R>
__global__ void k_copy_q(int N, const double* __restrict__ q, R* __restrict__ qr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) qr[i] = (R)q[i];
}

// --------------------------------------------------------------- launchers
template <class R>
void launch_cg_begin(const DevState& S, const TypeParams& T, cudaStream_t st, double tol, const double* rhs) {
  k_cg_prep<<<1, 256, 0, st>>>(S.N, S.R, S.cg, S.cg_rmax, S.cg_conv, S.cg_iters, S.cg_it, S.cg_blocks, S.cg_active);
  if (S.N == 0) return;
  const auto* binv = S.precond ? (const typename BlockStore<R>::T*)S.binv : nullptr;
  k_cg_extrap<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.q, S.cqh1, S.cqh2, (R*)S.qr,
                                                    (const R*)(S.precond ? S.bsum : S.dinv),
                                                    (R*)S.cd, S.rep, S.cg, S.R, S.cg_hist, S.cg_blocks);
  k_cg_init<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.ld, S.nl, S.nmat, S.M, (const R*)S.Dg,
                                     (const R*)S.dinv, binv, S.type, S.rep, T, S.q, (const R*)S.qr, (const R*)S.cd,
                                     (R*)S.cr, (R*)S.cy, (R*)S.cv, (R*)S.cdq, S.cg, S.cg_rmax, S.R, S.cg_conv, S.cg_iters,
                                     S.cg_blocks, S.cg_active, tol, rhs);
}

template <class R, int B>
static void launch_cg_mv_b(const DevState& S, cudaStream_t st) {
  k_cg_mv<R, B><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.ld, S.nl, S.nmat, S.M, (const R*)S.Dg, S.rep,
                                                   S.cg_conv, S.cg_it, (const R*)S.cy, (const R*)S.cd,
                                                   (const R*)S.cv, (const R*)S.cr, (R*)S.cw, S.cg, S.R,
                                                   S.cg_blocks, S.cg_active);
}

template <class R>
void launch_cg_mv(const DevState& S, cudaStream_t st) {
  if (S.N == 0) return;
  if (S.mv_batch == 4) launch_cg_mv_b<R, 4>(S, st);
  else if (S.mv_batch == 8) launch_cg_mv_b<R, 8>(S, st);
  else launch_cg_mv_b<R, 16>(S, st);
}

// Autotuner of the matrix pass: times each instantiated depth (entries in
// flight per thread: 4, 8, 16) on the current lists, one warm-up and three
// timed launches each with CUDA events on the system's stream, and keeps the
// fastest in S.mv_batch. It runs the pass on whatever the CG vectors hold
// (the timing does not depend on their values) after resetting the solver's
// per-solve state, which every solve resets again anyway. Returns the
// milliseconds per launch of each depth in ms_out[3].
template <class R>
cudaError_t tune_cg_mv(DevState& S, cudaStream_t st, float* ms_out) {
  if (S.N == 0) return cudaSuccess;
  const int depth[3] = {4, 8, 16};
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  float best = 1e30f;
  int pick = 16;
  // the solver state the timing runs overwrite (per-replica scalars and
  // maxima, convergence flags, counters), kept and put back
  const size_t ncg = (size_t)S.R * CG_STRIDE * sizeof(double), nrm = (size_t)S.R * 6 * sizeof(unsigned long long);
  const size_t nri = (size_t)S.R * sizeof(int);
  char* keep = nullptr;
  e = cudaMallocAsync(&keep, ncg + nrm + 2 * nri + 5 * sizeof(int), st);
  auto save = [&](bool back) {
    char* p = keep;
    auto mv = [&](void* dev, size_t n) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(back ? dev : p, back ? p : dev, n, cudaMemcpyDeviceToDevice, st);
      p += n;
    };
    mv(S.cg, ncg);
    mv(S.cg_rmax, nrm);
    mv(S.cg_conv, nri);
    mv(S.cg_iters, nri);
    mv(S.cg_it, sizeof(int));
    mv(S.cg_active, sizeof(int));
    mv(S.cg_blocks, 3 * sizeof(int));
  };
  save(false);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    S.mv_batch = depth[k];
    k_cg_prep<<<1, 256, 0, st>>>(S.N, S.R, S.cg, S.cg_rmax, S.cg_conv, S.cg_iters, S.cg_it, S.cg_blocks, S.cg_active);
    launch_cg_mv<R>(S, st);
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 3; ++rep) launch_cg_mv<R>(S, st);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.0f;
    if (ms_out) ms_out[k] = ms;
    if (ms < best) { best = ms; pick = depth[k]; }
  }
  save(true);
  if (keep) cudaFreeAsync(keep, st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.mv_batch = pick;
  return e == cudaSuccess ? cudaGetLastError() : e;
}

template <class R>
void launch_cg_up(const DevState& S, const SolveCfg& cfg, cudaStream_t st) {
  // launched even without atoms: inside the graph's WHILE node this kernel
  // is what ends the loop (it finds the loop inactive and clears the
  // condition)
  int grid = stride_grid(S.N, S.nsm, (const void*)k_cg_up<R>);
  k_cg_up<R><<<grid, 256, 0, st>>>(S.N, S.rep, (const R*)S.dinv,
                                   S.precond ? (const typename BlockStore<R>::T*)S.binv : nullptr,
                                   S.cg_conv, S.cg_iters, S.cg_it, (const R*)S.cw,
                                   (const R*)S.cd, (R*)S.cdq, (R*)S.cr, (R*)S.cp, (R*)S.cs, (R*)S.cy, S.cg, S.cg_rmax,
                                   S.R, S.cg_blocks, S.cg_active, S.err, cfg.tol, cfg.max_iter, cfg.use_cond,
                                   cfg.cond);
}

template <class R>
void launch_cg_iter(const DevState& S, const SolveCfg& cfg, cudaStream_t st) {
  launch_cg_mv<R>(S, st);
  launch_cg_up<R>(S, cfg, st);
}

template <class R>
void launch_cg_end(const DevState& S, cudaStream_t st) {
  if (S.N > 0) {
    int grid = stride_grid(S.N, S.nsm, (const void*)k_cg_qsum<R>);
    k_cg_qsum<R><<<grid, 256, 0, st>>>(S.N, S.rep, S.q, (const R*)S.cdq, S.cg);
  }
  int n = S.N > 0 ? S.N : 1;
  k_cg_final<R><<<(n + 255) / 256, 256, 0, st>>>(S.N, S.rep, S.cg, S.q, (const R*)S.cdq, (R*)S.qr, S.cg_it,
                                                 S.cg_total, S.cg_hist);
}

template <class R>
void launch_copy_q(const DevState& S, cudaStream_t st) {
  if (S.N == 0) return;
  k_copy_q<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.q, (R*)S.qr);
}

template void launch_block_setup<float>(const DevState&, cudaStream_t);
template void launch_block_setup<double>(const DevState&, cudaStream_t);
template void launch_cg_begin<float>(const DevState&, const TypeParams&, cudaStream_t, double, const double*);
template void launch_cg_begin<double>(const DevState&, const TypeParams&, cudaStream_t, double, const double*);
template void launch_cg_mv<float>(const DevState&, cudaStream_t);
template cudaError_t tune_cg_mv<float>(DevState&, cudaStream_t, float*);
template cudaError_t tune_cg_mv<double>(DevState&, cudaStream_t, float*);
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
