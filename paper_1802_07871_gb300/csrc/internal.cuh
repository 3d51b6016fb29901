// internal.cuh — device-side types and helpers shared by the libctbop kernels.
//
// Layout (all device memory, N atoms, R replicas):
//   x, v, F          double[N*3]   master positions / velocities / forces
//   q                double[N]     charges
//   type, rep        int32[N]      atom type (0 Si, 1 C), replica id
//   cell4            int4[N]       cell coordinates (x,y,z) and global cell id, fixed between rebuilds
//   u                Real4[N]      position relative to the owning cell's origin (w = type)
//   nl               int2[cap*ld]  one list per atom of (j, code) pairs, column-major: entry e of
//                                  atom i at e*ld + i (ld = N rounded up to 32), so a warp reading
//                                  entry e of 32 consecutive atoms touches 256 contiguous bytes. Entries
//                                  [0, ncov) are the covalent list (r < S + skin), [ncov, nfix)
//                                  the core (r < Rc - skin when built, so inside Rc until the next
//                                  rebuild) and [nfix, nall) the shell, the rest inside Rc + skin
//   code             packed cell offset (dx,dy,dz) such that r_ij = u_j - u_i + d*h
//   rev              int32[N*capc] entry of j's list that points back to i (covalent part)
//   bo               Real4[N*capc] b_ij, db/dzeta_1, db/dzeta_2 per directed bond
//   gslot            Real4[N*capc] dE_i/du_e: gradient of the terms centred on i w.r.t. bond e
//   M                [cap*ld]      charge-Hessian off-diagonal entries K_ij - 2 w_ij (list layout):
//                                  FP32 (j, coefficient) int2 pairs, or FP64 coefficients
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define CT_WARP 32
#define CT_FULL 0xffffffffu

// device error bits
#define CT_ERR_NBR_OVERFLOW 1u
#define CT_ERR_COV_OVERFLOW 2u
#define CT_ERR_REV_MISSING 4u
#define CT_ERR_NONFINITE 8u
#define CT_ERR_CG_MAXITER 16u
#define CT_ERR_CODE_RANGE 32u

namespace ct {

template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };
template <class R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// Potential parameters in the working precision, passed by value to kernels.
template <class R> struct PotParams {
  // pair block [ti*2+tj]
  R A[4], B[4], lam1[4], lam2[4], Rin[4], Sout[4], kappa[4], pi_SR[4];
  R rcov_list2[4];                 // (S + skin)^2, covalent list radius squared
  // bond order block [ti*2+tj]
  R sigma[4], p[4], g1[4], g2[4], n1[4], n2[4], G[4], inv2s[4], inv2sp[4];
  // triplet block [(ti*2+tj)*2+tk][l]
  R gam[8][2], c2[8][2], d2[8][2], h[8][2], alpha[8][2], c2d2[8][2];
  // charge kernel
  R gshield3[4];                   // (gamma_i gamma_j)^(-3/2)
  R rcoul, inv_rcoul, ke;
  R rall_list2;                    // (Rc + skin)^2
  R rcore_list2;                   // (Rc - skin)^2 (0 if Rc <= skin): entries inside stay inside Rc
                                   // until the next rebuild
  // the pair block in FP64, for the stiff-bond pair terms of the FP32 path
  double A64[4], B64[4], lam1_64[4], lam2_64[4], Rin64[4], Sout64[4], kappa64[4];
};

// Per-type quantities that always stay double.
struct TypeParams {
  double E0[2], chi[2], J[2], inv_mass_acc[2], mass[2];
};

// Element t (0 or 1) of a two-entry kernel-parameter array: a select, not
// an indexed load (an indexed parameter array is copied to local memory).
template <class V>
__host__ __device__ inline V by_type(const V (&a)[2], int t) {
  return t ? a[1] : a[0];
}

// One replica's box and cell grid.
struct RepInfo {
  double L[3];        // box lengths (binning extent along open axes)
  double hc[3];       // cell edge
  float hcf[3];
  int pbc[3];
  int n[3];           // cells per axis
  int m[3];           // stencil half width per axis
  int cell_off;       // first global cell id
  int atom_off;       // first atom
  int natoms;
};

__host__ __device__ inline int pack_code(int dx, int dy, int dz) {
  return (dx + 512) | ((dy + 512) << 10) | ((dz + 512) << 20);
}
__host__ __device__ inline void unpack_code(int c, int& dx, int& dy, int& dz) {
  dx = (c & 1023) - 512;
  dy = ((c >> 10) & 1023) - 512;
  dz = ((c >> 20) & 1023) - 512;
}

template <class R> __device__ inline R ct_exp(R x);
template <> __device__ inline float ct_exp<float>(float x) { return expf(x); }
template <> __device__ inline double ct_exp<double>(double x) { return exp(x); }
template <class R> __device__ inline R ct_pow(R x, R y);
template <> __device__ inline float ct_pow<float>(float x, float y) { return powf(x, y); }
template <> __device__ inline double ct_pow<double>(double x, double y) { return pow(x, y); }
template <class R> __device__ inline R ct_sqrt(R x);
template <> __device__ inline float ct_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ inline double ct_sqrt<double>(double x) { return sqrt(x); }
template <class R> __device__ inline R ct_cbrt(R x);
template <> __device__ inline float ct_cbrt<float>(float x) { return cbrtf(x); }
template <> __device__ inline double ct_cbrt<double>(double x) { return cbrt(x); }
template <class R> __device__ inline R ct_rsqrt(R x);
template <> __device__ inline float ct_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double ct_rsqrt<double>(double x) { return 1.0 / sqrt(x); }
template <class R> __device__ inline R ct_rcbrt(R x);
// x^(-1/3) in FP32 for positive normal x (the charge kernel's
// r^3 + gamma^-3, a few to a few hundred): a first guess 2^(-log2(x)/3) from
// the hardware base-2 logarithm and exponential (relative error near 2^-21),
// then one Newton step for f(y) = y^-3 - x, written as a small correction,
// y <- y + y (1 - x y^3) / 3, which squares that error and rounds once at
// the end; the result is within about one ulp (checked against the library
// rcbrtf and an FP64 reference by the tests).
__device__ inline float rcbrt_newton(float x) {
  float l, y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  l *= -0.333333343f;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l));
  float e = fmaf(-x, y * y * y, 1.0f);
  return fmaf(y * 0.333333343f, e, y);
}
template <> __device__ inline float ct_rcbrt<float>(float x) { return rcbrt_newton(x); }
template <> __device__ inline double ct_rcbrt<double>(double x) { return 1.0 / cbrt(x); }
template <class R> __device__ inline R ct_cospi(R x);
template <> __device__ inline float ct_cospi<float>(float x) { return cospif(x); }
template <> __device__ inline double ct_cospi<double>(double x) { return cospi(x); }
template <class R> __device__ inline R ct_sinpi(R x);
template <> __device__ inline float ct_sinpi<float>(float x) { return sinpif(x); }
template <> __device__ inline double ct_sinpi<double>(double x) { return sinpi(x); }

// Tersoff cutoff and its derivative. In the taper, 1/2 [1 + cos(pi t)] is
// evaluated as cos^2(pi t / 2) and its derivative from sin(pi t / 2) and
// cos(pi t / 2): the sum 1 + cos(pi t) cancels near t = 1 (a pair just inside
// S), where FP32 then lost five digits of f_c (relative error 1e-5 at
// f_c = 3e-3); through zeta^n with n < 1, whose derivative grows without
// bound as zeta -> 0, that error reached the forces of atoms with a single
// neighbour in the taper.
template <class R>
__device__ inline void cutoff_fn(R r, R Rin, R Sout, R pi_SR, R& f, R& df) {
  if (r < Rin) { f = R(1); df = R(0); return; }
  if (r >= Sout) { f = R(0); df = R(0); return; }
  R h = R(0.5) * (r - Rin) / (Sout - Rin);
  R c = ct_cospi<R>(h), s = ct_sinpi<R>(h);
  f = c * c;
  df = -pi_SR * s * c;
}

// Shielded, tapered charge kernel K(r) and dK/dr.
template <class R>
__device__ inline void coul_fn(R r, R gs3, R inv_rc, R ke, R& K, R& dK) {
  R x = r * inv_rc;
  if (x >= R(1)) { K = R(0); dK = R(0); return; }
  R x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
  R T = R(1) + x4 * (R(-35) + x * (R(84) + x * (R(-70) + R(20) * x)));
  R xm = x - R(1);
  R dT = R(140) * x3 * xm * xm * xm;
  R r3 = r * r * r;
  R D = ct_cbrt<R>(r3 + gs3);
  R iD = R(1) / D;
  K = ke * T * iD;
  R iD3 = iD * iD * iD;
  dK = ke * (dT * inv_rc * iD - T * r * r * iD3 * iD);
}

// The same K(r) from r^2 for the streamed passes: 1/r and 1/(r^3 +
// gamma^-3)^(1/3) come from the reciprocal root functions (FP32 path) instead
// of a root and a division each. Returns r, 1/r, K and K'(r)/r.
template <class R>
__device__ inline void coul_fn_r2(R r2, R gs3, R inv_rc, R ke, R& r, R& ir, R& K, R& dK_r) {
  ir = ct_rsqrt<R>(r2);
  r = r2 * ir;
  R x = r * inv_rc;
  if (x >= R(1)) { K = R(0); dK_r = R(0); return; }
  R x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
  R T = R(1) + x4 * (R(-35) + x * (R(84) + x * (R(-70) + R(20) * x)));
  R xm = x - R(1);
  R dT = R(140) * x3 * xm * xm * xm;
  R iD = ct_rcbrt<R>(r2 * r + gs3);
  K = ke * T * iD;
  R iD3 = iD * iD * iD;
  dK_r = ke * (dT * inv_rc * iD * ir - T * r * iD3 * iD);
}
template <class R>
__device__ inline R coul_K_r2(R r2, R gs3, R inv_rc, R ke) {
  R r = r2 * ct_rsqrt<R>(r2);
  R x = r * inv_rc;
  if (x >= R(1)) return R(0);
  R x4 = (x * x) * (x * x);
  R T = R(1) + x4 * (R(-35) + x * (R(84) + x * (R(-70) + R(20) * x)));
  return ke * T * ct_rcbrt<R>(r2 * r + gs3);
}

// The stored charge matrix, one entry per list entry (e * ld + i). The FP32
// path keeps (j, coefficient bits) pairs, so a matrix pass streams one
// 8-byte load per entry instead of two 4-byte streams; the FP64 path keeps
// the FP64 coefficients beside the index list.
template <class R> struct MatView;
template <> struct MatView<float> {
  const int2* ml;
  __device__ MatView(const int2* /*nl*/, const void* m) : ml(static_cast<const int2*>(m)) {}
  __device__ inline void get(size_t idx, int& j, float& v) const {
    int2 t = __ldg(ml + idx);
    j = t.x;
    v = __int_as_float(t.y);
  }
};
template <> struct MatView<double> {
  const int2* nl;
  const double* M;
  __device__ MatView(const int2* n, const void* m) : nl(n), M(static_cast<const double*>(m)) {}
  __device__ inline void get(size_t idx, int& j, double& v) const {
    j = __ldg(&nl[idx].x);
    v = __ldg(M + idx);
  }
};
__device__ inline void mat_store(void* M, size_t idx, int j, float v) {
  static_cast<int2*>(M)[idx] = make_int2(j, __float_as_int(v));
}
__device__ inline void mat_store(void* M, size_t idx, int /*j*/, double v) { static_cast<double*>(M)[idx] = v; }

// Compensated (Neumaier) summation in the working precision: keeps the
// rounding of long per-lane sums at the level of a single term.
template <class R> struct CompSum {
  R s = R(0), c = R(0);
  __device__ inline void add(R x) {
    R t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ inline double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------- reductions
// Accumulate NV doubles per replica. Each warp keeps a running partial for
// the replica it is on and flushes with atomics when the replica changes; the
// block merges its warps' final partials so a block that stays inside one
// replica issues NV atomics in total.
template <int NV>
struct RepAcc {
  int rep;
  double v[NV];
  __device__ inline void init() {
    rep = -1;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
  }
  __device__ inline void flush(double* out, int stride) {
    if (rep >= 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (v[k] != 0.0) atomicAdd(out + (size_t)rep * stride + k, v[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
  }
  // lane 0 only: switch to replica r, flushing the old partial
  __device__ inline void to(int r, double* out, int stride) {
    if (r != rep) { flush(out, stride); rep = r; }
  }
};

template <int NV>
__device__ inline void block_flush(RepAcc<NV>& acc, double* out, int stride) {
  // acc is valid on lane 0 of every warp
  __shared__ int s_rep[32];
  __shared__ double s_v[32][NV];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int nw = blockDim.x >> 5;
  if (lane == 0) {
    s_rep[warp] = acc.rep;
#pragma unroll
    for (int k = 0; k < NV; ++k) s_v[warp][k] = acc.v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = -1;
    double sum[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) sum[k] = 0.0;
    for (int w = 0; w < nw; ++w) {
      int r = s_rep[w];
      if (r < 0) continue;
      if (r != cur) {
        if (cur >= 0)
          for (int k = 0; k < NV; ++k)
            if (sum[k] != 0.0) atomicAdd(out + (size_t)cur * stride + k, sum[k]);
        cur = r;
        for (int k = 0; k < NV; ++k) sum[k] = 0.0;
      }
      for (int k = 0; k < NV; ++k) sum[k] += s_v[w][k];
    }
    if (cur >= 0)
      for (int k = 0; k < NV; ++k)
        if (sum[k] != 0.0) atomicAdd(out + (size_t)cur * stride + k, sum[k]);
  }
  __syncthreads();
}

// End-of-kernel flush of per-lane replica partials: lanes of a warp that
// share a replica are summed with shuffles, the warps of a block merged in
// shared memory, then one atomic per value and replica.
template <int NV>
__device__ inline void lane_flush(RepAcc<NV>& a, double* out, int stride);

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CT_FULL, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CT_FULL, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(CT_FULL, v, o));
  return v;
}

template <int NV>
__device__ inline void lane_flush(RepAcc<NV>& a, double* out, int stride) {
  int lane = threadIdx.x & 31;
  int r0 = __shfl_sync(CT_FULL, a.rep, 0);
  bool same = __all_sync(CT_FULL, a.rep == r0);
  RepAcc<NV> w;
  w.init();
  if (same) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = warp_sum(a.v[k]);
      if (lane == 0) w.v[k] = t;
    }
    if (lane == 0) w.rep = r0;
  } else {
    a.flush(out, stride);
  }
  block_flush<NV>(w, out, stride);
}

// The live entries of a lane group's atom (G lanes per atom, G a power of
// two up to 32), in list order, into s_lv: entry e < nc is live when
// is_live(e). The count is returned to every lane of the group; dead(e) is
// called by the lane that tested an entry found not live. Lane l of the
// group tests e = l, l + G, ... (the entries it staged). Every lane of the
// warp takes part (ballots).
template <int G, class Live, class Dead>
__device__ inline int compact_live(bool live, int nc, int l, int* s_lv, Live is_live, Dead dead) {
  const int shift = (int)(threadIdx.x & 31) - l;   // the group's first lane in the warp
  const unsigned gm = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const int rounds = (int)__reduce_max_sync(CT_FULL, live ? (unsigned)((nc + G - 1) / G) : 0u);
  int n = 0;
  for (int r = 0; r < rounds; ++r) {
    const int e = r * G + l;
    const bool inr = live && e < nc;
    const bool lv = inr && is_live(e);
    const unsigned m = (__ballot_sync(CT_FULL, lv) >> shift) & gm;
    if (lv) s_lv[n + __popc(m & ((1u << l) - 1u))] = e;
    else if (inr) dead(e);
    n += __popc(m);
  }
  return n;
}

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

// atomic max for non-negative floats (bit patterns order like the values)
__device__ inline void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<unsigned*>(addr), __float_as_uint(v));
}

// atomic max for non-negative doubles (bit patterns order like the values)
__device__ inline void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace ct
