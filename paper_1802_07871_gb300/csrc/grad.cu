// grad.cu — derivatives of the energy with respect to the potential's
// parameters (the force-matching gradient of the differentiation pattern),
// FP64, with forward-mode tangents along a per-atom direction.
//
// At the charge minimiser the total derivative of E with respect to a
// parameter equals the partial derivative at fixed charges (the charges are
// stationary on sum q = Q, which no parameter changes), so dE/dtheta is a
// sum of per-term partial derivatives:
//   * pair terms 1/2 fc(r) [A e^{-l1 r} - c_ij b_ij B e^{-l2 r}] (A, B, l1,
//     l2, kappa, and R, S through fc);
//   * the bond order b (Eq. 7) through sigma, p, g_l, n_l, recomputing the
//     environment sums zeta_l (Eq. 2) instead of storing them;
//   * zeta_l through the triplet parameters gamma, c, d, h, alpha and through
//     the cutoff fc(r_ik) (R, S of the pair (i, k));
//   * the self energy E0 + chi q + J q^2 and the charge kernel (k_e, r_coul,
//     gamma_c).
// The gradient vector has the layout of ctbop_params (144 doubles); each
// atom's terms are weighted by a per-replica weight, so one pass gives
// sum_r a_r dE_r/dtheta.
//
// The force part of a force-matching gradient needs, for a direction g (one
// 3-vector per atom), the derivative of dE/dtheta along x + e g at fixed
// charges and the derivative of the charge gradient dE/dq = H q + chi along
// the same direction. Both come from the same kernels evaluated on dual
// numbers (value, derivative along g): every quantity that depends on the
// positions carries its exact directional derivative, with no step size.
#include <algorithm>

#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "internal.cuh"
#include "kernels.h"
#include "ctbop.h"

namespace ct {

namespace cg = cooperative_groups;

// ------------------------------------------------------------ dual numbers
// A value and its derivative along one direction, in T = float or double.
// Operators take the same T on both sides, so no double constant can slip
// into an FP32 expression.
template <class T> struct DualT {
  T v, d;
  DualT() = default;
  __device__ DualT(T x) : v(x), d(T(0)) {}
  __device__ DualT(T x, T dx) : v(x), d(dx) {}
};
template <class T> __device__ inline DualT<T> operator+(DualT<T> a, DualT<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __device__ inline DualT<T> operator-(DualT<T> a, DualT<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __device__ inline DualT<T> operator-(DualT<T> a) { return {-a.v, -a.d}; }
template <class T> __device__ inline DualT<T> operator*(DualT<T> a, DualT<T> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <class T> __device__ inline DualT<T> operator/(DualT<T> a, DualT<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> __device__ inline DualT<T> operator+(DualT<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __device__ inline DualT<T> operator+(T a, DualT<T> b) { return {a + b.v, b.d}; }
template <class T> __device__ inline DualT<T> operator-(DualT<T> a, T b) { return {a.v - b, a.d}; }
template <class T> __device__ inline DualT<T> operator-(T a, DualT<T> b) { return {a - b.v, -b.d}; }
template <class T> __device__ inline DualT<T> operator*(DualT<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __device__ inline DualT<T> operator*(T a, DualT<T> b) { return {a * b.v, a * b.d}; }
template <class T> __device__ inline DualT<T> operator/(DualT<T> a, T b) { return {a.v / b, a.d / b}; }
template <class T> __device__ inline DualT<T> operator/(T a, DualT<T> b) {
  T q = a / b.v;
  return {q, -q * b.d / b.v};
}
template <class T> __device__ inline DualT<T>& operator+=(DualT<T>& a, DualT<T> b) { a = a + b; return a; }

__device__ inline double val(double x) { return x; }
__device__ inline float val(float x) { return x; }
template <class T> __device__ inline T val(DualT<T> x) { return x.v; }
__device__ inline double tng(double) { return 0.0; }
__device__ inline float tng(float) { return 0.0f; }
template <class T> __device__ inline T tng(DualT<T> x) { return x.d; }

// elementary functions on T and on DualT<T> (CUDA's own float and double
// routines for the values; the derivatives from their closed forms)
__device__ inline double fexp(double x) { return exp(x); }
__device__ inline float fexp(float x) { return expf(x); }
__device__ inline double flog(double x) { return log(x); }
__device__ inline float flog(float x) { return logf(x); }
__device__ inline double fpow(double x, double n) { return pow(x, n); }
__device__ inline float fpow(float x, float n) { return powf(x, n); }
__device__ inline double fcbrt(double x) { return cbrt(x); }
__device__ inline float fcbrt(float x) { return cbrtf(x); }
__device__ inline double fcospi(double x) { return cospi(x); }
__device__ inline float fcospi(float x) { return cospif(x); }
__device__ inline double fsinpi(double x) { return sinpi(x); }
__device__ inline float fsinpi(float x) { return sinpif(x); }
template <class T> __device__ inline DualT<T> fexp(DualT<T> x) { T e = fexp(x.v); return {e, e * x.d}; }
template <class T> __device__ inline DualT<T> flog(DualT<T> x) { return {flog(x.v), x.d / x.v}; }
template <class T> __device__ inline DualT<T> fpow(DualT<T> x, T n) {   // x.v > 0
  T p = fpow(x.v, n);
  return {p, n * p / x.v * x.d};
}
template <class T> __device__ inline DualT<T> fcbrt(DualT<T> x) {
  T c = fcbrt(x.v);
  return {c, x.d / (T(3) * c * c)};
}
template <class T> __device__ inline DualT<T> fcospi(DualT<T> x) {
  return {fcospi(x.v), -T(M_PI) * fsinpi(x.v) * x.d};
}
template <class T> __device__ inline DualT<T> fsinpi(DualT<T> x) {
  return {fsinpi(x.v), T(M_PI) * fcospi(x.v) * x.d};
}

// A value with its derivative (kept for DualT, dropped for a plain T).
template <class S> struct Mk;
template <> struct Mk<double> { __device__ static double f(double v, double) { return v; } };
template <> struct Mk<float> { __device__ static float f(float v, float) { return v; } };
template <class T> struct Mk<DualT<T>> { __device__ static DualT<T> f(T v, T d) { return DualT<T>(v, d); } };

// The parameter struct in the working precision: ctbop_params' fields, in
// the same order, as R.
template <class R> struct ParamsT {
  R A[4], B[4], lambda1[4], lambda2[4], R_[4], S[4], kappa[4];
  R sigma[4], p[4], g[4][2], n[4][2];
  R gamma[8][2], c[8][2], d[8][2], h[8][2], alpha[8][2];
  R E0[2], chi[2], J[2], gamma_c[2], mass[2];
  R r_coul, k_e;
};
static_assert(sizeof(ParamsT<double>) == sizeof(ctbop_params), "ParamsT mirrors ctbop_params");
static_assert(sizeof(ParamsT<float>) * 2 == sizeof(ctbop_params), "ParamsT mirrors ctbop_params");

// Cutoff fc(r) and its derivatives with respect to R and S.
template <class R, class S>
__device__ inline void fc_params(S r, R Rin, R Sc, S& fc, S& dR, S& dS) {
  dR = dS = S(R(0));
  if (val(r) < Rin) { fc = S(R(1)); return; }
  if (val(r) >= Sc) { fc = S(R(0)); return; }
  R w = Sc - Rin;
  // 1/2 [1 + cos(pi t)] as cos^2(pi t / 2), free of the cancellation near
  // t = 1 (the cutoff function of the force kernels does the same)
  S h = R(0.5) * ((r - Rin) / w);
  S c = fcospi(h), sn = fsinpi(h);
  fc = c * c;
  S dfdt = R(-M_PI) * sn * c;
  dR = dfdt * (r - Sc) / (w * w);
  dS = dfdt * (Rin - r) / (w * w);
}

template <class R, class S>
__device__ inline S fc_only(S r, R Rin, R Sc) {
  if (val(r) < Rin) return S(R(1));
  if (val(r) >= Sc) return S(R(0));
  S c = fcospi(R(0.5) * ((r - Rin) / (Sc - Rin)));
  return c * c;
}

// Block accumulator in FP64: values weighted by wv, tangents by wt. With
// Agg, the lanes of a warp that reach one call together and name the same
// slot first sum their shares with shuffles and one of them adds the sum
// (the charge-kernel pass, whose lanes all name the same few slots at the
// end of their rows); without, every lane adds its own share.
template <bool Agg> struct Acc {
  double* g;    // [PG_NPARAM] values
  double* t;    // [PG_NPARAM] tangents
  double wv, wt;
  __device__ void put(int k, double a) const {
    if (!Agg) {
      atomicAdd(&g[k], a);
      return;
    }
    cg::coalesced_group grp = cg::labeled_partition(cg::coalesced_threads(), k);
    double sa = cg::reduce(grp, a, cg::plus<double>());
    if (grp.thread_rank() == 0) atomicAdd(&g[k], sa);
  }
  __device__ void put2(int k, double a, double b) const {
    if (!Agg) {
      atomicAdd(&g[k], a);
      atomicAdd(&t[k], b);
      return;
    }
    cg::coalesced_group grp = cg::labeled_partition(cg::coalesced_threads(), k);
    double sa = cg::reduce(grp, a, cg::plus<double>());
    double sb = cg::reduce(grp, b, cg::plus<double>());
    if (grp.thread_rank() == 0) {
      atomicAdd(&g[k], sa);
      atomicAdd(&t[k], sb);
    }
  }
  __device__ void operator()(int k, double x) const { put(k, wv * x); }
  __device__ void operator()(int k, float x) const { put(k, wv * (double)x); }
  template <class T> __device__ void operator()(int k, DualT<T> x) const {
    put2(k, wv * (double)x.v, wt * (double)x.d);
  }
};

// Partial sums of working-precision terms (values, or values with their
// tangents) over one bond's few third atoms of one type, kept in registers
// in the working precision: at most a handful of terms, so FP32 adds lose
// nothing that matters, and the FP64 pipe (a small fraction of the FP32
// rate on this GPU) sees only the block sums, once per bond and slot.
template <class S> struct SumT { using type = S; };
template <class S> __device__ inline S to_sum(S x) { return x; }

#define PG_GRP 8     // lanes per atom
#define PG_APB 16    // atoms per block

// One covalent list entry as staged in shared memory: the bond vector and
// length, and their derivatives along the direction (zero without one).
template <class R> struct __align__(16) Ent {
  R x, y, z, r;
  R tx, ty, tz, tr;
};

template <class R, class S> __device__ inline void ent_vec(const Ent<R>& a, S& x, S& y, S& z, S& r) {
  x = Mk<S>::f(a.x, a.tx); y = Mk<S>::f(a.y, a.ty); z = Mk<S>::f(a.z, a.tz); r = Mk<S>::f(a.r, a.tr);
}

// Bond vector from atom i to the image of j named by the list code, in the
// cell-local coordinates the positions are stored in.
template <class R>
__device__ inline void bond_vec(const typename Vec4<R>::T& ui, const typename Vec4<R>::T& uj, int code,
                                const RepInfo& ri, R& rx, R& ry, R& rz) {
  int dx, dy, dz;
  unpack_code(code, dx, dy, dz);
  R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
  if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
  rx = (uj.x - ui.x) + (R)dx * hx;
  ry = (uj.y - ui.y) + (R)dy * hy;
  rz = (uj.z - ui.z) + (R)dz * hz;
}

// Covalent terms: one 8-lane group per atom, the atom's covalent entries
// staged in shared memory; each lane takes bonds e. Block sums in shared
// memory (FP64), then one atomicAdd per parameter and block. R is the
// working precision, S either R (values only) or DualT<R>: then the entries
// carry their derivatives along dir and the charges theirs along qdir, the
// tangents of every term go to the second half of grad, and (with vout) each
// bond's share of d(Hq + chi)/de goes to vout: the charge-coupling term
// 1/2 fc kappa (q_i - q_j)^2 b_ij f_A contributes +-kappa fc f_A b_ij
// (q_i - q_j) to rows i and j.
template <class R, class S>
__global__ void __launch_bounds__(PG_APB * PG_GRP)
    k_pgrad_cov(int N, int cap_cov, int ld, const typename Vec4<R>::T* __restrict__ u,
                const int* __restrict__ rep, const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
                const int* __restrict__ ncov, const double* __restrict__ q, const double* __restrict__ qdir,
                const double* __restrict__ wval, const double* __restrict__ wtan, const double* __restrict__ dir,
                ParamsT<R> P, double* __restrict__ grad, double* __restrict__ vout) {
  using R4 = typename Vec4<R>::T;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ double s_g[2 * PG_NPARAM];
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  int g = threadIdx.x / PG_GRP, l = threadIdx.x % PG_GRP;
  Ent<R>* s_e = reinterpret_cast<Ent<R>*>(smem_raw) + (size_t)g * cap_cov;
  int* s_t = reinterpret_cast<int*>(reinterpret_cast<Ent<R>*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)g * cap_cov;
  int* s_j = reinterpret_cast<int*>(reinterpret_cast<Ent<R>*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)PG_APB * cap_cov + (size_t)g * cap_cov;
  int* s_lv = s_j + (size_t)PG_APB * cap_cov;   // the live bonds (r < S), in list order
  int i = blockIdx.x * PG_APB + g;
  bool live = i < N;
  int nc = 0, ti = 0;
  Acc<false> acc{s_g, s_g + PG_NPARAM, 0.0, 0.0};
  S qi = S(R(0));
  if (live) {
    R4 ui = u[i];
    ti = (int)ui.w;
    nc = min(ncov[i], cap_cov);
    const RepInfo& ri = reps[rep[i]];
    acc.wv = wval[rep[i]];
    acc.wt = wtan ? wtan[rep[i]] : 0.0;
    qi = Mk<S>::f((R)q[i], qdir ? (R)qdir[i] : R(0));
    R gix = 0, giy = 0, giz = 0;
    if (dir) { gix = (R)dir[3 * i]; giy = (R)dir[3 * i + 1]; giz = (R)dir[3 * i + 2]; }
    for (int e = l; e < nc; e += PG_GRP) {
      size_t idx = (size_t)e * ld + i;
      int j = nl[idx].x;
      R4 uj = u[j];
      Ent<R> w;
      bond_vec<R>(ui, uj, nl[idx].y, ri, w.x, w.y, w.z);
      w.r = sqrt(w.x * w.x + w.y * w.y + w.z * w.z);
      w.tx = w.ty = w.tz = w.tr = R(0);
      if (dir) {
        w.tx = (R)dir[3 * j] - gix; w.ty = (R)dir[3 * j + 1] - giy; w.tz = (R)dir[3 * j + 2] - giz;
        w.tr = (w.x * w.tx + w.y * w.ty + w.z * w.tz) / w.r;
      }
      s_e[e] = w;
      s_t[e] = (int)uj.w;
      s_j[e] = j;
    }
  }
  __syncthreads();
  // bonds past S have f_c = 0 and no parameter derivative: the loops below
  // run over the live ones only, in list order
  const int nlive = compact_live<PG_GRP>(
      live, nc, l, s_lv, [&](int e) { return s_e[e].r < P.S[ti * 2 + s_t[e]]; }, [](int) {});
  __syncwarp();
  if (live && (acc.wv != 0.0 || acc.wt != 0.0)) {
    for (int b_ = l; b_ < nlive; b_ += PG_GRP) {
      const int e = s_lv[b_];
      S ex, ey, ez, re;
      ent_vec(s_e[e], ex, ey, ez, re);
      int tj = s_t[e], pb = ti * 2 + tj;
      S fc, fcR, fcS;
      fc_params(re, P.R_[pb], P.S[pb], fc, fcR, fcS);
      if (val(fc) == R(0)) continue;
      // environment sums of bond e (recomputed)
      S z[2] = {S(R(0)), S(R(0))};
      for (int kk = 0; kk < nlive; ++kk) {
        const int k = s_lv[kk];
        if (k == e) continue;
        S kx, ky, kz, rk;
        ent_vec(s_e[k], kx, ky, kz, rk);
        int tk = s_t[k], pk = ti * 2 + tk;
        S fck = fc_only(rk, P.R_[pk], P.S[pk]);
        if (val(fck) == R(0)) continue;
        S ct = (ex * kx + ey * ky + ez * kz) / (re * rk);
        int tri = pb * 2 + tk;
        for (int ll = 0; ll < 2; ++ll) {
          R c2 = P.c[tri][ll] * P.c[tri][ll], d2 = P.d[tri][ll] * P.d[tri][ll];
          S hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
          S ang = P.gamma[tri][ll] * (R(1) + c2 * hm * hm / (d2 * den));
          z[ll] += fck * ang * fexp(P.alpha[tri][ll] * (re - rk));
        }
      }
      // bond order (Eq. 7) and its parameter derivatives, via ln b = e (ln S - ln S0)
      R pp = P.p[pb], sg = P.sigma[pb], ex_ = R(1) / (R(2) * sg * pp);
      S zn[2], Z[2], t[2], lnz[2];
      for (int ll = 0; ll < 2; ++ll) {
        bool pos = val(z[ll]) > R(0);
        zn[ll] = pos ? fpow(z[ll], P.n[pb][ll]) : S(R(0));
        lnz[ll] = pos ? flog(z[ll]) : S(R(0));
        Z[ll] = P.g[pb][ll] + zn[ll];
        t[ll] = fpow(Z[ll], -pp);
      }
      S Ssum = t[0] + t[1];
      R s0a = fpow(P.g[pb][0], -pp), s0b = fpow(P.g[pb][1], -pp), S0 = s0a + s0b;
      S lnb = ex_ * (flog(Ssum) - flog(S0));
      S b = fexp(lnb);
      S dq = qi - Mk<S>::f((R)q[s_j[e]], qdir ? (R)qdir[s_j[e]] : R(0));
      S dq2 = dq * dq;
      S cq = R(1) - P.kappa[pb] * dq2;
      S e1 = fexp(-P.lambda1[pb] * re), e2 = fexp(-P.lambda2[pb] * re);
      S fR = P.A[pb] * e1, fA = P.B[pb] * e2;
      S V = fR - cq * b * fA;
      S Eb = R(-0.5) * cq * fc * fA;   // dE/db
      if (vout) {
        double wq = (double)tng(P.kappa[pb] * (fc * fA * b)) * (double)val(dq);
        if (wq != 0.0) {
          atomicAdd(vout + i, wq);
          atomicAdd(vout + s_j[e], -wq);
        }
      }
      // pair parameters
      acc(PG_A + pb, R(0.5) * fc * e1);
      acc(PG_B + pb, R(-0.5) * cq * fc * b * e2);
      acc(PG_L1 + pb, R(-0.5) * fc * re * fR);
      acc(PG_L2 + pb, R(0.5) * cq * fc * b * fA * re);
      acc(PG_KAPPA + pb, R(0.5) * dq2 * fc * b * fA);
      acc(PG_R + pb, R(0.5) * fcR * V);
      acc(PG_S + pb, R(0.5) * fcS * V);
      // bond-order parameters
      S dlnS_dp = -(t[0] * flog(Z[0]) + t[1] * flog(Z[1])) / Ssum;
      R dlnS0_dp = -(s0a * flog(P.g[pb][0]) + s0b * flog(P.g[pb][1])) / S0;
      S wb = Eb * b;
      acc(PG_SIGMA + pb, wb * (-lnb / sg));
      acc(PG_P + pb, wb * (-lnb / pp + ex_ * (dlnS_dp - dlnS0_dp)));
      for (int ll = 0; ll < 2; ++ll) {
        S dg = ex_ * (-pp * t[ll] / (Z[ll] * Ssum) + pp * fpow(P.g[pb][ll], -pp - R(1)) / S0);
        acc(PG_G + pb * 2 + ll, wb * dg);
        S dn = val(z[ll]) > R(0) ? ex_ * (-pp * t[ll] / (Z[ll] * Ssum)) * zn[ll] * lnz[ll] : S(R(0));
        acc(PG_N + pb * 2 + ll, wb * dn);
      }
      // dE/dzeta_l = Eb db/dzeta_l = Eb b (d ln b / d zeta_l)
      S Ez[2];
      for (int ll = 0; ll < 2; ++ll)
        Ez[ll] = val(z[ll]) > R(0)
                     ? Eb * b * ex_ * (-pp * t[ll] / (Z[ll] * Ssum)) * P.n[pb][ll] * zn[ll] / z[ll]
                     : S(R(0));
      // triplet parameters and the cutoff of the (i, k) pairs inside zeta:
      // the terms of the k of one type share their slots, so they are summed
      // in registers (FP64) and added once per bond and type of k
      using ST = typename SumT<S>::type;
      for (int tk = 0; tk < 2; ++tk) {
        const int tri = pb * 2 + tk, pk = ti * 2 + tk;
        ST sg_[2], sc_[2], sd_[2], sh_[2], sa_[2], sR(0.0), sS(0.0);
        for (int ll = 0; ll < 2; ++ll) sg_[ll] = sc_[ll] = sd_[ll] = sh_[ll] = sa_[ll] = ST(0.0);
        bool any = false;
        for (int kk = 0; kk < nlive; ++kk) {
          const int k = s_lv[kk];
          if (k == e || s_t[k] != tk) continue;
          S kx, ky, kz, rk;
          ent_vec(s_e[k], kx, ky, kz, rk);
          S fck, fkR, fkS;
          fc_params(rk, P.R_[pk], P.S[pk], fck, fkR, fkS);
          if (val(fck) == R(0)) continue;
          S ct = (ex * kx + ey * ky + ez * kz) / (re * rk);
          for (int ll = 0; ll < 2; ++ll) {
            if (val(Ez[ll]) == R(0)) continue;
            R cc = P.c[tri][ll], dd = P.d[tri][ll], gm = P.gamma[tri][ll];
            R c2 = cc * cc, d2 = dd * dd;
            S hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
            S angg = R(1) + c2 * hm * hm / (d2 * den);   // ang / gamma
            S dr = re - rk;
            S exl = fexp(P.alpha[tri][ll] * dr);
            S wz = Ez[ll] * exl;
            sg_[ll] += to_sum(wz * fck * angg);
            sc_[ll] += to_sum(wz * fck * (gm * R(2) * cc) * hm * hm / (d2 * den));
            sd_[ll] += to_sum(wz * fck * (R(2) * gm * c2 * dd) * (R(1) / (den * den) - R(1) / (d2 * d2)));
            sh_[ll] += to_sum(wz * fck * (gm * R(2) * c2) * hm / (den * den));
            sa_[ll] += to_sum(wz * fck * gm * angg * dr);
            sR += to_sum(wz * fkR * gm * angg);
            sS += to_sum(wz * fkS * gm * angg);
            any = true;
          }
        }
        if (!any) continue;
        for (int ll = 0; ll < 2; ++ll) {
          acc(PG_GAMMA + tri * 2 + ll, sg_[ll]);
          acc(PG_C + tri * 2 + ll, sc_[ll]);
          acc(PG_D + tri * 2 + ll, sd_[ll]);
          acc(PG_H + tri * 2 + ll, sh_[ll]);
          acc(PG_ALPHA + tri * 2 + ll, sa_[ll]);
        }
        acc(PG_R + pk, sR);
        acc(PG_S + pk, sS);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// Charge-kernel and self-energy parameters: one thread per atom over all of
// its entries (each unordered pair appears in both atoms' lists, hence the
// 1/2 of the energy). Block sums in shared memory (FP64). With S = DualT<R>
// the distances carry their derivatives along dir and the charges theirs
// along qdir, and (with vout) vout_i gets the Coulomb share of
// d(Hq + chi)_i/de, sum_j q_j dK(r_ij)/de.
template <class R, class S>
__global__ void __launch_bounds__(256)
    k_pgrad_coul(int N, int ld, const typename Vec4<R>::T* __restrict__ u, const int* __restrict__ rep,
                 const RepInfo* __restrict__ reps, const int2* __restrict__ nl, const int* __restrict__ nall,
                 const double* __restrict__ q, const double* __restrict__ qdir, const double* __restrict__ wval,
                 const double* __restrict__ wtan, const double* __restrict__ dir, ParamsT<R> P,
                 double* __restrict__ grad, double* __restrict__ vout) {
  using R4 = typename Vec4<R>::T;
  __shared__ double s_g[2 * PG_NPARAM];
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    Acc<true> acc{s_g, s_g + PG_NPARAM, wval[rep[i]], wtan ? wtan[rep[i]] : 0.0};
    if (acc.wv != 0.0 || acc.wt != 0.0) {
      R4 ui = u[i];
      int ti = (int)ui.w;
      S qi = Mk<S>::f((R)q[i], qdir ? (R)qdir[i] : R(0));
      acc(PG_E0 + ti, R(1));
      acc(PG_CHI + ti, qi);
      acc(PG_J + ti, qi * qi);
      const RepInfo& ri = reps[rep[i]];
      R rc = P.r_coul, ke = P.k_e;
      R gix = 0, giy = 0, giz = 0;
      if (dir) { gix = (R)dir[3 * i]; giy = (R)dir[3 * i + 1]; giz = (R)dir[3 * i + 2]; }
      S gke(R(0)), grc(R(0)), gga0(R(0)), gga1(R(0));
      double vi = 0.0;
      int na = nall[i];
      for (int e = 0; e < na; ++e) {
        size_t idx = (size_t)e * ld + i;
        int j = nl[idx].x;
        R4 uj = u[j];
        R rx, ry, rz;
        bond_vec<R>(ui, uj, nl[idx].y, ri, rx, ry, rz);
        R rv = sqrt(rx * rx + ry * ry + rz * rz);
        R tr = R(0);
        if (dir) tr = (rx * ((R)dir[3 * j] - gix) + ry * ((R)dir[3 * j + 1] - giy) +
                       rz * ((R)dir[3 * j + 2] - giz)) / rv;
        S r = Mk<S>::f(rv, tr);
        S x = r / rc;
        if (val(x) >= R(1)) continue;
        int tj = (int)uj.w;
        R ga = P.gamma_c[ti], gb = P.gamma_c[tj];
        R gs3 = fpow(ga * gb, R(-1.5));
        S x2 = x * x, x3 = x2 * x, x4 = x2 * x2, xm = x - R(1);
        S T = R(1) + x4 * (R(-35) + x * (R(84) + x * (R(-70) + R(20) * x)));
        S dT = R(140) * x3 * xm * xm * xm;
        S D = fcbrt(r * r * r + gs3), iD = R(1) / D;
        S K = ke * T * iD;
        S qj = Mk<S>::f((R)q[j], qdir ? (R)qdir[j] : R(0));
        vi += (double)tng(K) * (double)val(qj);
        S w = R(0.5) * qi * qj;
        gke += w * K / ke;
        grc += (ke / (rc * rc)) * w * dT * (-r) * iD;
        S dK_dgs3 = (-ke / R(3)) * T * iD * iD * iD * iD;
        S c0 = w * dK_dgs3 * (R(-1.5) * gs3);
        if (ti == 0) gga0 += c0 / ga; else gga1 += c0 / ga;
        if (tj == 0) gga0 += c0 / gb; else gga1 += c0 / gb;
      }
      acc(PG_KE, gke);
      acc(PG_RCOUL, grc);
      acc(PG_GAMMA_C, gga0);
      acc(PG_GAMMA_C + 1, gga1);
      if (vout && vi != 0.0) atomicAdd(vout + i, vi);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// ---------------------------------------------------------------- launchers
template <class R, class S>
static cudaError_t pgrad_launch(const DevState& D, const ParamsT<R>& P, const double* wval, const double* wtan,
                                const double* dir, const double* qdir, double* grad, double* vout,
                                cudaStream_t st) {
  using R4 = typename Vec4<R>::T;
  size_t sm = (size_t)PG_APB * D.cap_cov * (sizeof(Ent<R>) + 3 * sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(k_pgrad_cov<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_pgrad_cov<R, S><<<(D.N + PG_APB - 1) / PG_APB, PG_APB * PG_GRP, sm, st>>>(
      D.N, D.cap_cov, D.ld, (const R4*)D.u, D.rep, D.reps, D.nl, D.ncov, D.q, qdir, wval, wtan, dir, P, grad,
      vout);
  k_pgrad_coul<R, S><<<(D.N + 255) / 256, 256, 0, st>>>(D.N, D.ld, (const R4*)D.u, D.rep, D.reps, D.nl, D.nall,
                                                       D.q, qdir, wval, wtan, dir, P, grad, vout);
  return cudaGetLastError();
}

template <class R>
static cudaError_t pgrad_prec(const DevState& D, const ctbop_params& P, const double* wval, const double* wtan,
                              const double* dir, const double* qdir, double* grad, double* vout,
                              cudaStream_t st) {
  ParamsT<R> Pr;
  const double* src = reinterpret_cast<const double*>(&P);
  R* dst = reinterpret_cast<R*>(&Pr);
  for (int k = 0; k < PG_NPARAM; ++k) dst[k] = (R)src[k];
  if (dir || qdir) return pgrad_launch<R, DualT<R>>(D, Pr, wval, wtan, dir, qdir, grad, vout, st);
  return pgrad_launch<R, R>(D, Pr, wval, nullptr, nullptr, nullptr, grad, nullptr, st);
}

cudaError_t launch_param_grad(const DevState& D, const ctbop_params& P, bool fp32, const double* wval,
                              const double* wtan, const double* dir, const double* qdir, double* grad,
                              double* vout, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(double) * 2 * PG_NPARAM, st);
  if (e == cudaSuccess && vout) e = cudaMemsetAsync(vout, 0, sizeof(double) * std::max(D.N, 1), st);
  if (e != cudaSuccess || D.N == 0) return e;
  if (fp32) return pgrad_prec<float>(D, P, wval, wtan, dir, qdir, grad, vout, st);
  return pgrad_prec<double>(D, P, wval, wtan, dir, qdir, grad, vout, st);
}

}  // namespace ct
