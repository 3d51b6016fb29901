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

#include "internal.cuh"
#include "kernels.h"
#include "ctbop.h"

namespace ct {

// ------------------------------------------------------------ dual numbers
struct Dual {
  double v, d;
  Dual() = default;
  __device__ Dual(double x) : v(x), d(0.0) {}
  __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__device__ inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ inline Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ inline Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ inline Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ inline Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ inline Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ inline Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ inline Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__device__ inline Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return {q, -q * b.d / b.v};
}
__device__ inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }

__device__ inline double val(double x) { return x; }
__device__ inline double val(Dual x) { return x.v; }
__device__ inline double tng(double) { return 0.0; }
__device__ inline double tng(Dual x) { return x.d; }

__device__ inline double exp_(double x) { return exp(x); }
__device__ inline Dual exp_(Dual x) { double e = exp(x.v); return {e, e * x.d}; }
__device__ inline double log_(double x) { return log(x); }
__device__ inline Dual log_(Dual x) { return {log(x.v), x.d / x.v}; }
__device__ inline double pow_(double x, double n) { return pow(x, n); }
__device__ inline Dual pow_(Dual x, double n) {   // x.v > 0
  double p = pow(x.v, n);
  return {p, n * p / x.v * x.d};
}
__device__ inline double sqrt_(double x) { return sqrt(x); }
__device__ inline Dual sqrt_(Dual x) { double s = sqrt(x.v); return {s, 0.5 * x.d / s}; }
__device__ inline double cbrt_(double x) { return cbrt(x); }
__device__ inline Dual cbrt_(Dual x) { double c = cbrt(x.v); return {c, x.d / (3.0 * c * c)}; }
__device__ inline double cospi_(double x) { return cospi(x); }
__device__ inline Dual cospi_(Dual x) { return {cospi(x.v), -M_PI * sinpi(x.v) * x.d}; }
__device__ inline double sinpi_(double x) { return sinpi(x); }
__device__ inline Dual sinpi_(Dual x) { return {sinpi(x.v), M_PI * cospi(x.v) * x.d}; }

// Cutoff fc(r) and its derivatives with respect to R and S.
template <class S>
__device__ inline void fc_params(S r, double Rin, double Sc, S& fc, S& dR, S& dS) {
  dR = dS = S(0.0);
  if (val(r) < Rin) { fc = S(1.0); return; }
  if (val(r) >= Sc) { fc = S(0.0); return; }
  double w = Sc - Rin;
  S t = (r - Rin) / w;
  fc = 0.5 * (1.0 + cospi_(t));
  S dfdt = -0.5 * M_PI * sinpi_(t);
  dR = dfdt * (r - Sc) / (w * w);
  dS = dfdt * (Rin - r) / (w * w);
}

template <class S>
__device__ inline S fc_only(S r, double Rin, double Sc) {
  if (val(r) < Rin) return S(1.0);
  if (val(r) >= Sc) return S(0.0);
  return 0.5 * (1.0 + cospi_((r - Rin) / (Sc - Rin)));
}

// Block accumulator: values weighted by wv, tangents by wt.
struct Acc {
  double* g;    // [PG_NPARAM] values
  double* t;    // [PG_NPARAM] tangents
  double wv, wt;
  __device__ void operator()(int k, double x) const { atomicAdd(&g[k], wv * x); }
  __device__ void operator()(int k, Dual x) const {
    atomicAdd(&g[k], wv * x.v);
    atomicAdd(&t[k], wt * x.d);
  }
};

#define PG_GRP 8     // lanes per atom
#define PG_APB 16    // atoms per block

// One covalent list entry as staged in shared memory: the bond vector and
// length, and their derivatives along the direction (zero without one).
struct __align__(16) Ent {
  double x, y, z, r;
  double tx, ty, tz, tr;
};

// A value with its derivative (kept for Dual, dropped for double).
template <class S> __device__ inline S mk(double v, double d);
template <> __device__ inline double mk<double>(double v, double) { return v; }
template <> __device__ inline Dual mk<Dual>(double v, double d) { return Dual(v, d); }

template <class S> __device__ inline void ent_vec(const Ent& a, S& x, S& y, S& z, S& r) {
  x = mk<S>(a.x, a.tx); y = mk<S>(a.y, a.ty); z = mk<S>(a.z, a.tz); r = mk<S>(a.r, a.tr);
}

// Covalent terms: one 8-lane group per atom, the atom's covalent entries
// staged in shared memory; each lane takes bonds e. Block sums in shared
// memory, then one atomicAdd per parameter and block. With S = Dual the
// entries carry their derivatives along dir, the tangents of every term go
// to the second half of grad, and each bond's share of d(Hq + chi)/de goes
// to vout: the charge-coupling term 1/2 fc kappa (q_i - q_j)^2 b_ij f_A
// contributes +-kappa fc f_A b_ij (q_i - q_j) to rows i and j.
template <class S>
__global__ void __launch_bounds__(PG_APB * PG_GRP)
    k_pgrad_cov(int N, int cap_cov, int ld, const double4_32a* __restrict__ u, const int* __restrict__ rep,
                const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
                const int* __restrict__ ncov, const double* __restrict__ q, const double* __restrict__ wval,
                const double* __restrict__ wtan, const double* __restrict__ dir, ctbop_params P,
                double* __restrict__ grad, double* __restrict__ vout) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ double s_g[2 * PG_NPARAM];
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  int g = threadIdx.x / PG_GRP, l = threadIdx.x % PG_GRP;
  Ent* s_e = reinterpret_cast<Ent*>(smem_raw) + (size_t)g * cap_cov;
  int* s_t = reinterpret_cast<int*>(reinterpret_cast<Ent*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)g * cap_cov;
  int* s_j = reinterpret_cast<int*>(reinterpret_cast<Ent*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)PG_APB * cap_cov + (size_t)g * cap_cov;
  int i = blockIdx.x * PG_APB + g;
  bool live = i < N;
  int nc = 0, ti = 0;
  Acc acc{s_g, s_g + PG_NPARAM, 0.0, 0.0};
  double qi = 0.0;
  if (live) {
    double4_32a ui = u[i];
    ti = (int)ui.w;
    nc = min(ncov[i], cap_cov);
    const RepInfo& ri = reps[rep[i]];
    acc.wv = wval[rep[i]];
    acc.wt = wtan ? wtan[rep[i]] : 0.0;
    qi = q[i];
    double gix = 0.0, giy = 0.0, giz = 0.0;
    if (dir) { gix = dir[3 * i]; giy = dir[3 * i + 1]; giz = dir[3 * i + 2]; }
    for (int e = l; e < nc; e += PG_GRP) {
      size_t idx = (size_t)e * ld + i;
      int j = nl[idx].x;
      double4_32a uj = u[j];
      int dx, dy, dz;
      unpack_code(nl[idx].y, dx, dy, dz);
      Ent w;
      w.x = (uj.x - ui.x) + dx * ri.hc[0];
      w.y = (uj.y - ui.y) + dy * ri.hc[1];
      w.z = (uj.z - ui.z) + dz * ri.hc[2];
      w.r = sqrt(w.x * w.x + w.y * w.y + w.z * w.z);
      w.tx = w.ty = w.tz = w.tr = 0.0;
      if (dir) {
        w.tx = dir[3 * j] - gix; w.ty = dir[3 * j + 1] - giy; w.tz = dir[3 * j + 2] - giz;
        w.tr = (w.x * w.tx + w.y * w.ty + w.z * w.tz) / w.r;
      }
      s_e[e] = w;
      s_t[e] = (int)uj.w;
      s_j[e] = j;
    }
  }
  __syncthreads();
  if (live && (acc.wv != 0.0 || acc.wt != 0.0)) {
    for (int e = l; e < nc; e += PG_GRP) {
      S ex, ey, ez, re;
      ent_vec<S>(s_e[e], ex, ey, ez, re);
      int tj = s_t[e], pb = ti * 2 + tj;
      S fc, fcR, fcS;
      fc_params(re, P.R[pb], P.S[pb], fc, fcR, fcS);
      if (val(fc) == 0.0) continue;
      // environment sums of bond e (recomputed)
      S z[2] = {S(0.0), S(0.0)};
      for (int k = 0; k < nc; ++k) {
        if (k == e) continue;
        S kx, ky, kz, rk;
        ent_vec<S>(s_e[k], kx, ky, kz, rk);
        int tk = s_t[k], pk = ti * 2 + tk;
        S fck = fc_only(rk, P.R[pk], P.S[pk]);
        if (val(fck) == 0.0) continue;
        S ct = (ex * kx + ey * ky + ez * kz) / (re * rk);
        int tri = pb * 2 + tk;
        for (int ll = 0; ll < 2; ++ll) {
          double c2 = P.c[tri][ll] * P.c[tri][ll], d2 = P.d[tri][ll] * P.d[tri][ll];
          S hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
          S ang = P.gamma[tri][ll] * (1.0 + c2 * hm * hm / (d2 * den));
          z[ll] += fck * ang * exp_(P.alpha[tri][ll] * (re - rk));
        }
      }
      // bond order (Eq. 7) and its parameter derivatives, via ln b = e (ln S - ln S0)
      double pp = P.p[pb], sg = P.sigma[pb], ex_ = 1.0 / (2.0 * sg * pp);
      S zn[2], Z[2], t[2], lnz[2];
      for (int ll = 0; ll < 2; ++ll) {
        bool pos = val(z[ll]) > 0.0;
        zn[ll] = pos ? pow_(z[ll], P.n[pb][ll]) : S(0.0);
        lnz[ll] = pos ? log_(z[ll]) : S(0.0);
        Z[ll] = P.g[pb][ll] + zn[ll];
        t[ll] = pow_(Z[ll], -pp);
      }
      S Ssum = t[0] + t[1];
      double s0a = pow(P.g[pb][0], -pp), s0b = pow(P.g[pb][1], -pp), S0 = s0a + s0b;
      S lnb = ex_ * (log_(Ssum) - log(S0));
      S b = exp_(lnb);
      double dq = qi - q[s_j[e]];
      double cq = 1.0 - P.kappa[pb] * dq * dq;
      S e1 = exp_(-P.lambda1[pb] * re), e2 = exp_(-P.lambda2[pb] * re);
      S fR = P.A[pb] * e1, fA = P.B[pb] * e2;
      S V = fR - cq * b * fA;
      S Eb = -0.5 * cq * fc * fA;   // dE/db
      if (vout) {
        double wq = tng(P.kappa[pb] * (fc * fA * b)) * dq;
        if (wq != 0.0) {
          atomicAdd(vout + i, wq);
          atomicAdd(vout + s_j[e], -wq);
        }
      }
      // pair parameters
      acc(PG_A + pb, 0.5 * fc * e1);
      acc(PG_B + pb, (-0.5 * cq) * fc * b * e2);
      acc(PG_L1 + pb, -0.5 * fc * re * fR);
      acc(PG_L2 + pb, (0.5 * cq) * fc * b * fA * re);
      acc(PG_KAPPA + pb, (0.5 * dq * dq) * fc * b * fA);
      acc(PG_R + pb, 0.5 * fcR * V);
      acc(PG_S + pb, 0.5 * fcS * V);
      // bond-order parameters
      S dlnS_dp = -(t[0] * log_(Z[0]) + t[1] * log_(Z[1])) / Ssum;
      double dlnS0_dp = -(s0a * log(P.g[pb][0]) + s0b * log(P.g[pb][1])) / S0;
      S wb = Eb * b;
      acc(PG_SIGMA + pb, wb * (-lnb / sg));
      acc(PG_P + pb, wb * (-lnb / pp + ex_ * (dlnS_dp - dlnS0_dp)));
      for (int ll = 0; ll < 2; ++ll) {
        S dg = ex_ * (-pp * t[ll] / (Z[ll] * Ssum) + pp * pow(P.g[pb][ll], -pp - 1.0) / S0);
        acc(PG_G + pb * 2 + ll, wb * dg);
        S dn = val(z[ll]) > 0.0 ? ex_ * (-pp * t[ll] / (Z[ll] * Ssum)) * zn[ll] * lnz[ll] : S(0.0);
        acc(PG_N + pb * 2 + ll, wb * dn);
      }
      // dE/dzeta_l = Eb db/dzeta_l = Eb b (d ln b / d zeta_l)
      S Ez[2];
      for (int ll = 0; ll < 2; ++ll)
        Ez[ll] = val(z[ll]) > 0.0
                     ? Eb * b * ex_ * (-pp * t[ll] / (Z[ll] * Ssum)) * P.n[pb][ll] * zn[ll] / z[ll]
                     : S(0.0);
      // triplet parameters and the cutoff of the (i, k) pairs inside zeta
      for (int k = 0; k < nc; ++k) {
        if (k == e) continue;
        S kx, ky, kz, rk;
        ent_vec<S>(s_e[k], kx, ky, kz, rk);
        int tk = s_t[k], pk = ti * 2 + tk;
        S fck, fkR, fkS;
        fc_params(rk, P.R[pk], P.S[pk], fck, fkR, fkS);
        if (val(fck) == 0.0) continue;
        S ct = (ex * kx + ey * ky + ez * kz) / (re * rk);
        int tri = pb * 2 + tk;
        for (int ll = 0; ll < 2; ++ll) {
          if (val(Ez[ll]) == 0.0) continue;
          double cc = P.c[tri][ll], dd = P.d[tri][ll], gm = P.gamma[tri][ll];
          double c2 = cc * cc, d2 = dd * dd;
          S hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
          S angg = 1.0 + c2 * hm * hm / (d2 * den);   // ang / gamma
          S dr = re - rk;
          S exl = exp_(P.alpha[tri][ll] * dr);
          S wz = Ez[ll] * exl;
          acc(PG_GAMMA + tri * 2 + ll, wz * fck * angg);
          acc(PG_C + tri * 2 + ll, wz * fck * (gm * 2.0 * cc) * hm * hm / (d2 * den));
          acc(PG_D + tri * 2 + ll, wz * fck * (2.0 * gm * c2 * dd) * (1.0 / (den * den) - 1.0 / (d2 * d2)));
          acc(PG_H + tri * 2 + ll, wz * fck * (gm * 2.0 * c2) * hm / (den * den));
          acc(PG_ALPHA + tri * 2 + ll, wz * fck * gm * angg * dr);
          acc(PG_R + pk, wz * fkR * gm * angg);
          acc(PG_S + pk, wz * fkS * gm * angg);
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// Charge-kernel and self-energy parameters: one thread per atom over all of
// its entries (each unordered pair appears in both atoms' lists, hence the
// 1/2 of the energy). Block sums in shared memory. With S = Dual the pair
// distances carry their derivatives along dir, and vout_i gets the Coulomb
// share of d(Hq + chi)_i/de, sum_j q_j dK(r_ij)/de.
template <class S>
__global__ void __launch_bounds__(256)
    k_pgrad_coul(int N, int ld, const double4_32a* __restrict__ u, const int* __restrict__ rep,
                 const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
                 const int* __restrict__ nall, const double* __restrict__ q, const double* __restrict__ wval,
                 const double* __restrict__ wtan, const double* __restrict__ dir, ctbop_params P,
                 double* __restrict__ grad, double* __restrict__ vout) {
  __shared__ double s_g[2 * PG_NPARAM];
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    Acc acc{s_g, s_g + PG_NPARAM, wval[rep[i]], wtan ? wtan[rep[i]] : 0.0};
    if (acc.wv != 0.0 || acc.wt != 0.0) {
      double4_32a ui = u[i];
      int ti = (int)ui.w;
      double qi = q[i];
      acc(PG_E0 + ti, 1.0);
      acc(PG_CHI + ti, qi);
      acc(PG_J + ti, qi * qi);
      const RepInfo& ri = reps[rep[i]];
      double rc = P.r_coul, ke = P.k_e;
      double gix = 0.0, giy = 0.0, giz = 0.0;
      if (dir) { gix = dir[3 * i]; giy = dir[3 * i + 1]; giz = dir[3 * i + 2]; }
      S gke(0.0), grc(0.0), gga[2] = {S(0.0), S(0.0)};
      double vi = 0.0;
      int na = nall[i];
      for (int e = 0; e < na; ++e) {
        size_t idx = (size_t)e * ld + i;
        int j = nl[idx].x;
        double4_32a uj = u[j];
        int dx, dy, dz;
        unpack_code(nl[idx].y, dx, dy, dz);
        double rx = (uj.x - ui.x) + dx * ri.hc[0], ry = (uj.y - ui.y) + dy * ri.hc[1],
               rz = (uj.z - ui.z) + dz * ri.hc[2];
        double rv = sqrt(rx * rx + ry * ry + rz * rz);
        double t = 0.0;
        if (dir) t = (rx * (dir[3 * j] - gix) + ry * (dir[3 * j + 1] - giy) + rz * (dir[3 * j + 2] - giz)) / rv;
        S r = mk<S>(rv, t);
        S x = r / rc;
        if (val(x) >= 1.0) continue;
        int tj = (int)uj.w;
        double ga = P.gamma_c[ti], gb = P.gamma_c[tj];
        double gs3 = pow(ga * gb, -1.5);
        S x2 = x * x, x3 = x2 * x, x4 = x2 * x2, xm = x - 1.0;
        S T = 1.0 + x4 * (-35.0 + x * (84.0 + x * (-70.0 + 20.0 * x)));
        S dT = 140.0 * x3 * xm * xm * xm;
        S D = cbrt_(r * r * r + gs3), iD = 1.0 / D;
        S K = ke * T * iD;
        double qj = q[j];
        vi += tng(K) * qj;
        double w = 0.5 * qi * qj;
        gke += w * K / ke;
        grc += (w * ke / (rc * rc)) * dT * (-r) * iD;
        S dK_dgs3 = (-ke / 3.0) * T * iD * iD * iD * iD;
        gga[ti] += (w * (-1.5 * gs3 / ga)) * dK_dgs3;
        gga[tj] += (w * (-1.5 * gs3 / gb)) * dK_dgs3;
      }
      acc(PG_KE, gke);
      acc(PG_RCOUL, grc);
      acc(PG_GAMMA_C, gga[0]);
      acc(PG_GAMMA_C + 1, gga[1]);
      if (vout && vi != 0.0) atomicAdd(vout + i, vi);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// ---------------------------------------------------------------- launchers
template <class S>
static cudaError_t pgrad_launch(const DevState& S_, const ctbop_params& P, const double* wval, const double* wtan,
                                const double* dir, double* grad, double* vout, cudaStream_t st) {
  size_t sm = (size_t)PG_APB * S_.cap_cov * (sizeof(Ent) + 2 * sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(k_pgrad_cov<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_pgrad_cov<S><<<(S_.N + PG_APB - 1) / PG_APB, PG_APB * PG_GRP, sm, st>>>(
      S_.N, S_.cap_cov, S_.ld, (const double4_32a*)S_.u, S_.rep, S_.reps, S_.nl, S_.ncov, S_.q, wval, wtan, dir,
      P, grad, vout);
  k_pgrad_coul<S><<<(S_.N + 255) / 256, 256, 0, st>>>(S_.N, S_.ld, (const double4_32a*)S_.u, S_.rep, S_.reps,
                                                      S_.nl, S_.nall, S_.q, wval, wtan, dir, P, grad, vout);
  return cudaGetLastError();
}

cudaError_t launch_param_grad(const DevState& S, const ctbop_params& P, const double* wval, const double* wtan,
                              const double* dir, double* grad, double* vout, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(double) * 2 * PG_NPARAM, st);
  if (e == cudaSuccess && vout) e = cudaMemsetAsync(vout, 0, sizeof(double) * std::max(S.N, 1), st);
  if (e != cudaSuccess || S.N == 0) return e;
  if (dir) return pgrad_launch<Dual>(S, P, wval, wtan, dir, grad, vout, st);
  return pgrad_launch<double>(S, P, wval, nullptr, nullptr, grad, nullptr, st);
}

}  // namespace ct
