// grad.cu — derivatives of the energy with respect to the potential's
// parameters (the force-matching gradient of the spec differentiation
// pattern), FP64.
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
#include "internal.cuh"
#include "kernels.h"
#include "ctbop.h"

namespace ct {

// Cutoff fc(r) and its derivatives with respect to R and S.
__device__ inline void fc_params(double r, double Rin, double S, double& fc, double& dR, double& dS) {
  dR = dS = 0.0;
  if (r < Rin) { fc = 1.0; return; }
  if (r >= S) { fc = 0.0; return; }
  double w = S - Rin, t = (r - Rin) / w;
  fc = 0.5 * (1.0 + cospi(t));
  double dfdt = -0.5 * M_PI * sinpi(t);
  dR = dfdt * (r - S) / (w * w);
  dS = dfdt * (-(r - Rin)) / (w * w);
}

__device__ inline double fc_only(double r, double Rin, double S) {
  if (r < Rin) return 1.0;
  if (r >= S) return 0.0;
  return 0.5 * (1.0 + cospi((r - Rin) / (S - Rin)));
}

#define PG_GRP 8     // lanes per atom
#define PG_APB 16    // atoms per block

// Covalent terms: one 8-lane group per atom, the atom's covalent entries
// staged in shared memory; each lane takes bonds e. Block sums in shared
// memory, then one atomicAdd per parameter and block.
__global__ void __launch_bounds__(PG_APB * PG_GRP)
    k_pgrad_cov(int N, int cap_cov, int ld, const double4_32a* __restrict__ u, const int* __restrict__ rep,
                const RepInfo* __restrict__ reps, const int2* __restrict__ nl, 
                const int* __restrict__ ncov, const double* __restrict__ q, const double* __restrict__ wrep,
                ctbop_params P, double* __restrict__ grad) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ double s_g[PG_NPARAM];
  for (int k = threadIdx.x; k < PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  int g = threadIdx.x / PG_GRP, l = threadIdx.x % PG_GRP;
  double4_32a* s_u = reinterpret_cast<double4_32a*>(smem_raw) + (size_t)g * cap_cov;   // (rx, ry, rz, r)
  int* s_t = reinterpret_cast<int*>(reinterpret_cast<double4_32a*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)g * cap_cov;
  int* s_j = reinterpret_cast<int*>(reinterpret_cast<double4_32a*>(smem_raw) + (size_t)PG_APB * cap_cov) +
             (size_t)PG_APB * cap_cov + (size_t)g * cap_cov;
  int i = blockIdx.x * PG_APB + g;
  bool live = i < N;
  int nc = 0, ti = 0;
  double wi = 0.0, qi = 0.0;
  if (live) {
    double4_32a ui = u[i];
    ti = (int)ui.w;
    nc = min(ncov[i], cap_cov);
    const RepInfo& ri = reps[rep[i]];
    wi = wrep[rep[i]];
    qi = q[i];
    for (int e = l; e < nc; e += PG_GRP) {
      size_t idx = (size_t)e * ld + i;
      int j = nl[idx].x;
      double4_32a uj = u[j];
      int dx, dy, dz;
      unpack_code(nl[idx].y, dx, dy, dz);
      double rx = (uj.x - ui.x) + dx * ri.hc[0], ry = (uj.y - ui.y) + dy * ri.hc[1],
             rz = (uj.z - ui.z) + dz * ri.hc[2];
      double4_32a w;
      w.x = rx; w.y = ry; w.z = rz; w.w = sqrt(rx * rx + ry * ry + rz * rz);
      s_u[e] = w;
      s_t[e] = (int)uj.w;
      s_j[e] = j;
    }
  }
  __syncthreads();
  if (live && wi != 0.0) {
    for (int e = l; e < nc; e += PG_GRP) {
      double4_32a ue = s_u[e];
      double re = ue.w;
      int tj = s_t[e], pb = ti * 2 + tj;
      double fc, fcR, fcS;
      fc_params(re, P.R[pb], P.S[pb], fc, fcR, fcS);
      if (fc == 0.0) continue;
      // environment sums of bond e (recomputed)
      double z[2] = {0.0, 0.0};
      for (int k = 0; k < nc; ++k) {
        if (k == e) continue;
        double4_32a uk = s_u[k];
        int tk = s_t[k], pk = ti * 2 + tk;
        double fck = fc_only(uk.w, P.R[pk], P.S[pk]);
        if (fck == 0.0) continue;
        double ct = (ue.x * uk.x + ue.y * uk.y + ue.z * uk.z) / (re * uk.w);
        int tri = pb * 2 + tk;
        for (int ll = 0; ll < 2; ++ll) {
          double c2 = P.c[tri][ll] * P.c[tri][ll], d2 = P.d[tri][ll] * P.d[tri][ll];
          double hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
          double ang = P.gamma[tri][ll] * (1.0 + c2 * hm * hm / (d2 * den));
          z[ll] += fck * ang * exp(P.alpha[tri][ll] * (re - uk.w));
        }
      }
      // bond order (Eq. 7) and its parameter derivatives, via ln b = e (ln S - ln S0)
      double pp = P.p[pb], sg = P.sigma[pb], ex = 1.0 / (2.0 * sg * pp);
      double zn[2], Z[2], t[2], lnz[2];
      for (int ll = 0; ll < 2; ++ll) {
        zn[ll] = z[ll] > 0.0 ? pow(z[ll], P.n[pb][ll]) : 0.0;
        lnz[ll] = z[ll] > 0.0 ? log(z[ll]) : 0.0;
        Z[ll] = P.g[pb][ll] + zn[ll];
        t[ll] = pow(Z[ll], -pp);
      }
      double Ssum = t[0] + t[1];
      double s0a = pow(P.g[pb][0], -pp), s0b = pow(P.g[pb][1], -pp), S0 = s0a + s0b;
      double lnb = ex * (log(Ssum) - log(S0));
      double b = exp(lnb);
      double dq = qi - q[s_j[e]];
      double cq = 1.0 - P.kappa[pb] * dq * dq;
      double e1 = exp(-P.lambda1[pb] * re), e2 = exp(-P.lambda2[pb] * re);
      double fR = P.A[pb] * e1, fA = P.B[pb] * e2;
      double V = fR - cq * b * fA;
      double Eb = -0.5 * fc * cq * fA;   // dE/db
      // pair parameters
      atomicAdd(&s_g[PG_A + pb], wi * 0.5 * fc * e1);
      atomicAdd(&s_g[PG_B + pb], wi * (-0.5) * fc * cq * b * e2);
      atomicAdd(&s_g[PG_L1 + pb], wi * (-0.5) * fc * re * fR);
      atomicAdd(&s_g[PG_L2 + pb], wi * 0.5 * fc * cq * b * fA * re);
      atomicAdd(&s_g[PG_KAPPA + pb], wi * 0.5 * fc * dq * dq * b * fA);
      atomicAdd(&s_g[PG_R + pb], wi * 0.5 * fcR * V);
      atomicAdd(&s_g[PG_S + pb], wi * 0.5 * fcS * V);
      // bond-order parameters
      double dlnS_dp = -(t[0] * log(Z[0]) + t[1] * log(Z[1])) / Ssum;
      double dlnS0_dp = -(s0a * log(P.g[pb][0]) + s0b * log(P.g[pb][1])) / S0;
      double wb = wi * Eb * b;
      atomicAdd(&s_g[PG_SIGMA + pb], wb * (-lnb / sg));
      atomicAdd(&s_g[PG_P + pb], wb * (-lnb / pp + ex * (dlnS_dp - dlnS0_dp)));
      for (int ll = 0; ll < 2; ++ll) {
        double dg = ex * (-pp * t[ll] / (Z[ll] * Ssum) + pp * pow(P.g[pb][ll], -pp - 1.0) / S0);
        atomicAdd(&s_g[PG_G + pb * 2 + ll], wb * dg);
        double dn = z[ll] > 0.0 ? ex * (-pp * t[ll] / (Z[ll] * Ssum)) * zn[ll] * lnz[ll] : 0.0;
        atomicAdd(&s_g[PG_N + pb * 2 + ll], wb * dn);
      }
      // dE/dzeta_l = Eb db/dzeta_l = Eb b (d ln b / d zeta_l)
      double Ez[2];
      for (int ll = 0; ll < 2; ++ll)
        Ez[ll] = z[ll] > 0.0
                     ? Eb * b * ex * (-pp * t[ll] / (Z[ll] * Ssum)) * P.n[pb][ll] * zn[ll] / z[ll]
                     : 0.0;
      // triplet parameters and the cutoff of the (i, k) pairs inside zeta
      for (int k = 0; k < nc; ++k) {
        if (k == e) continue;
        double4_32a uk = s_u[k];
        int tk = s_t[k], pk = ti * 2 + tk;
        double fck, fkR, fkS;
        fc_params(uk.w, P.R[pk], P.S[pk], fck, fkR, fkS);
        if (fck == 0.0) continue;
        double ct = (ue.x * uk.x + ue.y * uk.y + ue.z * uk.z) / (re * uk.w);
        int tri = pb * 2 + tk;
        for (int ll = 0; ll < 2; ++ll) {
          if (Ez[ll] == 0.0) continue;
          double cc = P.c[tri][ll], dd = P.d[tri][ll], gm = P.gamma[tri][ll];
          double c2 = cc * cc, d2 = dd * dd;
          double hm = P.h[tri][ll] - ct, den = d2 + hm * hm;
          double angg = 1.0 + c2 * hm * hm / (d2 * den);   // ang / gamma
          double dr = re - uk.w;
          double exl = exp(P.alpha[tri][ll] * dr);
          double wz = wi * Ez[ll];
          atomicAdd(&s_g[PG_GAMMA + tri * 2 + ll], wz * fck * angg * exl);
          atomicAdd(&s_g[PG_C + tri * 2 + ll], wz * fck * gm * 2.0 * cc * hm * hm / (d2 * den) * exl);
          atomicAdd(&s_g[PG_D + tri * 2 + ll],
                    wz * fck * 2.0 * gm * c2 * dd * (1.0 / (den * den) - 1.0 / (d2 * d2)) * exl);
          atomicAdd(&s_g[PG_H + tri * 2 + ll], wz * fck * gm * 2.0 * c2 * hm / (den * den) * exl);
          atomicAdd(&s_g[PG_ALPHA + tri * 2 + ll], wz * fck * gm * angg * dr * exl);
          atomicAdd(&s_g[PG_R + pk], wz * fkR * gm * angg * exl);
          atomicAdd(&s_g[PG_S + pk], wz * fkS * gm * angg * exl);
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// Charge-kernel and self-energy parameters: one thread per atom over all of
// its entries (each unordered pair appears in both atoms' lists, hence the
// 1/2 of the energy). Block sums in shared memory.
__global__ void __launch_bounds__(256)
    k_pgrad_coul(int N, int ld, const double4_32a* __restrict__ u, const int* __restrict__ rep,
                 const RepInfo* __restrict__ reps, const int2* __restrict__ nl, 
                 const int* __restrict__ nall, const double* __restrict__ q, const double* __restrict__ wrep,
                 ctbop_params P, double* __restrict__ grad) {
  __shared__ double s_g[PG_NPARAM];
  for (int k = threadIdx.x; k < PG_NPARAM; k += blockDim.x) s_g[k] = 0.0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double wi = wrep[rep[i]];
    if (wi != 0.0) {
      double4_32a ui = u[i];
      int ti = (int)ui.w;
      double qi = q[i];
      atomicAdd(&s_g[PG_E0 + ti], wi);
      atomicAdd(&s_g[PG_CHI + ti], wi * qi);
      atomicAdd(&s_g[PG_J + ti], wi * qi * qi);
      const RepInfo& ri = reps[rep[i]];
      double rc = P.r_coul, ke = P.k_e;
      double gke = 0.0, grc = 0.0, gga[2] = {0.0, 0.0};
      int na = nall[i];
      for (int e = 0; e < na; ++e) {
        size_t idx = (size_t)e * ld + i;
        int j = nl[idx].x;
        double4_32a uj = u[j];
        int dx, dy, dz;
        unpack_code(nl[idx].y, dx, dy, dz);
        double rx = (uj.x - ui.x) + dx * ri.hc[0], ry = (uj.y - ui.y) + dy * ri.hc[1],
               rz = (uj.z - ui.z) + dz * ri.hc[2];
        double r = sqrt(rx * rx + ry * ry + rz * rz);
        double x = r / rc;
        if (x >= 1.0) continue;
        int tj = (int)uj.w;
        double ga = P.gamma_c[ti], gb = P.gamma_c[tj];
        double gs3 = pow(ga * gb, -1.5);
        double x2 = x * x, x3 = x2 * x, x4 = x2 * x2, xm = x - 1.0;
        double T = 1.0 + x4 * (-35.0 + x * (84.0 + x * (-70.0 + 20.0 * x)));
        double dT = 140.0 * x3 * xm * xm * xm;
        double D = cbrt(r * r * r + gs3), iD = 1.0 / D;
        double K = ke * T * iD;
        double w = 0.5 * qi * q[j];
        gke += w * K / ke;
        grc += w * ke * dT * (-r / (rc * rc)) * iD;
        double dK_dgs3 = -ke * T * iD * iD * iD * iD / 3.0;
        gga[ti] += w * dK_dgs3 * (-1.5 * gs3 / ga);
        gga[tj] += w * dK_dgs3 * (-1.5 * gs3 / gb);
      }
      atomicAdd(&s_g[PG_KE], wi * gke);
      atomicAdd(&s_g[PG_RCOUL], wi * grc);
      atomicAdd(&s_g[PG_GAMMA_C], wi * gga[0]);
      atomicAdd(&s_g[PG_GAMMA_C + 1], wi * gga[1]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < PG_NPARAM; k += blockDim.x)
    if (s_g[k] != 0.0) atomicAdd(grad + k, s_g[k]);
}

// dE/dq_i = (H q)_i + chi_i at the assembled matrix (diagonal without
// self-images plus every stored entry, self-images included), FP64.
__global__ void k_charge_grad(int N, int ld, const int2* __restrict__ nl, const int* __restrict__ nall,
                              const double* __restrict__ M, const double* __restrict__ Dg,
                              const int* __restrict__ type, TypeParams T, const double* __restrict__ q,
                              double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = Dg[i] * q[i] + T.chi[type[i]];
  int na = nall[i];
  for (int e = 0; e < na; ++e) {
    size_t idx = (size_t)e * ld + i;
    s += M[idx] * q[nl[idx].x];
  }
  out[i] = s;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_param_grad(const DevState& S, const ctbop_params& P, const double* wrep, double* grad,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(double) * PG_NPARAM, st);
  if (e != cudaSuccess || S.N == 0) return e;
  size_t sm = (size_t)PG_APB * S.cap_cov * (sizeof(double4_32a) + 2 * sizeof(int));
  e = cudaFuncSetAttribute(k_pgrad_cov, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_pgrad_cov<<<(S.N + PG_APB - 1) / PG_APB, PG_APB * PG_GRP, sm, st>>>(
      S.N, S.cap_cov, S.ld, (const double4_32a*)S.u, S.rep, S.reps, S.nl, S.ncov, S.q, wrep, P, grad);
  k_pgrad_coul<<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.ld, (const double4_32a*)S.u, S.rep, S.reps, S.nl,
                                                   S.nall, S.q, wrep, P, grad);
  return cudaGetLastError();
}

void launch_charge_grad(const DevState& S, const TypeParams& T, double* out, cudaStream_t st) {
  if (S.N == 0) return;
  k_charge_grad<<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.ld, S.nl, S.nall, (const double*)S.M,
                                                    (const double*)S.Dg, S.type, T, S.q, out);
}

}  // namespace ct
