// relax.cu — energy minimisation (the paper relaxes and cools structures to
// 0 K, Sec. 3, without naming a method): FIRE (Bitzek et al., Phys. Rev.
// Lett. 97, 170201 (2006)) with the semi-implicit Euler step, one FIRE state
// per replica, on E(x) = min_q E(x, q) (each evaluation solves the charges).
//
// One iteration: k_fire_reduce sums P = F.v, |v|^2, |F|^2 and max |F_i|^2
// over each replica's mobile atoms and, in its last block, advances every
// replica's state (converged, or the downhill/uphill rule that sets dt,
// alpha and the velocity mixing); k_fire_move mixes, kicks and drifts; then
// the usual evaluation. Converged replicas stop moving.
#include "internal.cuh"
#include "kernels.h"

namespace ct {

__global__ void k_fire_reduce(int N, int R, const int* __restrict__ rep, const uint8_t* __restrict__ frozen,
                              const double* __restrict__ F, const double* __restrict__ v,
                              double* __restrict__ fire, FireCfg cfg, int* __restrict__ blocks,
                              int* __restrict__ active) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  RepAcc<3> acc;
  acc.init();
  double f2 = 0.0;
  int r = -1;
  if (i < N) {
    int ri = rep[i];
    if (!frozen[i] && fire[(size_t)ri * FI_STRIDE + FI_DONE] == 0.0) {
      r = ri;
      double fx = F[3 * i], fy = F[3 * i + 1], fz = F[3 * i + 2];
      double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
      acc.to(r, fire, FI_STRIDE);
      acc.v[0] += fx * vx + fy * vy + fz * vz;
      acc.v[1] += vx * vx + vy * vy + vz * vz;
      f2 = fx * fx + fy * fy + fz * fz;
      acc.v[2] += f2;
    }
  }
  lane_flush<3>(acc, fire, FI_STRIDE);   // slots FI_P, FI_VV, FI_FF
  int r0 = __shfl_sync(CT_FULL, r, 0);
  if (__all_sync(CT_FULL, r == r0)) {
    double m = warp_max(f2);
    if ((threadIdx.x & 31) == 0 && r0 >= 0 && m > 0.0) atomic_max_nonneg(fire + (size_t)r0 * FI_STRIDE + FI_FMAX2, m);
  } else if (r >= 0 && f2 > 0.0) {
    atomic_max_nonneg(fire + (size_t)r * FI_STRIDE + FI_FMAX2, f2);
  }
  if (last_block(blocks)) {
    __shared__ int s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < R; q += blockDim.x) {
      double* f = fire + (size_t)q * FI_STRIDE;
      double P = __ldcg(f + FI_P), vv = __ldcg(f + FI_VV), ff = __ldcg(f + FI_FF), fm2 = __ldcg(f + FI_FMAX2);
      f[FI_P] = f[FI_VV] = f[FI_FF] = f[FI_FMAX2] = 0.0;
      f[FI_LASTF2] = fm2;
      if (f[FI_DONE] != 0.0) continue;
      if (fm2 < cfg.fmax2 || f[FI_ITERS] >= cfg.max_iter) {
        f[FI_DONE] = fm2 < cfg.fmax2 ? 1.0 : -1.0;   // converged / gave up
        continue;
      }
      f[FI_ITERS] += 1.0;
      if (P >= 0.0) {   // downhill (a start from rest included)
        f[FI_NPOS] += 1.0;
        if (f[FI_NPOS] > cfg.n_min) {
          f[FI_DT] = fmin(f[FI_DT] * cfg.f_inc, cfg.dt_max);
          f[FI_ALPHA] *= cfg.f_alpha;
        }
        f[FI_CV] = 1.0 - f[FI_ALPHA];
        f[FI_CF] = ff > 0.0 ? f[FI_ALPHA] * sqrt(vv / ff) : 0.0;
      } else {          // uphill: slow down and restart from rest
        f[FI_NPOS] = 0.0;
        f[FI_DT] *= cfg.f_dec;
        f[FI_ALPHA] = cfg.alpha0;
        f[FI_CV] = f[FI_CF] = 0.0;
      }
      atomicAdd(&s_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *active = s_active;
      blocks[0] = 0;
    }
  }
}

// v = cv v + cf F; v += dt F / m; x += dt v (mobile atoms of moving
// replicas; everything else keeps v = 0); cell-local coordinates refreshed
// and a list rebuild requested past half the skin, as in the MD drift.
template <class R>
__global__ void k_fire_move(int N, double half_skin2, const int* __restrict__ type, const uint8_t* __restrict__ frozen,
                            const int* __restrict__ rep, const RepInfo* __restrict__ reps,
                            const int4* __restrict__ cell4, const double* __restrict__ F, double* __restrict__ v,
                            double* __restrict__ x, const double* __restrict__ xref,
                            typename Vec4<R>::T* __restrict__ u, TypeParams T, const double* __restrict__ fire,
                            int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int r = rep[i];
  const double* f = fire + (size_t)r * FI_STRIDE;
  if (frozen[i] || f[FI_DONE] != 0.0) {
    v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
    return;
  }
  double cv = f[FI_CV], cf = f[FI_CF], dt = f[FI_DT];
  int ti = type[i];
  double s = dt * by_type(T.inv_mass_acc, ti);
  double xi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double Fd = F[3 * i + d];
    double vv = cv * v[3 * i + d] + cf * Fd + s * Fd;
    v[3 * i + d] = vv;
    xi[d] = x[3 * i + d] + dt * vv;
    x[3 * i + d] = xi[d];
  }
  const RepInfo& ri = reps[r];
  int4 c = cell4[i];
  typename Vec4<R>::T uu;
  uu.x = (R)(xi[0] - c.x * ri.hc[0]);
  uu.y = (R)(xi[1] - c.y * ri.hc[1]);
  uu.z = (R)(xi[2] - c.z * ri.hc[2]);
  uu.w = (R)ti;
  u[i] = uu;
  double dx = xi[0] - xref[3 * i], dy = xi[1] - xref[3 * i + 1], dz = xi[2] - xref[3 * i + 2];
  if (dx * dx + dy * dy + dz * dz > half_skin2) *flag = 1;
}

void launch_fire_reduce(const DevState& S, double* fire, const FireCfg& cfg, int* blocks, int* active,
                        cudaStream_t st) {
  int n = S.N > 0 ? S.N : 1;
  k_fire_reduce<<<(n + 255) / 256, 256, 0, st>>>(S.N, S.R, S.rep, S.frozen, S.F, S.v, fire, cfg, blocks, active);
}

template <class R>
void launch_fire_move(const DevState& S, const TypeParams& T, const double* fire, double half_skin2,
                      cudaStream_t st) {
  if (S.N == 0) return;
  k_fire_move<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, half_skin2, S.type, S.frozen, S.rep, S.reps, S.cell4,
                                                    S.F, S.v, S.x, S.xref, (typename Vec4<R>::T*)S.u, T, fire,
                                                    S.flag_rebuild);
}

template void launch_fire_move<float>(const DevState&, const TypeParams&, const double*, double, cudaStream_t);
template void launch_fire_move<double>(const DevState&, const TypeParams&, const double*, double, cudaStream_t);

}  // namespace ct
