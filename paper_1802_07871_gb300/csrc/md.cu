// md.cu — velocity-Verlet kick + drift, cell-local coordinates and the
// neighbour-skin test (the MD of Sec. 3.3: frozen substrate atoms never
// move; their forces are still computed).
#include "internal.cuh"
#include "kernels.h"

namespace ct {

// v += dt/2 F/m; x += dt v (mobile atoms); refresh the cell-local
// coordinates; request a list rebuild when an atom moved more than half the
// skin since the last rebuild. With a Nose-Hoover thermostat on the replica
// (NVT, Sec. 3.3), first the thermostat's half-step xi' = xi + dt/2 (2K - g kB
// T0) / Qm from the kinetic energy K the previous step left in rep_acc, and
// the velocity scaling by exp(-xi' dt / 2); the replica's first atom records
// xi' for the end of the step.
template <class R>
__global__ void k_kick_drift(int N, double dt, double half_skin2, const int* __restrict__ type,
                             const uint8_t* __restrict__ frozen, const int* __restrict__ rep,
                             const RepInfo* __restrict__ reps, const int4* __restrict__ cell4,
                             const double* __restrict__ F, double* __restrict__ v, double* __restrict__ x,
                             const double* __restrict__ xref, typename Vec4<R>::T* __restrict__ u,
                             TypeParams T, int* __restrict__ flag, double* __restrict__ nh,
                             const double* __restrict__ rep_acc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int ti = type[i];
  double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  int r = rep[i];
  double scale = 1.0;
  if (nh[(size_t)r * NH_STRIDE + NH_ON] != 0.0) {
    const double* h = nh + (size_t)r * NH_STRIDE;
    double K = rep_acc[(size_t)r * RA_STRIDE + RA_KE];
    double xh = h[NH_XI] + 0.5 * dt * (2.0 * K - h[NH_GKT]) * h[NH_QINV];
    scale = exp(-0.5 * dt * xh);
    if (i == reps[r].atom_off) nh[(size_t)r * NH_STRIDE + NH_XIH] = xh;
  }
  if (!frozen[i]) {
    v[3 * i] *= scale;
    v[3 * i + 1] *= scale;
    v[3 * i + 2] *= scale;
    double s = 0.5 * dt * by_type(T.inv_mass_acc, ti);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double vv = v[3 * i + d] + s * F[3 * i + d];
      v[3 * i + d] = vv;
      xi[d] += dt * vv;
      x[3 * i + d] = xi[d];
    }
  }
  const RepInfo& ri = reps[rep[i]];
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

// End of an NVT step, one thread per replica: xi = xi' + dt/2 (2K - g kB T0)
// / Qm with the kinetic energy of the step's final velocities, eta += dt xi'.
__global__ void k_nh_end(int R, double dt, double* __restrict__ nh, const double* __restrict__ rep_acc) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    double* h = nh + (size_t)r * NH_STRIDE;
    if (h[NH_ON] == 0.0) continue;
    double K = rep_acc[(size_t)r * RA_STRIDE + RA_KE];
    h[NH_ETA] += dt * h[NH_XIH];
    h[NH_XI] = h[NH_XIH] + 0.5 * dt * (2.0 * K - h[NH_GKT]) * h[NH_QINV];
  }
}

void launch_nh_end(const DevState& S, double dt, cudaStream_t st) {
  k_nh_end<<<1, 256, 0, st>>>(S.R, dt, S.nh, S.rep_acc);
}

__global__ void k_zero_acc(int n, double* __restrict__ a, int* __restrict__ stiff_n, int* __restrict__ acc_mode,
                           const RepInfo* __restrict__ reps, int* __restrict__ flag_n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    // the previous evaluation's sum of |F|^2 selects this one's precision
    // mode (the accurate mode below an RMS force of ACC_RMS, and after a
    // reset of the sum)
    if (i % RA_STRIDE == RA_F2) {
      const int r = i / RA_STRIDE;
      acc_mode[r] = a[i] < 3.0 * (double)reps[r].natoms * (ACC_RMS * ACC_RMS) ? 1 : 0;
    }
    a[i] = 0.0;
  }
  if (i == 0) {   // the queues of this evaluation
    *stiff_n = 0;
    if (flag_n) *flag_n = 0;
  }
}

template <class R>
void launch_kick_drift(const DevState& S, const TypeParams& T, double dt, double half_skin2, cudaStream_t st) {
  if (S.N == 0) return;
  k_kick_drift<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, dt, half_skin2, S.type, S.frozen, S.rep, S.reps,
                                                     S.cell4, S.F, S.v, S.x, S.xref,
                                                     (typename Vec4<R>::T*)S.u, T, S.flag_rebuild, S.nh,
                                                     S.rep_acc);
}

void launch_zero_acc(const DevState& S, cudaStream_t st) {
  int n = S.R * RA_STRIDE;
  k_zero_acc<<<(n + 255) / 256, 256, 0, st>>>(n, S.rep_acc, S.stiff_n, S.acc_mode, S.reps, S.flag_n);
}

template void launch_kick_drift<float>(const DevState&, const TypeParams&, double, double, cudaStream_t);
template void launch_kick_drift<double>(const DevState&, const TypeParams&, double, double, cudaStream_t);

}  // namespace ct
