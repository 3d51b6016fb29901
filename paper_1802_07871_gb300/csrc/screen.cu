// screen.cu — the Si desorption screening of Sec. 3.3: covalent
// coordination (to find the surface atoms) and the leave-one-out batches
// whose energies give each candidate's removal energy.
//
// The removal energy of atom i is E(system without i) + E0_{t_i} - E(system),
// the rest held in place and both charge sets at their minimiser (the atom
// leaves neutral). The library evaluates the systems without i as replicas
// of one batch: k_loo_gather copies a source replica minus one atom into
// each batch replica, on the device.
#include <algorithm>

#include "internal.cuh"
#include "kernels.h"

namespace ct {

// Covalent coordination: list entries of atom i closer than the cutoff S of
// the pair (f_c > 0). The covalent part of the list holds every neighbour
// within S + skin, so the count is exact while the lists are valid.
template <class R>
__global__ void k_coordination(int N, int ld, const typename Vec4<R>::T* __restrict__ u,
                               const int* __restrict__ rep, const RepInfo* __restrict__ reps,
                               const int2* __restrict__ nl, const int* __restrict__ ncov, PotParams<R> P,
                               double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  typename Vec4<R>::T ui = u[i];
  int ti = (int)ui.w;
  const RepInfo& ri = reps[rep[i]];
  R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
  if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
  int n = 0, nc = ncov[i];
  for (int e = 0; e < nc; ++e) {
    int2 jc = nl[(size_t)e * ld + i];
    typename Vec4<R>::T uj = u[jc.x];
    int dx, dy, dz;
    unpack_code(jc.y, dx, dy, dz);
    R rx = (uj.x - ui.x) + (R)dx * hx, ry = (uj.y - ui.y) + (R)dy * hy, rz = (uj.z - ui.z) + (R)dz * hz;
    R S = P.Sout[ti * 2 + (int)uj.w];
    if (rx * rx + ry * ry + rz * rz < S * S) ++n;
  }
  out[i] = (double)n;
}

template <class R>
void launch_coordination(const DevState& S, const PotParams<R>& P, double* out, cudaStream_t st) {
  if (S.N == 0) return;
  k_coordination<R><<<(S.N + 255) / 256, 256, 0, st>>>(S.N, S.ld, (const typename Vec4<R>::T*)S.u, S.rep,
                                                       S.reps, S.nl, S.ncov, P, out);
}

// Leave-one-out gather. Batch replica c copies source replica atoms
// [src_off[c], src_off[c] + src_n[c]) except the one at local index
// drop[c], in order, to [dst_off[c], dst_off[c] + src_n[c] - 1): positions,
// types, frozen flags and charges. Grid: x over atoms, y over replicas.
__global__ void k_loo_gather(const LooItem* __restrict__ items, const double* __restrict__ x,
                             const int* __restrict__ type, const uint8_t* __restrict__ frozen,
                             const double* __restrict__ q, double* __restrict__ ox, int* __restrict__ otype,
                             uint8_t* __restrict__ ofrozen, double* __restrict__ oq) {
  const LooItem it = items[blockIdx.y];
  int n = it.src_n - 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    long long src = it.src_off + (k < it.drop ? k : k + 1);
    long long dst = it.dst_off + k;
    ox[3 * dst] = x[3 * src];
    ox[3 * dst + 1] = x[3 * src + 1];
    ox[3 * dst + 2] = x[3 * src + 2];
    otype[dst] = type[src];
    ofrozen[dst] = frozen[src];
    oq[dst] = q[src];
  }
}

void launch_loo_gather(const LooItem* items, int n_items, int max_n, const DevState& S, double* ox, int* otype,
                       uint8_t* ofrozen, double* oq, cudaStream_t st) {
  if (n_items == 0 || max_n <= 1) return;
  dim3 grid((unsigned)std::min((max_n - 1 + 255) / 256, 64), (unsigned)n_items);
  k_loo_gather<<<grid, 256, 0, st>>>(items, S.x, S.type, S.frozen, S.q, ox, otype, ofrozen, oq);
}

template void launch_coordination<float>(const DevState&, const PotParams<float>&, double*, cudaStream_t);
template void launch_coordination<double>(const DevState&, const PotParams<double>&, double*, cudaStream_t);

}  // namespace ct
