// rings.cu — ring statistics of the C network (Sec. 3.3 follows the numbers
// of 5-, 6- and 7-membered C rings and the in-plane orientation of the
// 6-membered ones). The paper gives no ring criterion; the library counts
// primitive rings: closed paths of distinct C atoms joined by C-C bonds
// shorter than a cutoff, whose bond vectors sum to zero (a path around a
// periodic box is no ring), with no shorter path in the graph between any
// two of their atoms (same displacement) than along the ring.
//
// One thread per C atom a enumerates the rings whose lowest atom index is a
// by a depth-first search over the covalent lists (atoms above a only,
// second atom below the last, so each ring is found once), checks the
// primitive condition with walks of at most three bonds (rings have at most
// 8 atoms), and appends a record.
#include <math.h>

#include "ctbop.h"
#include "internal.cuh"
#include "kernels.h"

namespace ct {

#define RING_MAX 8
#define RING_CLOSE2 0.01   // |sum of bond vectors|^2 below which a path closes (0.1 A)

template <class R>
struct RingGraph {
  const typename Vec4<R>::T* u;
  const int* rep;
  const RepInfo* reps;
  const int2* nl;
  const int* ncov;
  int ld;
  R cut2;
  // neighbour e of atom v if it is a C-C bond: bond vector out, true
  __device__ bool bond(int v, int e, int& w, R& bx, R& by, R& bz) const {
    int2 jc = nl[(size_t)e * ld + v];
    typename Vec4<R>::T uv = u[v], uw = u[jc.x];
    if ((int)uw.w != 1) return false;
    const RepInfo& ri = reps[rep[v]];
    R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
    if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
    int dx, dy, dz;
    unpack_code(jc.y, dx, dy, dz);
    bx = (uw.x - uv.x) + (R)dx * hx;
    by = (uw.y - uv.y) + (R)dy * hy;
    bz = (uw.z - uv.z) + (R)dz * hz;
    if (bx * bx + by * by + bz * bz >= cut2) return false;
    w = jc.x;
    return true;
  }
};

// A walk of 1..len bonds from s reaching t with displacement (dx, dy, dz)?
template <class R>
__device__ bool shortcut(const RingGraph<R>& G, int s, int t, R dx, R dy, R dz, int len) {
  int node[3], eix[3];
  R px[3], py[3], pz[3];
  int depth = 0;
  node[0] = s;
  eix[0] = 0;
  px[0] = py[0] = pz[0] = R(0);
  while (depth >= 0) {
    int v = node[depth];
    if (eix[depth] >= G.ncov[v]) {
      --depth;
      continue;
    }
    int e = eix[depth]++;
    int w;
    R bx, by, bz;
    if (!G.bond(v, e, w, bx, by, bz)) continue;
    R qx = px[depth] + bx, qy = py[depth] + by, qz = pz[depth] + bz;
    if (w == t) {
      R ex = qx - dx, ey = qy - dy, ez = qz - dz;
      if (ex * ex + ey * ey + ez * ez < R(RING_CLOSE2)) return true;
    }
    if (depth + 1 < len) {
      ++depth;
      node[depth] = w;
      eix[depth] = 0;
      px[depth] = qx;
      py[depth] = qy;
      pz[depth] = qz;
    }
  }
  return false;
}

template <class R>
__global__ void k_rings(int N, RingGraph<R> G, const double* __restrict__ x, int max_size,
                        ctbop_ring* __restrict__ out, long long cap, unsigned long long* __restrict__ count) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= N || (int)G.u[a].w != 1 || G.ncov[a] == 0) return;
  int path[RING_MAX], eix[RING_MAX];
  R px[RING_MAX], py[RING_MAX], pz[RING_MAX];
  int depth = 0;
  path[0] = a;
  eix[0] = 0;
  px[0] = py[0] = pz[0] = R(0);
  while (depth >= 0) {
    int v = path[depth];
    if (eix[depth] >= G.ncov[v]) {
      --depth;
      continue;
    }
    int e = eix[depth]++;
    int w;
    R bx, by, bz;
    if (!G.bond(v, e, w, bx, by, bz)) continue;
    R qx = px[depth] + bx, qy = py[depth] + by, qz = pz[depth] + bz;
    if (w == a) {
      int n = depth + 1;
      if (n < 3 || qx * qx + qy * qy + qz * qz >= R(RING_CLOSE2) || path[1] >= path[depth]) continue;
      bool prim = true;
      for (int s = 0; s < n && prim; ++s)
        for (int t = s + 2; t < n && prim; ++t) {
          int k = min(t - s, n - (t - s));
          if (k >= 2 && shortcut(G, path[s], path[t], px[t] - px[s], py[t] - py[s], pz[t] - pz[s], k - 1))
            prim = false;
        }
      if (!prim) continue;
      double cx = 0, cy = 0, cz = 0;
      for (int k = 0; k < n; ++k) {
        cx += (double)px[k];
        cy += (double)py[k];
        cz += (double)pz[k];
      }
      double orient = nan("");
      if (n == 6) {
        double sc = 0.0, ss = 0.0;
        for (int k = 0; k < 3; ++k) {
          double psi = 6.0 * atan2((double)(py[k + 3] - py[k]), (double)(px[k + 3] - px[k]));
          sc += cos(psi);
          ss += sin(psi);
        }
        orient = fmod(atan2(ss, sc) / 6.0 * (180.0 / M_PI) + 60.0, 60.0);
      }
      unsigned long long slot = atomicAdd(count, 1ull);
      if ((long long)slot < cap) {
        ctbop_ring rr;
        rr.replica = G.rep[a];
        rr.size = n;
        rr.centre[0] = x[3 * a] + cx / n;
        rr.centre[1] = x[3 * a + 1] + cy / n;
        rr.centre[2] = x[3 * a + 2] + cz / n;
        rr.orientation = orient;
        out[slot] = rr;
      }
      continue;
    }
    if (w <= a || depth + 1 >= max_size) continue;
    bool seen = false;
    for (int k = 1; k <= depth; ++k) seen = seen || path[k] == w;
    if (seen) continue;
    ++depth;
    path[depth] = w;
    eix[depth] = 0;
    px[depth] = qx;
    py[depth] = qy;
    pz[depth] = qz;
  }
}

template <class R>
void launch_rings(const DevState& S, double bond_cut, int max_size, ctbop_ring* out, long long cap,
                  unsigned long long* count, cudaStream_t st) {
  if (S.N == 0) return;
  RingGraph<R> G{(const typename Vec4<R>::T*)S.u, S.rep, S.reps, S.nl, S.ncov, S.ld, (R)(bond_cut * bond_cut)};
  k_rings<R><<<(S.N + 127) / 128, 128, 0, st>>>(S.N, G, S.x, max_size, out, cap, count);
}

template void launch_rings<float>(const DevState&, double, int, ctbop_ring*, long long, unsigned long long*,
                                  cudaStream_t);
template void launch_rings<double>(const DevState&, double, int, ctbop_ring*, long long, unsigned long long*,
                                   cudaStream_t);

}  // namespace ct
