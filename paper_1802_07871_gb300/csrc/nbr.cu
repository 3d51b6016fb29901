// nbr.cu — cell binning, counting sort and the per-atom neighbour lists.
//
// Every replica has its own orthorhombic cell grid (edge >= half the list
// radius, so a +-2 cell stencil covers the list sphere in large boxes; small
// periodic boxes get a wider stencil that walks through periodic images,
// self-images included). One list per atom: the covalent entries
// (r < S_ij + skin) first, then every other entry inside Rc + skin. An entry
// stores the atom index j and the stencil offset d in cells, which is exactly
// the cell-lattice vector from i's cell to j's image cell, so
// r_ij = u_j - u_i + d * h with u the offset from the owning cell's origin.
// Lists are stored column-major (entry e of atom i at e * ld + i) for the
// thread-per-atom consumers.
#include "internal.cuh"
#include "kernels.h"

namespace ct {

// ---------------------------------------------------------------- binning
template <class R>
__global__ void k_bin(int N, double* __restrict__ x, double* __restrict__ xref,
                      const int* __restrict__ type, const int* __restrict__ rep,
                      const RepInfo* __restrict__ reps, int4* __restrict__ cell4,
                      typename Vec4<R>::T* __restrict__ u, int* __restrict__ cell_count,
                      unsigned* __restrict__ err, const int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *flag == 0) return;
  const RepInfo& ri = reps[rep[i]];
  int c[3];
  double xi[3];
  bool bad = false;
  for (int d = 0; d < 3; ++d) {
    double v = x[3 * i + d];
    if (!isfinite(v)) { bad = true; v = 0.0; }
    if (ri.pbc[d]) {
      v = v - floor(v / ri.L[d]) * ri.L[d];
      if (v >= ri.L[d]) v -= ri.L[d];
      if (v < 0.0) v = 0.0;
    }
    xi[d] = v;
    int cc = (int)floor(v / ri.hc[d]);
    cc = cc < 0 ? 0 : (cc >= ri.n[d] ? ri.n[d] - 1 : cc);
    c[d] = cc;
  }
  if (bad) atomicOr(err, CT_ERR_NONFINITE);
  for (int d = 0; d < 3; ++d) {
    x[3 * i + d] = xi[d];
    xref[3 * i + d] = xi[d];
  }
  int gid = ri.cell_off + (c[2] * ri.n[1] + c[1]) * ri.n[0] + c[0];
  cell4[i] = make_int4(c[0], c[1], c[2], gid);
  typename Vec4<R>::T uu;
  uu.x = (R)(xi[0] - c[0] * ri.hc[0]);
  uu.y = (R)(xi[1] - c[1] * ri.hc[1]);
  uu.z = (R)(xi[2] - c[2] * ri.hc[2]);
  uu.w = (R)type[i];
  u[i] = uu;
  atomicAdd(cell_count + gid, 1);
}

// Exclusive scan in three launches: per-block scan + block totals, scan of
// the totals in one block, add back. 4096 elements per block, at most 1024
// blocks.
#define SCAN_T 1024
#define SCAN_E 4
__global__ void k_scan_block(int n, const int* __restrict__ in, int* __restrict__ out,
                             int* __restrict__ bsum, const int* __restrict__ flag) {
  __shared__ int s[SCAN_T];
  if (*flag == 0) return;
  int base = blockIdx.x * SCAN_T * SCAN_E + threadIdx.x * SCAN_E;
  int v[SCAN_E], tot = 0;
  for (int k = 0; k < SCAN_E; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    tot += v[k];
  }
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < SCAN_T; o <<= 1) {
    int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int run = s[threadIdx.x] - tot;
  for (int k = 0; k < SCAN_E; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = s[SCAN_T - 1];
}
__global__ void k_scan_top(int nb, int* __restrict__ bsum, int* __restrict__ total,
                           const int* __restrict__ flag) {
  __shared__ int s[SCAN_T];
  if (*flag == 0) return;
  int v = threadIdx.x < nb ? bsum[threadIdx.x] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < SCAN_T; o <<= 1) {
    int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (threadIdx.x < nb) bsum[threadIdx.x] = s[threadIdx.x] - v;
  if (threadIdx.x == SCAN_T - 1) *total = s[SCAN_T - 1];
}
__global__ void k_scan_add(int n, int* __restrict__ out, const int* __restrict__ bsum,
                           const int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && *flag) out[i] += bsum[i / (SCAN_T * SCAN_E)];
}

__global__ void k_scatter(int N, const int4* __restrict__ cell4, const int* __restrict__ cell_start,
                          int* __restrict__ cell_fill, int* __restrict__ cell_atoms,
                          const int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *flag == 0) return;
  int g = cell4[i].w;
  int slot = atomicAdd(cell_fill + g, 1);
  cell_atoms[cell_start[g] + slot] = i;
}

// Sort each cell's atoms by index so the lists do not depend on atomic order.
__global__ void k_sort_cells(int C, const int* __restrict__ cell_start,
                             const int* __restrict__ cell_count, int* __restrict__ cell_atoms,
                             const int* __restrict__ flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C || *flag == 0) return;
  int* a = cell_atoms + cell_start[c];
  int n = cell_count[c];
  for (int k = 1; k < n; ++k) {
    int v = a[k], m = k - 1;
    while (m >= 0 && a[m] > v) { a[m + 1] = a[m]; --m; }
    a[m + 1] = v;
  }
}

// ---------------------------------------------------------------- lists
#define MAXR 17  // stencil cells along x per row (half width <= 8)

__device__ inline int wrap_cell(int c, int n) {
  c %= n;
  return c < 0 ? c + n : c;
}

// One warp per atom. Two sweeps over the stencil: covalent entries first,
// then the remaining entries inside the charge cutoff.
template <class R>
__global__ void k_build(int N, const typename Vec4<R>::T* __restrict__ u,
                        const int4* __restrict__ cell4, const int* __restrict__ rep,
                        const RepInfo* __restrict__ reps, const int* __restrict__ cell_start,
                        const int* __restrict__ cell_count, const int* __restrict__ cell_atoms,
                        PotParams<R> P, int cap_cov, int cap_all, int ld, int* __restrict__ nbr,
                        int* __restrict__ code, int* __restrict__ ncov, int* __restrict__ nall,
                        int* __restrict__ maxcnt, unsigned* __restrict__ err,
                        const int* __restrict__ flag) {
  __shared__ int s_start[8][MAXR], s_cnt[8][MAXR], s_dx[8][MAXR];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= N || *flag == 0) return;
  const RepInfo& ri = reps[rep[i]];
  typename Vec4<R>::T ui = u[i];
  int ti = (int)ui.w;
  int4 ci = cell4[i];
  R hx = (R)ri.hc[0], hy = (R)ri.hc[1], hz = (R)ri.hc[2];
  int* col_nbr = nbr + i;
  int* col_code = code + i;
  // `count` is the number of stored entries (never above the capacities, so
  // every stored entry is a valid atom even after an overflow); `need`
  // counts what the lists would need, for regrowing them.
  int count = 0, count_cov = 0, need_cov = 0, need_all = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int cap_pass = pass == 0 ? cap_cov : cap_all;
    for (int dz = -ri.m[2]; dz <= ri.m[2]; ++dz) {
      int cz = ci.z + dz;
      if (ri.pbc[2]) cz = wrap_cell(cz, ri.n[2]);
      else if (cz < 0 || cz >= ri.n[2]) continue;
      for (int dy = -ri.m[1]; dy <= ri.m[1]; ++dy) {
        int cy = ci.y + dy;
        if (ri.pbc[1]) cy = wrap_cell(cy, ri.n[1]);
        else if (cy < 0 || cy >= ri.n[1]) continue;
        // the x cells of this row
        int nx = 2 * ri.m[0] + 1;
        __syncwarp();
        if (lane < nx) {
          int dx = lane - ri.m[0];
          int cx = ci.x + dx;
          bool ok = true;
          if (ri.pbc[0]) cx = wrap_cell(cx, ri.n[0]);
          else ok = (cx >= 0 && cx < ri.n[0]);
          int g = ok ? ri.cell_off + (cz * ri.n[1] + cy) * ri.n[0] + cx : 0;
          s_start[warp][lane] = ok ? cell_start[g] : 0;
          s_cnt[warp][lane] = ok ? cell_count[g] : 0;
          s_dx[warp][lane] = dx;
        }
        __syncwarp();
        int tot = 0;
        for (int k = 0; k < nx; ++k) tot += s_cnt[warp][k];
        for (int t0 = 0; t0 < tot; t0 += 32) {
          int t = t0 + lane;
          bool take = false;
          int j = 0, cd = 0;
          if (t < tot) {
            int k = 0, off = t;
            while (off >= s_cnt[warp][k]) { off -= s_cnt[warp][k]; ++k; }
            j = cell_atoms[s_start[warp][k] + off];
            int dx = s_dx[warp][k];
            typename Vec4<R>::T uj = u[j];
            R rx = (uj.x - ui.x) + (R)dx * hx;
            R ry = (uj.y - ui.y) + (R)dy * hy;
            R rz = (uj.z - ui.z) + (R)dz * hz;
            R r2 = rx * rx + ry * ry + rz * rz;
            int tj = (int)uj.w;
            bool self0 = (j == i) && dx == 0 && dy == 0 && dz == 0;
            bool cov = r2 < P.rcov_list2[ti * 2 + tj];
            take = !self0 && (pass == 0 ? cov : (!cov && r2 < P.rall_list2));
            cd = pack_code(dx, dy, dz);
          }
          unsigned bal = __ballot_sync(CT_FULL, take);
          if (take) {
            int pos = count + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap_pass) {
              col_nbr[(size_t)pos * ld] = j;
              col_code[(size_t)pos * ld] = cd;
            }
          }
          int nt = __popc(bal);
          if (pass == 0) need_cov += nt;
          need_all += nt;
          count = min(count + nt, cap_pass);
        }
      }
    }
    if (pass == 0) count_cov = count;
  }
  if (lane == 0) {
    ncov[i] = count_cov;
    nall[i] = count;
    atomicMax(maxcnt + 0, need_cov);
    atomicMax(maxcnt + 1, need_all);
    if (need_cov > cap_cov) atomicOr(err, CT_ERR_COV_OVERFLOW);
    if (need_all > cap_all) atomicOr(err, CT_ERR_NBR_OVERFLOW);
  }
}

// Reverse covalent entry: for entry e of i pointing at (j, d), the entry of
// j pointing at (i, -d).
__global__ void k_rev(int N, int cap_cov, int ld, const int* __restrict__ nbr,
                      const int* __restrict__ code, const int* __restrict__ ncov,
                      int* __restrict__ rev, unsigned* __restrict__ err,
                      const int* __restrict__ flag) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * cap_cov || *flag == 0) return;
  int i = (int)(t % N), e = (int)(t / N);   // consecutive threads: consecutive atoms
  int nc = min(ncov[i], cap_cov);
  if (e >= nc) return;
  int j = nbr[(size_t)e * ld + i];
  int dx, dy, dz;
  unpack_code(code[(size_t)e * ld + i], dx, dy, dz);
  int want = pack_code(-dx, -dy, -dz);
  int ncj = min(ncov[j], cap_cov);
  int found = -1;
  for (int k = 0; k < ncj; ++k) {
    if (nbr[(size_t)k * ld + j] == i && code[(size_t)k * ld + j] == want) { found = k; break; }
  }
  if (found < 0) { atomicOr(err, CT_ERR_REV_MISSING); found = 0; }
  rev[(size_t)i * cap_cov + e] = found;
}

__global__ void k_zero_cells(int C, int* __restrict__ cell_count, int* __restrict__ cell_fill,
                             int* __restrict__ maxcnt, const int* __restrict__ flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (*flag == 0) return;
  if (c < C) { cell_count[c] = 0; cell_fill[c] = 0; }
  if (c < 2) maxcnt[c] = 0;
}

// Clear the rebuild request and count the rebuild (one thread).
__global__ void k_finish_rebuild(int* __restrict__ flag, long long* __restrict__ counter) {
  if (*flag) { *flag = 0; *counter += 1; }
}

// ---------------------------------------------------------------- launcher
template <class R>
void launch_rebuild(const DevState& S, const PotParams<R>& P, cudaStream_t st) {
  int N = S.N;
  if (N == 0) return;
  int tb = 256;
  int C = S.ncells;
  const int* f = S.flag_rebuild;
  k_zero_cells<<<(max(C, 2) + tb - 1) / tb, tb, 0, st>>>(C, S.cell_count, S.cell_fill, S.maxcnt, f);
  k_bin<R><<<(N + tb - 1) / tb, tb, 0, st>>>(N, S.x, S.xref, S.type, S.rep, S.reps, S.cell4,
                                              (typename Vec4<R>::T*)S.u, S.cell_count, S.err, f);
  int nb = (C + SCAN_T * SCAN_E - 1) / (SCAN_T * SCAN_E);
  k_scan_block<<<nb, SCAN_T, 0, st>>>(C, S.cell_count, S.cell_start, S.scan_tmp, f);
  k_scan_top<<<1, SCAN_T, 0, st>>>(nb, S.scan_tmp, S.scan_tmp + 1024, f);
  k_scan_add<<<(C + tb - 1) / tb, tb, 0, st>>>(C, S.cell_start, S.scan_tmp, f);
  k_scatter<<<(N + tb - 1) / tb, tb, 0, st>>>(N, S.cell4, S.cell_start, S.cell_fill, S.cell_atoms, f);
  k_sort_cells<<<(C + tb - 1) / tb, tb, 0, st>>>(C, S.cell_start, S.cell_count, S.cell_atoms, f);
  int wpb = 8;
  k_build<R><<<(N + wpb - 1) / wpb, wpb * 32, 0, st>>>(
      N, (const typename Vec4<R>::T*)S.u, S.cell4, S.rep, S.reps, S.cell_start, S.cell_count,
      S.cell_atoms, P, S.cap_cov, S.cap_all, S.ld, S.nbr, S.code, S.ncov, S.nall, S.maxcnt, S.err, f);
  size_t tot = (size_t)N * S.cap_cov;
  k_rev<<<(unsigned)((tot + tb - 1) / tb), tb, 0, st>>>(N, S.cap_cov, S.ld, S.nbr, S.code, S.ncov, S.rev,
                                                        S.err, f);
  k_finish_rebuild<<<1, 1, 0, st>>>(S.flag_rebuild, S.rebuild_count);
}

template void launch_rebuild<float>(const DevState&, const PotParams<float>&, cudaStream_t);
template void launch_rebuild<double>(const DevState&, const PotParams<double>&, cudaStream_t);

}  // namespace ct
