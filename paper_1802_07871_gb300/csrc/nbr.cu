// nbr.cu — cell binning, counting sort and the per-atom neighbour lists.
//
// Every replica has its own orthorhombic cell grid (edge >= half the list
// radius, so a +-2 cell stencil covers the list sphere in large boxes; small
// periodic boxes get a wider stencil that walks through periodic images,
// self-images included). One list per atom: the covalent entries
// (r < S_ij + skin) first, then the core (r < Rc - skin: these stay inside
// Rc until the next rebuild, since a rebuild comes before any atom moves
// skin/2), then the shell (every other entry inside Rc + skin). An entry
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
__device__ inline int wrap_cell(int c, int n) {
  c %= n;
  return c < 0 ? c + n : c;
}

// Lists are built one warp per cell: the atoms of a cell share one stencil,
// so each candidate j of the stencil is loaded once and tested against every
// atom i of the cell (up to 32 at a time, staged in shared memory). The
// stencil's cells are taken in batches of BC; a warp scan of their counts
// flattens the batch into one candidate sequence that the lanes walk 32 at a
// time (a lane finds its cell by binary search over the prefix sums).
//
// A candidate farther than the list radius from the bounding box of the
// cell's atoms (of each group of up to 32 of them) cannot enter any of their
// rows: about half of the stencil's
// candidates on the SiC slabs (the stencil is a 5 x 5 x 5 block of
// half-radius cells). Each candidate is tested once against the box, and the
// survivors are staged in shared memory in stencil order; the pair tests
// against the cell's atoms, the costly part, run only on full batches of 32
// survivors (the last batch of a cell may be partial). The box test has a
// 1e-4 relative margin, so the rows are the same, entry for entry, as
// without it.
//
// The atoms of a cell have scattered indices, so the pass writes each atom's
// entries contiguously (row-major scratch `lst`, one int2 (j, code) per
// entry: a ballot's entries land on one or two lines) and k_list_transpose
// turns the rows into the column-major lists through shared-memory tiles.
// Column-major stores straight from here would each touch a different line,
// completed only much later by other warps: with lists far larger than L2
// the partial lines are evicted and written back piecemeal.
//
// One pass writes the three parts of a row into the scratch: covalent
// entries from slot 0, core entries from slot cap_cov up, shell entries
// from slot cap_all - 1 down. k_list_transpose then lays them out as
// [covalent | core | shell] without moving anything here. maxcnt receives
// the largest covalent count, the largest count of the rest (the list needs
// cap_cov + that) and the largest total.
//
// BW (warps per block) and BC (stencil cells per batch) only change how the
// cells are spread over blocks and how the stencil is chunked; every shape
// writes the same rows (see tune_build).
template <class R, int BW, int BC>
__global__ void __launch_bounds__(BW * 32)
    k_build(int C, const typename Vec4<R>::T* __restrict__ u, const int* __restrict__ cell_rep,
            const RepInfo* __restrict__ reps, const int* __restrict__ cell_start,
            const int* __restrict__ cell_count, const int* __restrict__ cell_atoms, PotParams<R> P,
            int cap_cov, int cap_all, int2* __restrict__ lst,
            int* __restrict__ ncov, int* __restrict__ nfix, int* __restrict__ nall, int* __restrict__ maxcnt,
            unsigned* __restrict__ err, const int* __restrict__ flag) {
  typedef typename Vec4<R>::T R4;
  __shared__ int s_st[BW][BC], s_pre[BW][BC + 1], s_cd[BW][BC];
  __shared__ R4 s_u[BW][32];
  __shared__ int s_i[BW][32];
  __shared__ int s_need[BW][3];
  // candidates that passed the box test, first in first out (up to 63 held)
  __shared__ R4 s_cu[BW][64];
  __shared__ int s_cj[BW][64], s_cc[BW][64];
  if (*flag == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int need_cov = 0, need_rest = 0, need_tot = 0;   // this lane's maxima over the atoms it owned
  // the largest list radius squared, widened by 1e-4 (relative) so that
  // rounding never drops a candidate the pair test below would keep
  R r2max = P.rall_list2;
#pragma unroll
  for (int k = 0; k < 4; ++k) r2max = max(r2max, P.rcov_list2[k]);
  r2max *= R(1.0001);
  for (int g = blockIdx.x * BW + warp; g < C; g += gridDim.x * BW) {
    int nci = cell_count[g];
    if (nci == 0) continue;
    const int ci0 = cell_start[g];
    const RepInfo& ri = reps[cell_rep[g]];
    const int loc = g - ri.cell_off;
    const int cx = loc % ri.n[0], cy = (loc / ri.n[0]) % ri.n[1], cz = loc / (ri.n[0] * ri.n[1]);
    const R hx = (R)ri.hc[0], hy = (R)ri.hc[1], hz = (R)ri.hc[2];
    const int sx = 2 * ri.m[0] + 1, sy = 2 * ri.m[1] + 1;
    const int ns = sx * sy * (2 * ri.m[2] + 1);
    for (int ib = 0; ib < nci; ib += 32) {
      const int ni = min(32, nci - ib);
      int my_i = -1, cnt_c = 0, cnt_k = 0, cnt_s = 0;
      // bounding box of this group's atoms (offsets from the cell origin)
      R lox = R(1e30), loy = R(1e30), loz = R(1e30), hix = R(-1e30), hiy = R(-1e30), hiz = R(-1e30);
      if (lane < ni) {
        my_i = cell_atoms[ci0 + ib + lane];
        const R4 ui = u[my_i];
        s_u[warp][lane] = ui;
        s_i[warp][lane] = my_i;
        lox = hix = ui.x;
        loy = hiy = ui.y;
        loz = hiz = ui.z;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lox = min(lox, __shfl_xor_sync(CT_FULL, lox, o));
        loy = min(loy, __shfl_xor_sync(CT_FULL, loy, o));
        loz = min(loz, __shfl_xor_sync(CT_FULL, loz, o));
        hix = max(hix, __shfl_xor_sync(CT_FULL, hix, o));
        hiy = max(hiy, __shfl_xor_sync(CT_FULL, hiy, o));
        hiz = max(hiz, __shfl_xor_sync(CT_FULL, hiz, o));
      }
      __syncwarp();
      // Pair tests of the first n staged candidates (one per lane) against
      // every atom of the group, in staging order, which is stencil order:
      // each row receives its entries in the same order as without staging.
      auto pair_tests = [&](int n) {
        const bool valid = lane < n;
        int j = -1, cd = 0;
        R4 uj;
        uj.x = uj.y = uj.z = uj.w = R(0);
        R ox = R(0), oy = R(0), oz = R(0);
        if (valid) {
          uj = s_cu[warp][lane];
          j = s_cj[warp][lane];
          cd = s_cc[warp][lane];
          int dx, dy, dz;
          unpack_code(cd, dx, dy, dz);
          ox = (R)dx * hx;
          oy = (R)dy * hy;
          oz = (R)dz * hz;
        }
        const int tj = (int)uj.w;
        const bool zero_off = cd == pack_code(0, 0, 0);
        for (int ii = 0; ii < ni; ++ii) {
          const R4 ui = s_u[warp][ii];
          const int i = s_i[warp][ii];
          R rx = (uj.x - ui.x) + ox, ry = (uj.y - ui.y) + oy, rz = (uj.z - ui.z) + oz;
          R r2 = rx * rx + ry * ry + rz * rz;
          bool self0 = zero_off && j == i;
          bool in = valid && !self0;
          bool cov = in && r2 < P.rcov_list2[(int)ui.w * 2 + tj];
          bool core = in && !cov && r2 < P.rcore_list2;
          bool shell = in && !cov && !core && r2 < P.rall_list2;
          unsigned bc = __ballot_sync(CT_FULL, cov), bk = __ballot_sync(CT_FULL, core);
          unsigned bs = __ballot_sync(CT_FULL, shell);
          int bcc = __shfl_sync(CT_FULL, cnt_c, ii), bck = __shfl_sync(CT_FULL, cnt_k, ii);
          int bcs = __shfl_sync(CT_FULL, cnt_s, ii);
          if (cov) {
            int pos = bcc + __popc(bc & lt);
            if (pos < cap_cov) lst[(size_t)i * cap_all + pos] = make_int2(j, cd);
          } else if (core) {
            int pos = cap_cov + bck + __popc(bk & lt);
            if (pos < cap_all) lst[(size_t)i * cap_all + pos] = make_int2(j, cd);
          } else if (shell) {
            // from the end of the row down; an overflow (core and shell
            // meeting) is flagged below and the lists regrow
            int pos = cap_all - 1 - (bcs + __popc(bs & lt));
            if (pos >= cap_cov) lst[(size_t)i * cap_all + pos] = make_int2(j, cd);
          }
          if (lane == ii) {
            cnt_c += __popc(bc);
            cnt_k += __popc(bk);
            cnt_s += __popc(bs);
          }
        }
        __syncwarp();
      };
      int nst = 0;   // staged candidates (warp-uniform, < 32 between batches)
      for (int sb = 0; sb < ns; sb += BC) {
        const int nb = min(BC, ns - sb);
        // this batch's cells: start, count (0 outside an open box) and offset code
        int cnt[BC / 32];
#pragma unroll
        for (int k = 0; k < BC / 32; ++k) {
          int c = k * 32 + lane, st = 0, n = 0, cd = 0;
          if (c < nb) {
            int sidx = sb + c;
            int dx = sidx % sx - ri.m[0], dy = (sidx / sx) % sy - ri.m[1], dz = sidx / (sx * sy) - ri.m[2];
            int ax = cx + dx, ay = cy + dy, az = cz + dz;
            bool ok = true;
            if (ri.pbc[0]) ax = wrap_cell(ax, ri.n[0]); else ok = ok && ax >= 0 && ax < ri.n[0];
            if (ri.pbc[1]) ay = wrap_cell(ay, ri.n[1]); else ok = ok && ay >= 0 && ay < ri.n[1];
            if (ri.pbc[2]) az = wrap_cell(az, ri.n[2]); else ok = ok && az >= 0 && az < ri.n[2];
            if (ok) {
              int gc = ri.cell_off + (az * ri.n[1] + ay) * ri.n[0] + ax;
              st = cell_start[gc];
              n = cell_count[gc];
            }
            cd = pack_code(dx, dy, dz);
            s_st[warp][c] = st;
            s_cd[warp][c] = cd;
          }
          cnt[k] = n;
        }
        // exclusive prefix sums of the counts, in batch order (cell k * 32 + lane)
        int T = 0;
#pragma unroll
        for (int k = 0; k < BC / 32; ++k) {
          int v = cnt[k], sc = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(CT_FULL, sc, o);
            if (lane >= o) sc += t;
          }
          if (k * 32 + lane < nb) s_pre[warp][k * 32 + lane] = T + sc - v;
          T += __shfl_sync(CT_FULL, sc, 31);
        }
        if (lane == 0) s_pre[warp][nb] = T;
        __syncwarp();
        for (int t0 = 0; t0 < T; t0 += 32) {
          const int t = t0 + lane;
          bool keep = false;
          int j = -1, cd = 0;
          R4 uj;
          if (t < T) {
            int lo = 0, hi = nb;   // largest k with s_pre[k] <= t
            while (hi - lo > 1) {
              int mid = (lo + hi) >> 1;
              if (s_pre[warp][mid] <= t) lo = mid; else hi = mid;
            }
            j = cell_atoms[s_st[warp][lo] + (t - s_pre[warp][lo])];
            cd = s_cd[warp][lo];
            uj = u[j];
            int dx, dy, dz;
            unpack_code(cd, dx, dy, dz);
            // distance from the candidate's image to the group's box: past
            // the list radius, no atom of the group can take it
            const R px = uj.x + (R)dx * hx, py = uj.y + (R)dy * hy, pz = uj.z + (R)dz * hz;
            const R bx = max(max(lox - px, px - hix), R(0));
            const R by = max(max(loy - py, py - hiy), R(0));
            const R bz = max(max(loz - pz, pz - hiz), R(0));
            keep = bx * bx + by * by + bz * bz <= r2max;
          }
          const unsigned bk = __ballot_sync(CT_FULL, keep);
          if (keep) {
            const int pos = nst + __popc(bk & lt);
            s_cu[warp][pos] = uj;
            s_cj[warp][pos] = j;
            s_cc[warp][pos] = cd;
          }
          nst += __popc(bk);
          __syncwarp();
          if (nst >= 32) {
            pair_tests(32);
            // move the rest (fewer than 32) to the front
            if (lane < nst - 32) {
              const R4 a = s_cu[warp][32 + lane];
              const int b = s_cj[warp][32 + lane], c = s_cc[warp][32 + lane];
              s_cu[warp][lane] = a;
              s_cj[warp][lane] = b;
              s_cc[warp][lane] = c;
            }
            nst -= 32;
            __syncwarp();
          }
        }
        __syncwarp();
      }
      if (nst > 0) pair_tests(nst);
      // counts of the three parts (k_list_transpose closes the gaps)
      if (lane < ni) {
        int cnt_r = cnt_k + cnt_s;
        int nc = min(cnt_c, cap_cov);
        bool over = cap_cov + cnt_r > cap_all;
        int nk = over ? 0 : cnt_k, ns = over ? 0 : cnt_s;   // an overflowed row is rebuilt after regrowth
        ncov[my_i] = nc;
        nfix[my_i] = nc + nk;
        nall[my_i] = nc + nk + ns;
        need_cov = max(need_cov, cnt_c);
        need_rest = max(need_rest, cnt_r);
        need_tot = max(need_tot, cnt_c + cnt_r);
        if (cnt_c > cap_cov) atomicOr(err, CT_ERR_COV_OVERFLOW);
        if (over) atomicOr(err, CT_ERR_NBR_OVERFLOW);
      }
      __syncwarp();
    }
  }
  // one atomicMax per block for each count
  need_cov = __reduce_max_sync(CT_FULL, (unsigned)need_cov);
  need_rest = __reduce_max_sync(CT_FULL, (unsigned)need_rest);
  need_tot = __reduce_max_sync(CT_FULL, (unsigned)need_tot);
  if (lane == 0) {
    s_need[warp][0] = need_cov;
    s_need[warp][1] = need_rest;
    s_need[warp][2] = need_tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0, c = 0;
    for (int w = 0; w < BW; ++w) {
      a = max(a, s_need[w][0]);
      b = max(b, s_need[w][1]);
      c = max(c, s_need[w][2]);
    }
    atomicMax(maxcnt + 0, a);
    atomicMax(maxcnt + 1, b);
    atomicMax(maxcnt + 2, c);
  }
}

// Row-major scratch -> column-major lists (entry e of atom i at e * ld + i),
// 32 atoms x TE entries per tile through shared memory (TE / 4 loads and
// stores in flight per thread); tiles past every row's end are skipped.
// Grid-strided over the tiles. Entry e of atom a comes from scratch slot e
// (covalent, e < ncov), cap_cov + e - ncov (core, e < nfix) or
// cap_all - 1 - (e - nfix) (shell).
#define TE 64
__global__ void __launch_bounds__(256)
    k_list_transpose(int N, int cap_cov, int cap_all, int ld, const int2* __restrict__ lst,
                     const int* __restrict__ ncov, const int* __restrict__ nfix, const int* __restrict__ nall,
                     int2* __restrict__ nl, const int* __restrict__ flag) {
  __shared__ int2 tile[32][TE + 1];
  if (*flag == 0) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ta = (N + 31) / 32, te = (cap_all + TE - 1) / TE;
  for (long long t = blockIdx.x; t < (long long)ta * te; t += gridDim.x) {
    const int a0 = (int)(t % ta) * 32, e0 = (int)(t / ta) * TE;
    int na = a0 + tx < N ? nall[a0 + tx] : 0;
    int nmax = __reduce_max_sync(CT_FULL, (unsigned)na);
    if (e0 >= nmax) continue;   // uniform over the block: every warp reads the same 32 counts
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int a = a0 + ty + 8 * r;
      if (a < N) {
        const int n = nall[a], nc = ncov[a], nf = nfix[a];
#pragma unroll
        for (int h = 0; h < TE / 32; ++h) {
          const int e = e0 + 32 * h + tx;
          if (e < n) {
            const int src = e < nc ? e : (e < nf ? cap_cov + (e - nc) : cap_all - 1 - (e - nf));
            tile[ty + 8 * r][32 * h + tx] = lst[(size_t)a * cap_all + src];
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TE / 8; ++r) {
      const int e = e0 + ty + 8 * r, a = a0 + tx;
      if (e < na) nl[(size_t)e * ld + a] = tile[tx][ty + 8 * r];
    }
    __syncthreads();
  }
}

// Reverse covalent entry: for entry e of i pointing at (j, d), the entry of
// j pointing at (i, -d). One thread per atom, grid-strided.
__global__ void k_rev(int N, int cap_cov, int ld, const int2* __restrict__ nl, const int* __restrict__ ncov,
                      int* __restrict__ rev, unsigned* __restrict__ err,
                      const int* __restrict__ flag) {
  if (*flag == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int nc = min(ncov[i], cap_cov);
    for (int e = 0; e < nc; ++e) {
      int j = nl[(size_t)e * ld + i].x;
      int dx, dy, dz;
      unpack_code(nl[(size_t)e * ld + i].y, dx, dy, dz);
      int want = pack_code(-dx, -dy, -dz);
      int ncj = min(ncov[j], cap_cov);
      int found = -1;
      for (int k = 0; k < ncj; ++k) {
        if (nl[(size_t)k * ld + j].x == i && nl[(size_t)k * ld + j].y == want) { found = k; break; }
      }
      if (found < 0) { atomicOr(err, CT_ERR_REV_MISSING); found = 0; }
      rev[(size_t)i * cap_cov + e] = found;
    }
  }
}

__global__ void k_zero_cells(int C, int* __restrict__ cell_count, int* __restrict__ cell_fill,
                             int* __restrict__ maxcnt, const int* __restrict__ flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (*flag == 0) return;
  if (c < C) { cell_count[c] = 0; cell_fill[c] = 0; }
  if (c < 3) maxcnt[c] = 0;
}

// Clear the rebuild request and count the rebuild (one thread).
__global__ void k_finish_rebuild(int* __restrict__ flag, long long* __restrict__ counter) {
  if (*flag) { *flag = 0; *counter += 1; }
}

// ---------------------------------------------------------------- launcher
// The list-build shapes (warps per block, stencil cells per batch), indexed
// by DevState::build_shape.
static const int kBuildShapes[BUILD_SHAPES][2] = {{2, 64}, {2, 128}, {4, 64}, {4, 128}, {8, 64}, {8, 128}};

template <class R, int BW, int BC>
static void launch_build_s(const DevState& S, const PotParams<R>& P, const int* f, cudaStream_t st) {
  // as many blocks as are resident at once (the cells are grid-strided, so
  // a block past that would run as a tail after the others)
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_build<R, BW, BC>, BW * 32, 0) != cudaSuccess || o < 1) o = 1;
    occ = o;
  }
  const int gb = S.nsm * occ;
  k_build<R, BW, BC><<<gb, BW * 32, 0, st>>>(S.ncells, (const typename Vec4<R>::T*)S.u, S.cell_rep, S.reps,
                                             S.cell_start, S.cell_count, S.cell_atoms, P, S.cap_cov, S.cap_all,
                                             S.lst, S.ncov, S.nfix, S.nall, S.maxcnt, S.err, f);
}

template <class R>
static void launch_build(const DevState& S, const PotParams<R>& P, int shape, const int* f, cudaStream_t st) {
  switch (shape) {
    case 0: launch_build_s<R, 2, 64>(S, P, f, st); break;
    case 1: launch_build_s<R, 2, 128>(S, P, f, st); break;
    case 2: launch_build_s<R, 4, 64>(S, P, f, st); break;
    case 4: launch_build_s<R, 8, 64>(S, P, f, st); break;
    case 5: launch_build_s<R, 8, 128>(S, P, f, st); break;
    default: launch_build_s<R, 4, 128>(S, P, f, st); break;
  }
}

int build_shape_index(int warps, int batch) {
  for (int k = 0; k < BUILD_SHAPES; ++k)
    if (kBuildShapes[k][0] == warps && kBuildShapes[k][1] == batch) return k;
  return -1;
}

void build_shape_of(int k, int* warps, int* batch) {
  if (k < 0 || k >= BUILD_SHAPES) k = 3;
  *warps = kBuildShapes[k][0];
  *batch = kBuildShapes[k][1];
}

// List-build shape, on the lists just built: each shape rebuilds the rows
// from the same cells and positions (the same rows again, so nothing needs
// restoring), one warm-up and two timed launches under an always-set flag;
// the fastest is kept. The rebuild flag itself is untouched.
template <class R>
cudaError_t tune_build(DevState& S, const PotParams<R>& P, const int* one, cudaStream_t st, float* ms_out) {
  if (S.N == 0) return cudaSuccess;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  int pick = S.build_shape;
  float best = 0.f;
  for (int k = 0; k < BUILD_SHAPES && e == cudaSuccess; ++k) {
    launch_build<R>(S, P, k, one, st);
    cudaEventRecord(e0, st);
    launch_build<R>(S, P, k, one, st);
    launch_build<R>(S, P, k, one, st);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms *= 0.5f;
    if (ms_out) ms_out[k] = ms;
    if (e == cudaSuccess && (best == 0.f || ms < best)) { best = ms; pick = k; }
  }
  S.build_shape = pick;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}
template cudaError_t tune_build<float>(DevState&, const PotParams<float>&, const int*, cudaStream_t, float*);
template cudaError_t tune_build<double>(DevState&, const PotParams<double>&, const int*, cudaStream_t, float*);

template <class R>
void launch_rebuild(const DevState& S, const PotParams<R>& P, cudaStream_t st) {
  int N = S.N;
  if (N == 0) return;
  int tb = 256;
  int C = S.ncells;
  const int* f = S.flag_rebuild;
  k_zero_cells<<<(max(C, 3) + tb - 1) / tb, tb, 0, st>>>(C, S.cell_count, S.cell_fill, S.maxcnt, f);
  k_bin<R><<<(N + tb - 1) / tb, tb, 0, st>>>(N, S.x, S.xref, S.type, S.rep, S.reps, S.cell4,
                                              (typename Vec4<R>::T*)S.u, S.cell_count, S.err, f);
  int nb = (C + SCAN_T * SCAN_E - 1) / (SCAN_T * SCAN_E);
  k_scan_block<<<nb, SCAN_T, 0, st>>>(C, S.cell_count, S.cell_start, S.scan_tmp, f);
  k_scan_top<<<1, SCAN_T, 0, st>>>(nb, S.scan_tmp, S.scan_tmp + 1024, f);
  k_scan_add<<<(C + tb - 1) / tb, tb, 0, st>>>(C, S.cell_start, S.scan_tmp, f);
  k_scatter<<<(N + tb - 1) / tb, tb, 0, st>>>(N, S.cell4, S.cell_start, S.cell_fill, S.cell_atoms, f);
  k_sort_cells<<<(C + tb - 1) / tb, tb, 0, st>>>(C, S.cell_start, S.cell_count, S.cell_atoms, f);
  // grid-strided: when no rebuild is due these launches return at once
  launch_build<R>(S, P, S.build_shape, f, st);
  k_list_transpose<<<S.nsm * 8, 256, 0, st>>>(N, S.cap_cov, S.cap_all, S.ld, S.lst, S.ncov, S.nfix, S.nall,
                                              S.nl, f);
  k_rev<<<S.nsm * 4, tb, 0, st>>>(N, S.cap_cov, S.ld, S.nl, S.ncov, S.rev, S.err, f);
  k_finish_rebuild<<<1, 1, 0, st>>>(S.flag_rebuild, S.rebuild_count);
}

template void launch_rebuild<float>(const DevState&, const PotParams<float>&, cudaStream_t);
template void launch_rebuild<double>(const DevState&, const PotParams<double>&, cudaStream_t);

}  // namespace ct
