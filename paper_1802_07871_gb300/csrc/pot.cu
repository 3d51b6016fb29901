// pot.cu — bond pass, charge-system assembly and forces.
//
// bond pass (k_bond): G lanes per atom i (4, 8 or 16, tuned); i's covalent
//   entries are staged in shared memory and its live bonds (f_c > 0)
//   compacted; each lane owns live bonds e and sums over the live third atoms k
//   the environment terms zeta_l,ie = sum_k fc(r_ik) ang_l(cos) e^{alpha_l (r_ie - r_ik)}
//   (Sec. 2, Eq. 2), then b_ie and db/dzeta_l from the L = 2 form (Eq. 7).
// assembly (k_assemble): one thread per atom over its column of the list;
//   the off-diagonal charge Hessian entries M_e = K(r_e) - 2 w_e
//   (w_e = 1/2 kappa fc B e^{-lambda2 r} (b_ij + b_ji) on covalent entries),
//   diagonal 2 J + 2 sum w and the Jacobi inverse.
// covalent forces (k_cov_force): G lanes per atom over its live bonds; for
//   every entry e the gradient dE_i/du_e of all terms centred on i (pair
//   part, and the environment-sum chain rule both with e as bond and e as
//   third atom); written to a per-bond slot (zero for bonds past S), no
//   atomics.
// charge forces + gather (k_coul_gather): one thread per atom over all entries;
//   F_i = sum_j q_i q_j K'(r) u_ij/r + sum_e slot(i,e) - sum_e slot(j_e, rev_e);
//   per-atom energy, the virial (evaluations; MD steps leave it out),
//   optional velocity-Verlet half kick; FP64 per-replica sums.
#include "internal.cuh"
#include "kernels.h"

namespace ct {

// Covalent kernels: blocks of CB threads, G lanes per atom (G = 4, 8 or 16,
// tuned on the live lists by tune_cov), CB / G atoms per block.
#define CB 128
#define GATHER_MINB 3
// Bonds whose repulsive radial derivative lambda1 * A e^(-lambda1 r) exceeds
// this (eV/A) get their pair term in FP64 on the FP32 path (queued by the
// bond pass, evaluated by k_stiff): there the repulsive and attractive
// derivatives cancel to a few eV/A and the FP32 rounding of both terms and
// of the bond length would stand out. Equilibrium Si-C bonds of the
// synthetic set sit at 17.7 eV/A (about twice below the threshold);
// compressed adatom bonds reach 40-80 eV/A.
#define STIFF_PAIR 35.0f

template <class R>
__device__ inline void bond_order7(R z1, R z2, int pb, const PotParams<R>& P, R& b, R& db1, R& db2) {
  R n1 = P.n1[pb], n2 = P.n2[pb], p = P.p[pb];
  R zn1 = z1 > R(0) ? ct_pow<R>(z1, n1) : R(0);
  R zn2 = z2 > R(0) ? ct_pow<R>(z2, n2) : R(0);
  R Z1 = P.g1[pb] + zn1, Z2 = P.g2[pb] + zn2;
  R t1 = ct_pow<R>(Z1, -p), t2 = ct_pow<R>(Z2, -p);
  R Ssum = t1 + t2;
  b = P.G[pb] * ct_pow<R>(Ssum, P.inv2sp[pb]);
  R pre = -b * P.inv2s[pb] / Ssum;
  db1 = z1 > R(0) ? pre * (t1 / Z1) * n1 * (zn1 / z1) : R(0);
  db2 = z2 > R(0) ? pre * (t2 / Z2) * n2 * (zn2 / z2) : R(0);
}

// The cell offsets of a packed code as exact FP32 values: a 10-bit field m
// placed in the mantissa of 2^23 reads as 2^23 + m, so one subtraction
// gives m - 512 (the same values an integer conversion gives, without one).
__device__ inline void unpack_code_f(int c, float& dx, float& dy, float& dz) {
  const float base = 8388608.0f + 512.0f;
  dx = __int_as_float(0x4B000000 | (c & 1023)) - base;
  dy = __int_as_float(0x4B000000 | ((c >> 10) & 1023)) - base;
  dz = __int_as_float(0x4B000000 | ((c >> 20) & 1023)) - base;
}

template <class R>
__device__ inline void rel_vec(const typename Vec4<R>::T& ui, const typename Vec4<R>::T& uj, int cd,
                               R hx, R hy, R hz, R& rx, R& ry, R& rz) {
  if (sizeof(R) == 4) {
    float dx, dy, dz;
    unpack_code_f(cd, dx, dy, dz);
    rx = (uj.x - ui.x) + (R)dx * hx;
    ry = (uj.y - ui.y) + (R)dy * hy;
    rz = (uj.z - ui.z) + (R)dz * hz;
    return;
  }
  int dx, dy, dz;
  unpack_code(cd, dx, dy, dz);
  rx = (uj.x - ui.x) + (R)dx * hx;
  ry = (uj.y - ui.y) + (R)dy * hy;
  rz = (uj.z - ui.z) + (R)dz * hz;
}

// Squared taper limits of the four pair types in FP64, for the FP32 path's
// cutoff of bonds inside the taper (see cutoff_fp64).
struct Taper64 {
  double R2[4], S2[4];
};

// Cutoff and its derivative of bond (i, j, cell code cd) of the FP32 path,
// placed in the taper from the FP64 master positions. The tapers are a few
// tenths of an angstrom wide, so the cutoff's curvature (up to
// pi^2 / (2 (S - R)^2) per A^2) turns the FP32 rounding of a cell-local
// position (about 2e-7 A) into force errors of 1e-4 to 3e-4 eV/A on atoms
// with a bond in the taper. Here r^2 - R^2 and S^2 - r^2 are formed in
// FP64 from the bond vector x_j - x_i + shift (no FP64 root or division),
// and the nearer end's distance follows in FP32 as (r^2 - R^2) / (r + R)
// or (S^2 - r^2) / (S + r): accurate to FP32 rounding of that small
// distance, so the cutoff is placed to about 3e-8 A. r32 is the FP32 bond
// length (it only scales the quotient).
__device__ inline void cutoff_fp64(int i, int j, int cd, int pb, const double* __restrict__ x,
                                   const int4* __restrict__ cell4, const RepInfo& ri, const Taper64& TP,
                                   float r32, float Rf, float Sf, float pi_SR, float& fc, float& dfc) {
  const int4 ci = cell4[i], cj = cell4[j];
  int dx, dy, dz;
  unpack_code(cd, dx, dy, dz);
  // u_j - u_i + d hc with u = x - c hc
  const double rx = (x[3 * j] - x[3 * i]) + (double)(dx + ci.x - cj.x) * ri.hc[0];
  const double ry = (x[3 * j + 1] - x[3 * i + 1]) + (double)(dy + ci.y - cj.y) * ri.hc[1];
  const double rz = (x[3 * j + 2] - x[3 * i + 2]) + (double)(dz + ci.z - cj.z) * ri.hc[2];
  const double r2 = rx * rx + ry * ry + rz * rz;
  // (selects, not an indexed load: an indexed parameter array is copied to
  // local memory)
  const double R2 = pb == 0 ? TP.R2[0] : pb == 1 ? TP.R2[1] : pb == 2 ? TP.R2[2] : TP.R2[3];
  const double S2 = pb == 0 ? TP.S2[0] : pb == 1 ? TP.S2[1] : pb == 2 ? TP.S2[2] : TP.S2[3];
  const double aR = r2 - R2, aS = S2 - r2;
  if (aR <= 0.0) { fc = 1.f; dfc = 0.f; return; }
  if (aS <= 0.0) { fc = 0.f; dfc = 0.f; return; }
  const float w = Sf - Rf;
  if (aR < aS) {   // t = (r - R) / (S - R) <= 1/2: fc = cos^2(pi t / 2)
    const float h = 0.5f * (float)aR / ((r32 + Rf) * w);
    const float c = ct_cospi<float>(h), sn = ct_sinpi<float>(h);
    fc = c * c;
    dfc = -pi_SR * sn * c;
  } else {         // u = 1 - t: fc = sin^2(pi u / 2), sin(pi t/2) cos(pi t/2) = cos(pi u/2) sin(pi u/2)
    const float h = 0.5f * (float)aS / ((Sf + r32) * w);
    const float c = ct_cospi<float>(h), sn = ct_sinpi<float>(h);
    fc = sn * sn;
    dfc = -pi_SR * c * sn;
  }
}

// FP32 path: bonds whose FP32 length lies within this of a taper end take
// the FP64 cutoff (the FP32 length is off by far less).
#define TAPER_MARGIN 1e-4f

// ---------------------------------------------------------------- bond pass
//
// Precision by need (FP32 path). Every bond in a cutoff's taper takes its
// cutoff from the FP64 positions (cutoff_fp64): without that, hot MD (RMS
// force near 1.7 eV/A) put its worst atoms at 2e-4 of the RMS force. A
// replica is in the accurate mode when the RMS force of its previous
// evaluation is below ACC_RMS (and on its first evaluation after positions
// or parameters were set, when there is none). Then every bond's pair term
// is queued for k_stiff (FP64), and every atom with a bond in the taper
// (R < r < S) or a compressed bond (the STIFF_PAIR criterion) is queued as
// a whole: k_bond<double> and k_cov_force<double, float> recompute its
// bond orders and force slots in FP64 from the master positions and
// overwrite the FP32 results: the FP32 rounding of such an atom's bonds
// (3e-7 A) moves its force by more than a 1e-4 bar relative to a small RMS
// force allows.
// qlist/qn: when given, block b takes the queued atoms qlist[b*CB/G ..], the
// rest of the grid exits at once.
//
// Live bonds. Of an atom's covalent entries (r < S + skin) only those with
// f_c > 0 take part in bond orders and three-body terms; the rest (the skin,
// about a fifth of the entries in hot MD) get their trivial outputs at once
// and the bond and three-body loops run over the compacted live list, in
// list order (the sums add in the same order as over the full list;
// compact_live in internal.cuh).
template <class R, int G>
__global__ void __launch_bounds__(CB)
k_bond(int N, int cap_cov, int ld, const typename Vec4<R>::T* __restrict__ u,
       const int* __restrict__ rep, const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
        const int* __restrict__ ncov, PotParams<R> P,
       typename Vec4<R>::T* __restrict__ bo, int* __restrict__ stiff_n, int* __restrict__ stiff_q,
       const int* __restrict__ acc_mode, int* __restrict__ flag_n, int* __restrict__ flag_q,
       const int* __restrict__ qlist, const int* __restrict__ qn,
       const double* __restrict__ x64, const int4* __restrict__ cell4, Taper64 TP) {
  using R4 = typename Vec4<R>::T;
  constexpr int APB_ = CB / G;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int s_nstiff, s_base, s_nflag, s_fbase;
  if (threadIdx.x == 0) { s_nstiff = 0; s_nflag = 0; }
  int g = threadIdx.x / G, l = threadIdx.x % G;
  // layout: R4 (ux,uy,uz,r)[APB_][cap] | R fc | int type | int live list
  R4* s_u = reinterpret_cast<R4*>(smem_raw);
  R* s_fc = reinterpret_cast<R*>(s_u + (size_t)APB_ * cap_cov);
  int* s_t = reinterpret_cast<int*>(s_fc + (size_t)APB_ * cap_cov);
  int* s_lv = s_t + (size_t)APB_ * cap_cov;
  s_u += (size_t)g * cap_cov; s_fc += (size_t)g * cap_cov; s_t += (size_t)g * cap_cov; s_lv += (size_t)g * cap_cov;
  int i = blockIdx.x * APB_ + g;
  if (qlist) {
    const int nq = *qn;
    if (blockIdx.x * APB_ >= nq) return;   // (uniform over the block)
    i = i < nq ? qlist[i] : N;
  }
  bool live = i < N;
  bool acc = false;   // this replica in the accurate mode (FP32 path)
  int nc = 0, ti = 0;
  R4 ui;
  if (live) {
    ui = u[i];
    ti = (int)ui.w;
    nc = min(ncov[i], cap_cov);
    const int rid = rep[i];
    const RepInfo& ri = reps[rid];
    if (sizeof(R) == 4 && acc_mode) acc = acc_mode[rid] != 0;
    R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
    if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
    for (int e = l; e < nc; e += G) {
      const int2 jcd = nl[(size_t)e * ld + i];
      const int j = jcd.x;
      R4 uj = u[j];
      R rx, ry, rz;
      rel_vec<R>(ui, uj, jcd.y, hx, hy, hz, rx, ry, rz);
      R r = ct_sqrt<R>(rx * rx + ry * ry + rz * rz);
      int tj = (int)uj.w;
      int pb = ti * 2 + tj;
      R fc, dfc;
      cutoff_fn<R>(r, P.Rin[pb], P.Sout[pb], P.pi_SR[pb], fc, dfc);
      if (sizeof(R) == 4 && x64 && r > P.Rin[pb] - R(TAPER_MARGIN) && r < P.Sout[pb] + R(TAPER_MARGIN)) {
        float f, df;
        cutoff_fp64(i, j, jcd.y, pb, x64, cell4, ri, TP, (float)r, (float)P.Rin[pb], (float)P.Sout[pb],
                    (float)P.pi_SR[pb], f, df);
        fc = (R)f;
      }
      R4 w;
      w.x = rx; w.y = ry; w.z = rz; w.w = r;
      s_u[e] = w;
      s_fc[e] = fc;
      s_t[e] = tj;
    }
  }
  __syncthreads();
  int my_stiff = 0, my_flag = 0;
  const int nlive = compact_live<G>(live, nc, l, s_lv, [&](int e) { return s_fc[e] > R(0); }, [&](int e) {
    R4 out;
    out.x = R(1); out.y = R(0); out.z = R(0); out.w = R(0);
    bo[(size_t)i * cap_cov + e] = out;
  });
  __syncwarp();
  for (int q = l; q < nlive; q += G) {
    const int e = s_lv[q];
    R4 ue = s_u[e];
    int tj = s_t[e];
    int pb = ti * 2 + tj;
    R4 out;
    // .w marks a stiff bond (FP32 path): its pair term is evaluated in FP64
    // by k_stiff, from the queue built below (every bond in the accurate mode)
    out.w = R(0);
    if (sizeof(R) == 4) {
      bool compressed = P.lam1[pb] * P.A[pb] * ct_exp<R>(-P.lam1[pb] * ue.w) > R(STIFF_PAIR);
      if (compressed || acc) {
        out.w = R(1);
        ++my_stiff;
      }
      if (acc && (compressed || ue.w > P.Rin[pb])) my_flag = 1;
    }
    R re = ue.w, ire = R(1) / re;
    R z1 = R(0), z2 = R(0);
    int tbase = pb * 2;
    for (int kk = 0; kk < nlive; ++kk) {
      const int k = s_lv[kk];
      if (k == e) continue;
      R fck = s_fc[k];
      R4 uk = s_u[k];
      int tri = tbase + s_t[k];
      R ct = (ue.x * uk.x + ue.y * uk.y + ue.z * uk.z) * ire / uk.w;
      R dr = re - uk.w;
      {
        R hm = P.h[tri][0] - ct;
        R hm2 = hm * hm;
        R ang = P.gam[tri][0] * (R(1) + P.c2d2[tri][0] * hm2 / (P.d2[tri][0] + hm2));
        z1 += fck * ang * ct_exp<R>(P.alpha[tri][0] * dr);
      }
      {
        R hm = P.h[tri][1] - ct;
        R hm2 = hm * hm;
        R ang = P.gam[tri][1] * (R(1) + P.c2d2[tri][1] * hm2 / (P.d2[tri][1] + hm2));
        z2 += fck * ang * ct_exp<R>(P.alpha[tri][1] * dr);
      }
    }
    R b, db1, db2;
    bond_order7<R>(z1, z2, pb, P, b, db1, db2);
    out.x = b; out.y = db1; out.z = db2;
    bo[(size_t)i * cap_cov + e] = out;
  }
  if (sizeof(R) != 4 || qlist) return;   // (uniform over the block)
  // this atom is queued for the FP64 pass when any lane of its group
  // flagged it (every lane of the warp takes part in the shuffles)
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) my_flag |= __shfl_xor_sync(CT_FULL, my_flag, o, G);
  // append this block's stiff bonds and flagged atoms to their queues: one
  // global atomic per block and queue
  int off = my_stiff ? atomicAdd(&s_nstiff, my_stiff) : 0;
  int foff = (my_flag && l == 0) ? atomicAdd(&s_nflag, 1) : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_base = s_nstiff ? atomicAdd(stiff_n, s_nstiff) : 0;
    s_fbase = s_nflag ? atomicAdd(flag_n, s_nflag) : 0;
  }
  __syncthreads();
  if (my_stiff) {   // (the live bonds this lane computed, as above)
    int pos = s_base + off;
    for (int q = l; q < nlive; q += G) {
      const int e = s_lv[q];
      if (bo[(size_t)i * cap_cov + e].w != R(0)) stiff_q[pos++] = i * cap_cov + e;
    }
  }
  if (my_flag && l == 0) flag_q[s_fbase + foff] = i;
}

// The pair term of every queued stiff bond in FP64 (fully occupied lanes,
// unlike a per-bond branch inside the force pass): the bond vector from the
// master positions (r_ij = x_j - x_i + the periodic shift of the stencil
// cell), c_ij from the FP64 charges, b_ij from the bond pass. Stores dE/dr
// and the energy 1/2 fc (A e^{-l1 r} - c b B e^{-l2 r}) as double2 (the
// energy stays FP64: the bonds of a crystal round alike, so FP32 energies
// would add up coherently).
__global__ void __launch_bounds__(256)
    k_stiff(int cap_cov, int ld, const int* __restrict__ nq, const int* __restrict__ q_ids,
            const int2* __restrict__ nl,  const int* __restrict__ rep,
            const RepInfo* __restrict__ reps, const double* __restrict__ x, const int4* __restrict__ cell4,
            const int* __restrict__ type, const float4* __restrict__ bo, const double* __restrict__ q,
            PotParams<float> P, double2* __restrict__ pe) {
  int n = *nq;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int id = q_ids[t];
    int i = id / cap_cov, e = id - i * cap_cov;
    size_t idx = (size_t)e * ld + i;
    int j = nl[idx].x;
    int dcx, dcy, dcz;
    unpack_code(nl[idx].y, dcx, dcy, dcz);
    const RepInfo& ri = reps[rep[i]];
    int4 ci4 = cell4[i], cj4 = cell4[j];
    double ax = x[3 * j] - x[3 * i] + (double)(ci4.x + dcx - cj4.x) * ri.hc[0];
    double ay = x[3 * j + 1] - x[3 * i + 1] + (double)(ci4.y + dcy - cj4.y) * ri.hc[1];
    double az = x[3 * j + 2] - x[3 * i + 2] + (double)(ci4.z + dcz - cj4.z) * ri.hc[2];
    double r = sqrt(ax * ax + ay * ay + az * az);
    int pb = type[i] * 2 + type[j];
    double fc = 1.0, dfc = 0.0;
    if (r >= P.Sout64[pb]) {
      fc = 0.0;
    } else if (r >= P.Rin64[pb]) {
      double w = P.Sout64[pb] - P.Rin64[pb], tt = (r - P.Rin64[pb]) / w;
      fc = 0.5 * (1.0 + cospi(tt));
      dfc = -0.5 * (M_PI / w) * sinpi(tt);
    }
    double dq = q[i] - q[j];
    double cq = 1.0 - P.kappa64[pb] * dq * dq;
    double fR = P.A64[pb] * exp(-P.lam1_64[pb] * r);
    double att = cq * (double)bo[id].x * P.B64[pb] * exp(-P.lam2_64[pb] * r);
    double pd = 0.5 * (dfc * (fR - att) + fc * (-P.lam1_64[pb] * fR + P.lam2_64[pb] * att));
    pe[id] = make_double2(pd, 0.5 * fc * (fR - att));
  }
}

// ---------------------------------------------------------------- assembly
// Entries past the covalent part are streamed: the list indices and offset
// codes of the next batch of entries are loaded before the current ones are
// used, so the list (the bound of these passes) always has loads in flight.
// The batch is AB in the assembly (4, 8 or 16, timed on the first solve of
// new lists, tune_assemble) and PB in the charge-force gather (4, 6 or 8,
// tune_gather).
//
// Matrix layout: entry e of atom i at row e (e * ld + i) for the covalent
// and core entries, so the assembly walks those rows warp-uniformly and
// every store of a warp fills one contiguous 256-byte row; the shell entries
// inside the charge cutoff are packed after the core (FP32 path: those
// beyond it have K = 0 and are dropped, about 15% of the list), the only
// stores whose rows differ between lanes. The FP64 path keeps every entry at
// its list row.
template <class R, int AB>
__global__ void __launch_bounds__(256)
    k_assemble(int N, int cap_cov, int ld, const typename Vec4<R>::T* __restrict__ u,
               const int* __restrict__ rep, const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
               const int* __restrict__ ncov, const int* __restrict__ nfix, const int* __restrict__ nall,
               const int* __restrict__ rev, const typename Vec4<R>::T* __restrict__ bo, PotParams<R> P,
               TypeParams T, void* __restrict__ M, R* __restrict__ Dg, R* __restrict__ dinv,
               int* __restrict__ nmat) {
  using R4 = typename Vec4<R>::T;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned wm = __ballot_sync(CT_FULL, i < N);   // the warp's live lanes
  if (i >= N) return;
  R4 ui = u[i];
  int ti = (int)ui.w;
  const RepInfo& ri = reps[rep[i]];
  R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
  if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
  int nc = ncov[i], nf = nfix[i], na = nall[i];
  R wsum = R(0), selfm = R(0);
  const int2* pl = nl + i;
  // covalent entries: K minus twice the bond-order coupling w
  for (int e = 0; e < nc; ++e) {
    size_t off = (size_t)e * ld;
    int2 jcd = __ldg(pl + off);
    int j = jcd.x;
    R4 uj = u[j];
    R rx, ry, rz;
    rel_vec<R>(ui, uj, jcd.y, hx, hy, hz, rx, ry, rz);
    R r2 = rx * rx + ry * ry + rz * rz;
    int tj = (int)uj.w;
    int pb = ti * 2 + tj;
    R m = coul_K_r2<R>(r2, P.gshield3[pb], P.inv_rcoul, P.ke);
    R r = ct_sqrt<R>(r2);
    if (r < P.Sout[pb]) {
      R fc, dfc;
      cutoff_fn<R>(r, P.Rin[pb], P.Sout[pb], P.pi_SR[pb], fc, dfc);
      R fA = P.B[pb] * ct_exp<R>(-P.lam2[pb] * r);
      R bij = bo[(size_t)i * cap_cov + e].x;
      R bji = bo[(size_t)j * cap_cov + rev[(size_t)i * cap_cov + e]].x;
      R w = R(0.5) * P.kappa[pb] * fc * fA * (bij + bji);
      m -= R(2) * w;
      wsum += w;
    }
    if (j == i) selfm += m;
    mat_store(M, off + i, j, m);
  }
  const R gs_i0 = P.gshield3[ti * 2], gs_i1 = P.gshield3[ti * 2 + 1];
  // core entries: rows [nc, nf) walked in step by the whole warp (lanes
  // outside their own range idle), each stored at its own row
  {
    const int e_lo = (int)__reduce_min_sync(wm, (unsigned)nc);
    const int e_hi = (int)__reduce_max_sync(wm, (unsigned)nf);
    int jn[AB], cn[AB];
#pragma unroll
    for (int k = 0; k < AB; ++k) {
      int en = e_lo + k;
      bool ok = en >= nc && en < nf;
      int2 t = ok ? __ldg(pl + (size_t)en * ld) : make_int2(i, pack_code(0, 0, 0));
      jn[k] = t.x;
      cn[k] = t.y;
    }
    for (int e = e_lo; e < e_hi; e += AB) {
      int jc[AB], cc[AB];
#pragma unroll
      for (int k = 0; k < AB; ++k) {
        jc[k] = jn[k];
        cc[k] = cn[k];
        int en = e + AB + k;
        bool ok = en >= nc && en < nf;
        int2 t = ok ? __ldg(pl + (size_t)en * ld) : make_int2(i, pack_code(0, 0, 0));
        jn[k] = t.x;
        cn[k] = t.y;
      }
      R4 uj[AB];
#pragma unroll
      for (int k = 0; k < AB; ++k) uj[k] = u[jc[k]];
#pragma unroll
      for (int k = 0; k < AB; ++k) {
        int row = e + k;
        if (row >= nc && row < nf) {
          R rx, ry, rz;
          rel_vec<R>(ui, uj[k], cc[k], hx, hy, hz, rx, ry, rz);
          R r2 = rx * rx + ry * ry + rz * rz;
          R m = coul_K_r2<R>(r2, uj[k].w != R(0) ? gs_i1 : gs_i0, P.inv_rcoul, P.ke);
          if (jc[k] == i) selfm += m;
          mat_store(M, (size_t)row * ld + i, jc[k], m);
        }
      }
    }
  }
  // shell entries: K only, streamed; the FP32 path stores only those inside
  // the charge cutoff, packed after the core
  int em = nf;
  int jn[AB], cn[AB];
#pragma unroll
  for (int k = 0; k < AB; ++k) {
    bool ok = nf + k < na;
    int2 t = ok ? __ldg(pl + (size_t)(nf + k) * ld) : make_int2(i, pack_code(0, 0, 0));
    jn[k] = t.x;
    cn[k] = t.y;
  }
  for (int e = nf; e < na; e += AB) {
    int jc[AB], cc[AB];
#pragma unroll
    for (int k = 0; k < AB; ++k) {
      jc[k] = jn[k];
      cc[k] = cn[k];
      int en = e + AB + k;
      bool ok = en < na;
      int2 t = ok ? __ldg(pl + (size_t)en * ld) : make_int2(i, pack_code(0, 0, 0));
      jn[k] = t.x;
      cn[k] = t.y;
    }
    R4 uj[AB];
#pragma unroll
    for (int k = 0; k < AB; ++k) uj[k] = u[jc[k]];
#pragma unroll
    for (int k = 0; k < AB; ++k) {
      if (e + k < na) {
        R rx, ry, rz;
        rel_vec<R>(ui, uj[k], cc[k], hx, hy, hz, rx, ry, rz);
        R r2 = rx * rx + ry * ry + rz * rz;
        R m = coul_K_r2<R>(r2, uj[k].w != R(0) ? gs_i1 : gs_i0, P.inv_rcoul, P.ke);
        if (jc[k] == i) selfm += m;
        if (sizeof(R) == 8) {
          mat_store(M, (size_t)(e + k) * ld + i, jc[k], m);
        } else if (m != R(0)) {
          mat_store(M, (size_t)em * ld + i, jc[k], m);
          ++em;
        }
      }
    }
  }
  if (sizeof(R) == 4) nmat[i] = em;
  R D = (R)(2.0 * by_type(T.J, ti)) + R(2) * wsum;
  Dg[i] = D;
  dinv[i] = R(1) / (D + selfm);
}

// ---------------------------------------------------------------- covalent forces
// O is the type of the stored slots: R, or float for the FP64 pass over the
// queued atoms of the FP32 path (qlist/qn as in k_bond).
template <class R, class O, int G>
__global__ void __launch_bounds__(CB)
k_cov_force(int N, int cap_cov, int ld, const typename Vec4<R>::T* __restrict__ u,
            const int* __restrict__ rep, const RepInfo* __restrict__ reps,
            const int2* __restrict__ nl,  const int* __restrict__ ncov,
            const typename Vec4<R>::T* __restrict__ bo, const double* __restrict__ q,
            const R* __restrict__ qr, PotParams<R> P, TypeParams T, typename Vec4<O>::T* __restrict__ gslot,
            double* __restrict__ e_atom, const void* __restrict__ stiff_pe,
            const int* __restrict__ qlist, const int* __restrict__ qn,
            const double* __restrict__ x64, const int4* __restrict__ cell4, Taper64 TP) {
  using R4 = typename Vec4<R>::T;
  using R2 = typename Vec2<R>::T;
  constexpr int APB_ = CB / G;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  int g = threadIdx.x / G, l = threadIdx.x % G;
  // layout: R4 u[APB_][cap] | R2 D[APB_][cap] | R fc | R dfc | R pair dE/dr | int type | int live list
  R4* s_u = reinterpret_cast<R4*>(smem_raw);
  R2* s_D = reinterpret_cast<R2*>(s_u + (size_t)APB_ * cap_cov);
  R* s_fc = reinterpret_cast<R*>(s_D + (size_t)APB_ * cap_cov);
  R* s_dfc = s_fc + (size_t)APB_ * cap_cov;
  R* s_pd = s_dfc + (size_t)APB_ * cap_cov;
  int* s_t = reinterpret_cast<int*>(s_pd + (size_t)APB_ * cap_cov);
  int* s_lv = s_t + (size_t)APB_ * cap_cov;
  s_u += (size_t)g * cap_cov; s_D += (size_t)g * cap_cov; s_fc += (size_t)g * cap_cov;
  s_dfc += (size_t)g * cap_cov; s_pd += (size_t)g * cap_cov; s_t += (size_t)g * cap_cov;
  s_lv += (size_t)g * cap_cov;

  int i = blockIdx.x * APB_ + g;
  if (qlist) {
    const int nq = *qn;
    if (blockIdx.x * APB_ >= nq) return;   // (uniform over the block)
    i = i < nq ? qlist[i] : N;
  }
  bool live = i < N;
  int nc = 0, ti = 0;
  CompSum<R> eacc;
  double estiff = 0.0;   // FP64 pair energies of the stiff bonds (FP32 path)
  int nstiff = 0;        // how many (the FP64 sum is skipped where a warp has none)
  if (live) {
    R4 ui = u[i];
    ti = (int)ui.w;
    nc = min(ncov[i], cap_cov);
    const RepInfo& ri = reps[rep[i]];
    R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
    if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
    R qi = qr[i];
    for (int e = l; e < nc; e += G) {
      size_t idx = (size_t)e * ld + i;
      int j = nl[idx].x;
      R4 uj = u[j];
      R rx, ry, rz;
      rel_vec<R>(ui, uj, nl[idx].y, hx, hy, hz, rx, ry, rz);
      R r = ct_sqrt<R>(rx * rx + ry * ry + rz * rz);
      int tj = (int)uj.w;
      int pb = ti * 2 + tj;
      R fc, dfc;
      cutoff_fn<R>(r, P.Rin[pb], P.Sout[pb], P.pi_SR[pb], fc, dfc);
      if (sizeof(R) == 4 && x64 && r > P.Rin[pb] - R(TAPER_MARGIN) && r < P.Sout[pb] + R(TAPER_MARGIN)) {
        float f, df;
        cutoff_fp64(i, j, nl[idx].y, pb, x64, cell4, ri, TP, (float)r, (float)P.Rin[pb], (float)P.Sout[pb],
                    (float)P.pi_SR[pb], f, df);
        fc = (R)f;
        dfc = (R)df;
      }
      R2 D;
      D.x = R(0); D.y = R(0);
      R pd = R(0);
      if (fc > R(0)) {
        R4 bb = bo[(size_t)i * cap_cov + e];
        R dq = qi - qr[j];
        R cq = R(1) - P.kappa[pb] * dq * dq;
        R fR = P.A[pb] * ct_exp<R>(-P.lam1[pb] * r);
        R fA = P.B[pb] * ct_exp<R>(-P.lam2[pb] * r);
        R att = cq * bb.x * fA;
        if (sizeof(R) == 4 && bb.w != R(0)) {
          // stiff bond: pair term evaluated in FP64 by k_stiff
          double2 v = static_cast<const double2*>(stiff_pe)[(size_t)i * cap_cov + e];
          estiff += v.y;
          ++nstiff;
          pd = (R)v.x;
        } else {
          eacc.add(R(0.5) * fc * (fR - att));
          pd = R(0.5) * (dfc * (fR - att) + fc * (-P.lam1[pb] * fR + P.lam2[pb] * att));
        }
        R pre = R(-0.5) * cq * fc * fA;
        D.x = pre * bb.y;
        D.y = pre * bb.z;
      }
      R4 w;
      w.x = rx; w.y = ry; w.z = rz; w.w = r;
      s_u[e] = w;
      s_D[e] = D;
      s_fc[e] = fc;
      s_dfc[e] = dfc;
      s_pd[e] = pd;
      s_t[e] = tj;
    }
  }
  __syncwarp();
  const int nlive = compact_live<G>(live, nc, l, s_lv, [&](int e) { return s_fc[e] > R(0); }, [&](int e) {
    typename Vec4<O>::T z;
    z.x = O(0); z.y = O(0); z.z = O(0); z.w = O(0);
    gslot[(size_t)i * cap_cov + e] = z;
  });
  __syncwarp();
  {
    for (int q = l; q < nlive; q += G) {
      const int e = s_lv[q];
      R4 ux = s_u[e];
      R rx = ux.w;
      R fcx = s_fc[e];
      typename Vec4<O>::T out;
      out.x = O(0); out.y = O(0); out.z = O(0); out.w = O(0);
      {
        R irx = R(1) / rx;
        R hx_ = ux.x * irx, hy_ = ux.y * irx, hz_ = ux.z * irx;
        R2 Dx = s_D[e];
        R dfcx = s_dfc[e];
        int tx = s_t[e];
        R c_ux = s_pd[e];
        R gx = R(0), gy = R(0), gz = R(0);
        for (int kk = 0; kk < nlive; ++kk) {
          const int k = s_lv[kk];
          if (k == e) continue;
          R fck = s_fc[k];
          R4 uk = s_u[k];
          R rk = uk.w, irk = R(1) / rk;
          R kx = uk.x * irk, ky = uk.y * irk, kz = uk.z * irk;
          R ct = hx_ * kx + hy_ * ky + hz_ * kz;
          int tk = s_t[k];
          R2 Dk = s_D[k];
          R c_perp = R(0);
          // e as the bond, k as the third atom: triplet (ti, tx, tk)
          {
            int tri = (ti * 2 + tx) * 2 + tk;
            R dr = rx - rk;
#pragma unroll
            for (int ll = 0; ll < 2; ++ll) {
              R Dl = ll == 0 ? Dx.x : Dx.y;
              R hm = P.h[tri][ll] - ct;
              R den = P.d2[tri][ll] + hm * hm;
              R ang = P.gam[tri][ll] * (R(1) + P.c2d2[tri][ll] * (hm * hm) / den);
              R dang = R(-2) * P.gam[tri][ll] * P.c2[tri][ll] * hm / (den * den);
              R ex = ct_exp<R>(P.alpha[tri][ll] * dr);
              c_ux += Dl * P.alpha[tri][ll] * fck * ang * ex;
              c_perp += Dl * fck * dang * ex;
            }
          }
          // k as the bond, e as the third atom: triplet (ti, tk, tx)
          {
            int tri = (ti * 2 + tk) * 2 + tx;
            R dr = rk - rx;
#pragma unroll
            for (int ll = 0; ll < 2; ++ll) {
              R Dl = ll == 0 ? Dk.x : Dk.y;
              R hm = P.h[tri][ll] - ct;
              R den = P.d2[tri][ll] + hm * hm;
              R ang = P.gam[tri][ll] * (R(1) + P.c2d2[tri][ll] * (hm * hm) / den);
              R dang = R(-2) * P.gam[tri][ll] * P.c2[tri][ll] * hm / (den * den);
              R ex = ct_exp<R>(P.alpha[tri][ll] * dr);
              c_ux += Dl * (dfcx * ang * ex - P.alpha[tri][ll] * fcx * ang * ex);
              c_perp += Dl * fcx * dang * ex;
            }
          }
          // c_perp multiplies d cos / d u_e = (u_k/r_k - cos u_e/r_e) / r_e
          R cp = c_perp * irx;
          gx += cp * (kx - ct * hx_);
          gy += cp * (ky - ct * hy_);
          gz += cp * (kz - ct * hz_);
        }
        out.x = (O)(gx + c_ux * hx_);
        out.y = (O)(gy + c_ux * hy_);
        out.z = (O)(gz + c_ux * hz_);
      }
      gslot[(size_t)i * cap_cov + e] = out;
    }
  }
  // per-atom energy: covalent part + self energy (all lanes take part). An
  // FP64 warp instruction costs the FP64 pipe as much as dozens of FP32
  // ones, so the FP64 work here is kept to the few operations the
  // precision needs: the stiff-bond sum only where the warp has one, the
  // self energy as two fused multiply-adds.
  R es = eacc.s, ec = eacc.c;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    es += __shfl_xor_sync(CT_FULL, es, o, G);
    ec += __shfl_xor_sync(CT_FULL, ec, o, G);
  }
  if (__any_sync(CT_FULL, nstiff != 0)) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) estiff += __shfl_xor_sync(CT_FULL, estiff, o, G);
  }
  if (live && l == 0) {
    const double qd = q[i];
    const double self = fma(fma(by_type(T.J, ti), qd, by_type(T.chi, ti)), qd, by_type(T.E0, ti));
    e_atom[i] = ((double)es + (double)ec) + (self + estiff);
  }
}

// ---------------------------------------------------------------- charge forces + gather
// One thread per atom over its column of the list: force, per-atom energy
// and virial in the working precision (compensated energy sum), then the
// FP64 store, half kick, kinetic energy and per-replica sums. Threads take
// 256-atom tiles strided over the grid, so the FP64 per-replica reductions
// are paid once per thread, not once per atom.
// Blocks per SM the register allocation must allow: three for the step
// variant at depth 4 (85 registers, no spills; 37.5% occupancy instead of
// 25%), one elsewhere (deeper pipelines and the virial spill under a cap).
template <int PB, bool VIR> constexpr int gather_min_blocks() { return (!VIR && PB <= 4) ? GATHER_MINB : 1; }

template <class R, int PB, bool VIR>
__global__ void __launch_bounds__(256, gather_min_blocks<PB, VIR>())
    k_coul_gather(int N, int cap_cov, int ld, const typename Vec4<R>::T* __restrict__ u,
                  const int* __restrict__ rep, const RepInfo* __restrict__ reps, const int2* __restrict__ nl,
                   const int* __restrict__ ncov, const int* __restrict__ nall,
                  const int* __restrict__ rev, const typename Vec4<R>::T* __restrict__ gslot,
                  const R* __restrict__ qr, PotParams<R> P, TypeParams T, int kick, double half_dt,
                  const uint8_t* __restrict__ frozen, double* __restrict__ F, double* __restrict__ v,
                  double* __restrict__ e_atom, double* __restrict__ rep_acc, unsigned* __restrict__ err,
                  const double* __restrict__ nh) {
  using R4 = typename Vec4<R>::T;
  // per-replica sums in one accumulator (the slot order of rep_acc): E, KE,
  // sum of |F|^2 (the RMS force that picks the next evaluation's mode),
  // virial. The virial and |F|^2 add up over this thread's atoms in the
  // working precision first (a dozen atoms at 1M; an FP64 warp instruction
  // costs the FP64 pipe as much as dozens of FP32 ones) and join the FP64
  // accumulator at each replica change and at the end.
  RepAcc<RA_STRIDE> acc;
  acc.init();
  R pw[10];   // virial, |F|^2
#pragma unroll
  for (int k = 0; k < 10; ++k) pw[k] = R(0);
  auto fold = [&]() {
#pragma unroll
    for (int k = 0; k < 9; ++k) acc.v[RA_W + k] += (double)pw[k];
    acc.v[RA_F2] += (double)pw[9];
#pragma unroll
    for (int k = 0; k < 10; ++k) pw[k] = R(0);
  };
  for (int t = blockIdx.x; (long long)t * 256 < N; t += gridDim.x) {
    int i = t * 256 + (int)threadIdx.x;
    if (i >= N) break;
    R4 ui = u[i];
    int ti = (int)ui.w;
    int ri_id = rep[i];
    const RepInfo& ri = reps[ri_id];
    R hx = ri.hcf[0], hy = ri.hcf[1], hz = ri.hcf[2];
    if (sizeof(R) == 8) { hx = (R)ri.hc[0]; hy = (R)ri.hc[1]; hz = (R)ri.hc[2]; }
    int nc = ncov[i], na = nall[i];
    R qi = qr[i];
    R fx = R(0), fy = R(0), fz = R(0);
    CompSum<R> ec;
    R w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = R(0);
    const int2* pl = nl + i;
    const R gs_i0 = P.gshield3[ti * 2], gs_i1 = P.gshield3[ti * 2 + 1];
    // covalent entries: charge term plus the slot gather
    for (int e = 0; e < nc; ++e) {
      size_t off = (size_t)e * ld;
      int2 jcd = __ldg(pl + off);
      int j = jcd.x;
      R4 uj = u[j];
      R rx, ry, rz;
      rel_vec<R>(ui, uj, jcd.y, hx, hy, hz, rx, ry, rz);
      R r2 = rx * rx + ry * ry + rz * rz;
      R r, ir, K, c;
      coul_fn_r2<R>(r2, uj.w != R(0) ? gs_i1 : gs_i0, P.inv_rcoul, P.ke, r, ir, K, c);
      R qq = qi * qr[j];
      c *= qq;
      R4 go = gslot[(size_t)i * cap_cov + e];
      R4 gr = gslot[(size_t)j * cap_cov + rev[(size_t)i * cap_cov + e]];
      R gx = c * rx + go.x - gr.x, gy = c * ry + go.y - gr.y, gz = c * rz + go.z - gr.z;
      fx += gx; fy += gy; fz += gz;
      ec.add(R(0.5) * qq * K);
      // virial: -1/2 qq K'/r r (x) r for the charge pair, -r (x) slot for the bond
      R hc = R(-0.5) * c;
      R tx = hc * rx - go.x, ty = hc * ry - go.y, tz = hc * rz - go.z;
      if (VIR) {
      w[0] += rx * tx; w[1] += rx * ty; w[2] += rx * tz;
      w[3] += ry * tx; w[4] += ry * ty; w[5] += ry * tz;
      w[6] += rz * tx; w[7] += rz * ty; w[8] += rz * tz;
      }
    }
    // remaining entries: charge term only, streamed
    int jn[PB], cn[PB];
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      bool ok = nc + k < na;
      int2 t = ok ? __ldg(pl + (size_t)(nc + k) * ld) : make_int2(i, pack_code(0, 0, 0));
      jn[k] = t.x;
      cn[k] = t.y;
    }
    for (int e = nc; e < na; e += PB) {
      int jc[PB], cc[PB];
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        jc[k] = jn[k];
        cc[k] = cn[k];
        int en = e + PB + k;
        bool ok = en < na;
        int2 t = ok ? __ldg(pl + (size_t)en * ld) : make_int2(i, pack_code(0, 0, 0));
        jn[k] = t.x;
        cn[k] = t.y;
      }
      R4 uj[PB];
      R qj[PB];
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        uj[k] = u[jc[k]];
        qj[k] = qr[jc[k]];
      }
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        if (e + k < na) {
          R rx, ry, rz;
          rel_vec<R>(ui, uj[k], cc[k], hx, hy, hz, rx, ry, rz);
          R r2 = rx * rx + ry * ry + rz * rz;
          R r, ir, K, c;
          coul_fn_r2<R>(r2, uj[k].w != R(0) ? gs_i1 : gs_i0, P.inv_rcoul, P.ke, r, ir, K, c);
          R qq = qi * qj[k];
          c *= qq;
          fx += c * rx; fy += c * ry; fz += c * rz;
          ec.add(R(0.5) * qq * K);
          R hc = R(-0.5) * c;
          R hx_ = hc * rx, hy_ = hc * ry, hz_ = hc * rz;
          if (VIR) {
          w[0] += rx * hx_; w[1] += rx * hy_; w[2] += rx * hz_;
          w[3] += ry * hx_; w[4] += ry * hy_; w[5] += ry * hz_;
          w[6] += rz * hx_; w[7] += rz * hy_; w[8] += rz * hz_;
          }
        }
      }
    }
    double Fx = fx, Fy = fy, Fz = fz;
    F[3 * i] = Fx; F[3 * i + 1] = Fy; F[3 * i + 2] = Fz;
    double ea = e_atom[i] + ec.value();
    e_atom[i] = ea;
    // finiteness from the working-precision sums and the FP64 exponent bits
    const bool bad_e = (__double_as_longlong(ea) & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;
    if (bad_e || !isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(err, CT_ERR_NONFINITE);
    if (ri_id != acc.rep) fold();
    acc.to(ri_id, rep_acc, RA_STRIDE);
    acc.v[RA_E] += ea;
    pw[9] += fx * fx + fy * fy + fz * fz;
#pragma unroll
    for (int k = 0; k < 9; ++k) pw[k] += w[k];
    if (kick && !frozen[i]) {
      double sc = half_dt * by_type(T.inv_mass_acc, ti);
      double vx = v[3 * i] + sc * Fx, vy = v[3 * i + 1] + sc * Fy, vz = v[3 * i + 2] + sc * Fz;
      const double* h = nh + (size_t)ri_id * NH_STRIDE;
      if (h[NH_ON] != 0.0) {   // NVT: the second velocity scaling, exp(-xi' dt/2)
        double s = exp(-half_dt * h[NH_XIH]);
        vx *= s; vy *= s; vz *= s;
      }
      v[3 * i] = vx; v[3 * i + 1] = vy; v[3 * i + 2] = vz;
    }
    {   // kinetic energy of the current velocities
      double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
      acc.v[RA_KE] += 0.5 * by_type(T.mass, ti) * (vx * vx + vy * vy + vz * vz);
    }
  }
  fold();
  lane_flush<RA_STRIDE>(acc, rep_acc, RA_STRIDE);
}

// FP64 offsets of every atom from its cell's origin (the layout of u), for
// the FP64 pass over queued atoms; nothing to do when the queue is empty.
__global__ void k_fill_u64(int N, const int* __restrict__ nq, const double* __restrict__ x,
                           const int4* __restrict__ cell4, const int* __restrict__ type,
                           const int* __restrict__ rep, const RepInfo* __restrict__ reps,
                           double4_32a* __restrict__ u64) {
  if (*nq == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const RepInfo& ri = reps[rep[i]];
    int4 c = cell4[i];
    double4_32a w;
    w.x = x[3 * i] - c.x * ri.hc[0];
    w.y = x[3 * i + 1] - c.y * ri.hc[1];
    w.z = x[3 * i + 2] - c.z * ri.hc[2];
    w.w = (double)type[i];
    u64[i] = w;
  }
}

// ---------------------------------------------------------------- launchers
// One thread per atom: as many 256-thread blocks as are resident at once
// (occupancy calculator), each a contiguous chunk of atoms.
int atom_dims(int N, int nsm, const void* kernel, int threads, int& chunk) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1) occ = 1;
  long long slots = (long long)nsm * occ;
  long long need = ((long long)N + threads - 1) / threads;
  long long grid = need < slots ? need : slots;
  if (grid < 1) grid = 1;
  long long ch = ((long long)N + grid - 1) / grid;
  ch = ((ch + threads - 1) / threads) * threads;
  chunk = (int)ch;
  return (int)(((long long)N + ch - 1) / ch);
}

static Taper64 taper64(const DevState& S) {
  Taper64 t;
  for (int k = 0; k < 4; ++k) {
    t.R2[k] = S.Pd->Rin[k] * S.Pd->Rin[k];
    t.S2[k] = S.Pd->Sout[k] * S.Pd->Sout[k];
  }
  return t;
}

template <class R> static size_t bond_smem(int cap, int G) {
  return (size_t)(CB / G) * cap * (sizeof(typename Vec4<R>::T) + sizeof(R) + 2 * sizeof(int));
}
template <class R> static size_t force_smem(int cap, int G) {
  return (size_t)(CB / G) * cap *
         (sizeof(typename Vec4<R>::T) + sizeof(typename Vec2<R>::T) + 3 * sizeof(R) + 2 * sizeof(int));
}

template <class R, int G>
static void launch_bond_g(const DevState& S, const PotParams<R>& P, cudaStream_t st) {
  size_t sm = bond_smem<R>(S.cap_cov, G);
  const int gb = (S.N + CB / G - 1) / (CB / G);
  const Taper64 tp = taper64(S);
  k_bond<R, G><<<gb, CB, sm, st>>>(
      S.N, S.cap_cov, S.ld, (const typename Vec4<R>::T*)S.u, S.rep, S.reps, S.nl,
      S.ncov, P, (typename Vec4<R>::T*)S.bo, S.stiff_n, S.stiff_q, S.acc_mode, S.flag_n, S.flag_q,
      nullptr, nullptr, sizeof(R) == 4 ? S.x : nullptr, S.cell4, tp);
  if constexpr (sizeof(R) == 4) {
    // the queued atoms in FP64: master-precision offsets, then their bond orders
    k_fill_u64<<<S.nsm * 4, 256, 0, st>>>(S.N, S.flag_n, S.x, S.cell4, S.type, S.rep, S.reps,
                                         (double4_32a*)S.u64);
    k_bond<double, G><<<gb, CB, bond_smem<double>(S.cap_cov, G), st>>>(
        S.N, S.cap_cov, S.ld, (const double4_32a*)S.u64, S.rep, S.reps, S.nl, S.ncov, *S.Pd,
        (double4_32a*)S.bo64, nullptr, nullptr, nullptr, nullptr, nullptr, S.flag_q, S.flag_n, nullptr, nullptr,
        tp);
  }
}

template <class R>
void launch_bond(const DevState& S, const PotParams<R>& P, cudaStream_t st) {
  if (S.N == 0) return;
  if (S.cov_lanes == 4) launch_bond_g<R, 4>(S, P, st);
  else if (S.cov_lanes == 16) launch_bond_g<R, 16>(S, P, st);
  else launch_bond_g<R, 8>(S, P, st);
}

template <class R>
void launch_assemble(const DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st) {
  if (S.N == 0) return;
#define ASM_ARGS                                                                                        \
  S.N, S.cap_cov, S.ld, (const typename Vec4<R>::T*)S.u, S.rep, S.reps, S.nl, S.ncov, S.nfix, S.nall, S.rev, \
      (const typename Vec4<R>::T*)S.bo, P, T, S.M, (R*)S.Dg, (R*)S.dinv, S.nmat
  const int g = (S.N + 255) / 256;
  if (S.asm_batch == 4) k_assemble<R, 4><<<g, 256, 0, st>>>(ASM_ARGS);
  else if (S.asm_batch == 16) k_assemble<R, 16><<<g, 256, 0, st>>>(ASM_ARGS);
  else k_assemble<R, 8><<<g, 256, 0, st>>>(ASM_ARGS);
#undef ASM_ARGS
}

template <class R, int G>
static void launch_cov_force_g(const DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st) {
  size_t sm = force_smem<R>(S.cap_cov, G);
  const int gb = (S.N + CB / G - 1) / (CB / G);
  const Taper64 tp = taper64(S);
  k_cov_force<R, R, G><<<gb, CB, sm, st>>>(
      S.N, S.cap_cov, S.ld, (const typename Vec4<R>::T*)S.u, S.rep, S.reps, S.nl, S.ncov,
      (const typename Vec4<R>::T*)S.bo, S.q, (const R*)S.qr, P, T, (typename Vec4<R>::T*)S.gslot, S.e_atom,
      S.stiff_pe, nullptr, nullptr, sizeof(R) == 4 ? S.x : nullptr, S.cell4, tp);
  if constexpr (sizeof(R) == 4) {
    // the queued atoms' slots and covalent energies again, in FP64
    k_cov_force<double, float, G><<<gb, CB, force_smem<double>(S.cap_cov, G), st>>>(
        S.N, S.cap_cov, S.ld, (const double4_32a*)S.u64, S.rep, S.reps, S.nl, S.ncov,
        (const double4_32a*)S.bo64, S.q, S.q, *S.Pd, T, (float4*)S.gslot, S.e_atom, nullptr, S.flag_q, S.flag_n,
        nullptr, nullptr, tp);
  }
}

template <class R>
void launch_cov_force(const DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st) {
  if (S.N == 0) return;
  if constexpr (sizeof(R) == 4) {
    // the stiff bonds queued by the bond pass, in FP64 (grid-strided over the queue)
    k_stiff<<<S.nsm * 4, 256, 0, st>>>(S.cap_cov, S.ld, S.stiff_n, S.stiff_q, S.nl, S.rep, S.reps, S.x,
                                       S.cell4, S.type, (const float4*)S.bo, S.q, P, (double2*)S.stiff_pe);
  }
  if (S.cov_lanes == 4) launch_cov_force_g<R, 4>(S, P, T, st);
  else if (S.cov_lanes == 16) launch_cov_force_g<R, 16>(S, P, T, st);
  else launch_cov_force_g<R, 8>(S, P, T, st);
}

template <class R>
void launch_coul_gather(const DevState& S, const PotParams<R>& P, const TypeParams& T, int kick, double half_dt,
                        cudaStream_t st, bool virial) {
  if (S.N == 0) return;
  auto go = [&](auto kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    long long tiles = ((long long)S.N + 255) / 256, slots = (long long)S.nsm * occ;
    int grid = (int)(tiles < slots ? tiles : slots);
    kernel<<<grid, 256, 0, st>>>(
        S.N, S.cap_cov, S.ld, (const typename Vec4<R>::T*)S.u, S.rep, S.reps, S.nl,
        S.ncov, S.nall, S.rev, (const typename Vec4<R>::T*)S.gslot, (const R*)S.qr, P, T, kick, half_dt,
        S.frozen, S.F, S.v, S.e_atom, S.rep_acc, S.err, S.nh);
  };
  if (virial) {
    if (S.gather_batch == 4) go(k_coul_gather<R, 4, true>);
    else if (S.gather_batch == 6) go(k_coul_gather<R, 6, true>);
    else go(k_coul_gather<R, 8, true>);
  } else {
    if (S.gather_batch == 4) go(k_coul_gather<R, 4, false>);
    else if (S.gather_batch == 6) go(k_coul_gather<R, 6, false>);
    else go(k_coul_gather<R, 8, false>);
  }
}

template <class R>
void launch_forces(const DevState& S, const PotParams<R>& P, const TypeParams& T, int kick, double half_dt,
                   cudaStream_t st, bool virial) {
  launch_cov_force<R>(S, P, T, st);
  launch_coul_gather<R>(S, P, T, kick, half_dt, st, virial);
}

template <class R, int G>
static cudaError_t setup_pot_g(int cap_cov) {
  cudaError_t e = cudaFuncSetAttribute(k_bond<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bond_smem<R>(cap_cov, G));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cov_force<R, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)force_smem<R>(cap_cov, G));
  if (e != cudaSuccess || sizeof(R) == 8) return e;
  // the FP32 path's FP64 pass over queued atoms
  e = cudaFuncSetAttribute(k_bond<double, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bond_smem<double>(cap_cov, G));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cov_force<double, float, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)force_smem<double>(cap_cov, G));
}

// Allow the dynamic shared memory the covalent kernels need for cap_cov
// entries per atom (call before launching or capturing them), at each lane
// count whose blocks fit the per-block limit: fewer lanes per atom stage
// more atoms per block. *lanes_ok gets a bit per usable count (1: 4 lanes,
// 2: 8, 4: 16); 16 lanes must fit.
template <class R>
cudaError_t setup_pot(int cap_cov, int* lanes_ok) {
  int dev = 0, lim = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  auto fits = [&](int G) {
    size_t need = std::max(force_smem<R>(cap_cov, G), bond_smem<R>(cap_cov, G));
    if (sizeof(R) == 4) need = std::max(need, force_smem<double>(cap_cov, G));
    return need <= (size_t)lim;
  };
  int ok = 0;
  if (fits(4)) { e = setup_pot_g<R, 4>(cap_cov); ok |= 1; }
  if (e == cudaSuccess && fits(8)) { e = setup_pot_g<R, 8>(cap_cov); ok |= 2; }
  if (e == cudaSuccess) { e = setup_pot_g<R, 16>(cap_cov); ok |= 4; }
  if (lanes_ok) *lanes_ok = ok;
  return e;
}
template cudaError_t setup_pot<float>(int, int*);
template cudaError_t setup_pot<double>(int, int*);

template void launch_bond<float>(const DevState&, const PotParams<float>&, cudaStream_t);
template void launch_bond<double>(const DevState&, const PotParams<double>&, cudaStream_t);
// Entries in flight per thread in the assembly (4, 8 or 16): each depth
// assembles the current matrix (the pass is idempotent: the same inputs give
// the same matrix), one warm-up and two timed launches. Another depth
// replaces the default 8 only when it is more than 10% faster: back to back
// on warm caches the depths time within a few per cent of each other, while
// inside a step (cold caches, moved atoms) depth 4 ran 28% slower than 8 on
// the 1M-atom slab after winning such a timing by 1%.
template <class R>
cudaError_t tune_assemble(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st,
                          float* ms_out) {
  if (S.N == 0) return cudaSuccess;
  const int depth[3] = {4, 8, 16};
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  float t[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    S.asm_batch = depth[k];
    launch_assemble<R>(S, P, T, st);
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 2; ++rep) launch_assemble<R>(S, P, T, st);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= 2.0f;
    if (ms_out) ms_out[k] = ms;
    t[k] = ms;
  }
  int pick = 8;
  float best = 0.9f * t[1];
  for (int k = 0; k < 3; k += 2)
    if (t[k] > 0.f && t[k] < best) { best = t[k]; pick = depth[k]; }
  S.asm_batch = pick;
  if (e == cudaSuccess) launch_assemble<R>(S, P, T, st);   // the matrix as the kept depth sums it
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}
template cudaError_t tune_assemble<float>(DevState&, const PotParams<float>&, const TypeParams&, cudaStream_t, float*);
template cudaError_t tune_assemble<double>(DevState&, const PotParams<double>&, const TypeParams&, cudaStream_t,
                                           float*);

// Streams up to 320 MB (about 2.5 L2 capacities) of the list-build scratch
// through L2 so that the next timed launch meets the cold cache it meets in
// a step (the scratch holds nothing between builds: one word per block is
// stored back into it only so that the loads are kept).
__global__ void k_l2_evict(const uint4* buf, size_t n, uint4* sink) {
  unsigned acc = 0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    uint4 v = __ldcg(buf + k);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  acc = __reduce_xor_sync(CT_FULL, acc);
  if (threadIdx.x == 0 && blockIdx.x < n) sink[blockIdx.x] = make_uint4(acc, 0, 0, 0);
}

static void evict_l2(const DevState& S, cudaStream_t st) {
  size_t n = (size_t)std::max(S.N, 1) * S.cap_all * sizeof(int2) / sizeof(uint4);
  n = std::min(n, (size_t)320 << 20 >> 4);
  if (n == 0 || S.lst == nullptr) return;
  k_l2_evict<<<S.nsm * 8, 256, 0, st>>>(reinterpret_cast<const uint4*>(S.lst), n, reinterpret_cast<uint4*>(S.lst));
}

// Lanes per atom in the covalent passes (4, 8 or 16; CB / G atoms per
// block): on the state of a completed evaluation, each lane count runs the
// bond pass (its queues emptied first, so repeated runs do not grow them)
// and the covalent force pass, three times each, the first a warm-up, each
// pass timed after an L2 eviction (in a step the matrix passes between them
// leave no covalent data in L2). The count with the least bond + force
// time is kept, and both passes, then the charge-force gather (no kick:
// forces, energies and sums as the evaluation left them), run once more in
// it. With fast set the timed runs take the FP32 path's fast mode (no
// previous force sums: the accurate mode of a first evaluation queues every
// pair term for FP64, a mix that MD steps above the RMS-force threshold
// never see); otherwise, and in the final run, the mode of the evaluation.
// Every count computes every bond alike (a lane owns whole bonds), so the
// results do not depend on the choice.
template <class R>
cudaError_t tune_cov(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st, float* ms_out,
                     bool fast) {
  if (S.N == 0) return cudaSuccess;
  const int lanes[3] = {4, 8, 16};
  const int start = S.cov_lanes;
  cudaEvent_t ev[3];
  cudaError_t e = cudaSuccess;
  int made = 0;
  for (; made < 3 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) {
    for (int k = 0; k < made - 1; ++k) cudaEventDestroy(ev[k]);
    return e;
  }
  auto clear_queues = [&]() {
    cudaMemsetAsync(S.stiff_n, 0, sizeof(int), st);
    if (S.flag_n) cudaMemsetAsync(S.flag_n, 0, sizeof(int), st);
  };
  float t[3] = {0.f, 0.f, 0.f};
  DevState F = S;
  if (fast) F.acc_mode = nullptr;   // the fast mode
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    if (!(S.cov_lanes_ok & (1 << k))) continue;
    F.cov_lanes = lanes[k];
    float sum = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      clear_queues();
      evict_l2(S, st);
      cudaEventRecord(ev[0], st);
      launch_bond<R>(F, P, st);
      cudaEventRecord(ev[1], st);
      e = cudaEventSynchronize(ev[1]);
      float a = 0.f, b = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
      evict_l2(S, st);
      cudaEventRecord(ev[1], st);
      launch_cov_force<R>(F, P, T, st);
      cudaEventRecord(ev[2], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
      if (rep > 0) sum += a + b;
    }
    t[k] = 0.5f * sum;
    if (ms_out) ms_out[k] = t[k];
  }
  int pick = start;
  float best = 0.f;
  for (int k = 0; k < 3; ++k)
    if (t[k] > 0.f && (best == 0.f || t[k] < best)) { best = t[k]; pick = lanes[k]; }
  S.cov_lanes = pick;
  if (e == cudaSuccess) {
    clear_queues();
    launch_bond<R>(S, P, st);
    launch_cov_force<R>(S, P, T, st);
    cudaMemsetAsync(S.rep_acc, 0, sizeof(double) * (size_t)S.R * RA_STRIDE, st);
    launch_coul_gather<R>(S, P, T, 0, 0.0, st, true);
  }
  for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
  return e == cudaSuccess ? cudaGetLastError() : e;
}
template cudaError_t tune_cov<float>(DevState&, const PotParams<float>&, const TypeParams&, cudaStream_t, float*,
                                     bool);
template cudaError_t tune_cov<double>(DevState&, const PotParams<double>&, const TypeParams&, cudaStream_t, float*,
                                      bool);

// Entries in flight per thread in the charge-force gather (4, 6 or 8; the
// depth sets the registers, 104 to 128, and so the resident blocks): on the
// state of a completed evaluation without a kick, each depth runs the
// covalent force pass (untimed: the gather adds to the per-atom energies it
// writes) and the gather without the virial (timed: the variant MD steps
// run), three times; the fastest is kept and the pair runs once more, with
// the virial, so the evaluation's results are as the kept depth sums them.
template <class R>
cudaError_t tune_gather(DevState& S, const PotParams<R>& P, const TypeParams& T, cudaStream_t st, float* ms_out) {
  if (S.N == 0) return cudaSuccess;
  const int depth[3] = {4, 6, 8};
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const size_t acc_bytes = sizeof(double) * (size_t)S.R * RA_STRIDE;
  float t[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    S.gather_batch = depth[k];
    float sum = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaMemsetAsync(S.rep_acc, 0, acc_bytes, st);
      launch_cov_force<R>(S, P, T, st);
      cudaEventRecord(e0, st);
      launch_coul_gather<R>(S, P, T, 0, 0.0, st, false);   // the variant MD steps run
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) sum += ms;   // the first is a warm-up
    }
    t[k] = 0.5f * sum;
    if (ms_out) ms_out[k] = t[k];
  }
  int pick = 8;
  float best = t[2];
  for (int k = 0; k < 2; ++k)
    if (t[k] > 0.f && t[k] < best) { best = t[k]; pick = depth[k]; }
  S.gather_batch = pick;
  if (e == cudaSuccess) {
    cudaMemsetAsync(S.rep_acc, 0, acc_bytes, st);
    launch_cov_force<R>(S, P, T, st);
    launch_coul_gather<R>(S, P, T, 0, 0.0, st, true);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}
template cudaError_t tune_gather<float>(DevState&, const PotParams<float>&, const TypeParams&, cudaStream_t, float*);
template cudaError_t tune_gather<double>(DevState&, const PotParams<double>&, const TypeParams&, cudaStream_t,
                                         float*);

template void launch_assemble<float>(const DevState&, const PotParams<float>&, const TypeParams&, cudaStream_t);
template void launch_assemble<double>(const DevState&, const PotParams<double>&, const TypeParams&, cudaStream_t);
template void launch_cov_force<float>(const DevState&, const PotParams<float>&, const TypeParams&, cudaStream_t);
template void launch_cov_force<double>(const DevState&, const PotParams<double>&, const TypeParams&, cudaStream_t);
template void launch_coul_gather<float>(const DevState&, const PotParams<float>&, const TypeParams&, int, double,
                                        cudaStream_t, bool);
template void launch_coul_gather<double>(const DevState&, const PotParams<double>&, const TypeParams&, int, double,
                                         cudaStream_t, bool);
template void launch_forces<float>(const DevState&, const PotParams<float>&, const TypeParams&, int, double,
                                   cudaStream_t, bool);
template void launch_forces<double>(const DevState&, const PotParams<double>&, const TypeParams&, int, double,
                                    cudaStream_t, bool);

}  // namespace ct
