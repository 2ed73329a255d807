// CUDA kernels of the short-characteristics library (sm_103a).
//
//   sc_sweep_kernel   formal solution of one sweep group for one frequency (Sec. 3.3)
//   ali_update_kernel Jacobi ALI update, FP64 (Sec. 3.4, Eq. 24) + max |dS|/S (Eq. 25)
//   lstar_kernel      diagonal Lambda* = sum_k w_k Psi0_k (Sec. 3.4)
//   finish_kernel     convergence decision and ghost-parity advance (one thread)
//   plus set-up kernels: validation, permuted sweep copies, ghost initialisation,
//   boundary intensities, J / moment reductions and the heating rate (Sec. 4).
//
// No kernel waits on another block: the only cross-CTA synchronisation is the
// hardware cluster barrier inside one cluster, which every CTA of the cluster
// reaches the same number of times.
#include <cooperative_groups.h>
#include <type_traits>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <utility>

#include "rt_common.cuh"
#include "rt_device.cuh"
#include "rt_kernels.h"

namespace cg = cooperative_groups;

namespace rtk {


// ------------------------------------------------------------------------ sweep


// One sweep group (rays sharing the crossed-face axis a and sign(mu_a)) for one
// frequency.  The plane normal to a is split into C strips of rows (v) over the C
// CTAs of a cluster.  Every step computes one plane from the previous plane:
//   I- , S-, chi- bilinear on the upwind face (weights wa..wd of the ray),
//   dtau = (chi- + chi0) s/2,  I0 = S- + E (I- - S-) + Psi0 (S0 - S-),
// which equals I- E + Psi- S- + Psi0 S0 with Psi- = 1 - E - Psi0 (Eq. 20, linear).
// The previous plane's intensities live in shared memory (double-buffered); a
// strip's edge row comes from the neighbouring CTA's shared memory (DSMEM).
// J partial of the group is the FP-T sum over its rays, written once per cell.
template <typename T, int AMAX, bool MOM>
__global__ void __launch_bounds__(512) sc_sweep_kernel(const SweepArgs<T> A) {
  if (A.skip_if_done && A.st->done) return;
  const int C = A.cluster;
  const int rank = blockIdx.x % C;
  const int inst = blockIdx.x / C;
  const int gi = inst % A.ngroups;
  const int f = inst / A.ngroups;
  const GroupParam gp = A.grp[gi];
  if (A.gs_forward && gp.axis == A.gs_axis && gp.sa < 0) return;   // swept in the reverse phase
  if (gp.na > A.ray_slots) {   // plan inconsistent with the shared-memory layout: refuse to run
    if (threadIdx.x == 0) atomicCAS(&A.st->err, 0, 30);
    return;
  }
  int cax[3];
  plane_axes(gp.axis, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const int perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
            perW = pick3(A.d.periodic, cax[2]);
  const long long csu = canon_stride(A.d.n, cax[0]), csv = canon_stride(A.d.n, cax[1]),
                  csw = canon_stride(A.d.n, cax[2]);   // canonical strides of u, v, w
  const int v0 = (int)(((long long)rank * Nv) / C);
  const int v1 = (int)(((long long)(rank + 1) * Nv) / C);
  const int R = v1 - v0;
  const int Rmax = (Nv + C - 1) / C;
  const long long plane = (long long)Nu * Nv;
  const long long cells = A.d.cells;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ibuf = reinterpret_cast<T *>(smem_raw);
  const int bufstride = A.ray_slots * Rmax * Nu;   // one plane of every ray slot
#ifdef RT_DEBUG_BOUNDS
  const long long smem_n = 2LL * bufstride;
#endif

  __shared__ AngleParam<T> P[AMAX];
  if (threadIdx.x < gp.na) P[threadIdx.x] = A.ang[gp.a0 + threadIdx.x];
  __syncthreads();

  const int fs = A.st->fs_count + A.parity_offset;
  const int prev = fs & 1;
  const T *Gp = A.G[prev];
  T *Gn = A.G[prev ^ 1];
  // Incremental ALI solves: the first formal solution is a full one that also
  // records its ghost increments; every later one sweeps dS with the ghost
  // increments as inflow (zero at fixed faces) and keeps the full ghosts current.
  const bool inc = A.incremental && A.st->iter > 0;
  const bool emit = A.incremental && A.st->iter == 0;
  const T *Gsrc = inc ? A.Gd[prev] : Gp;
  T *Gdn = A.incremental ? A.Gd[prev ^ 1] : nullptr;
  const T *chiP = A.chiP[gp.axis] + (long long)f * cells;
  const T *SP = A.SP[gp.axis] + (long long)f * cells;
  T *Jout = A.Jpart + ((long long)gi * A.d.nf + f) * cells;
  const int sa = gp.sa;
  const int wlast = sa > 0 ? Nw - 1 : 0;
  cg::cluster_group cluster = cg::this_cluster();
  // subdomain z faces: z is the sweep axis w (z sweeps) or the plane axis v (x,
  // y sweeps); the ghost layer's cells are [y][x], (x, y) = (u, v) for z sweeps,
  // (w, u) for x sweeps, (u, w) for y sweeps
  const bool zw = cax[2] == 2, zv = cax[1] == 2;
  const int xw = (zw && A.ext[sa > 0 ? 0 : 1]) ? (sa > 0 ? 0 : 1) : -1;   // beyond the first plane
  const int n0 = A.d.n[0];
  const long long f2 = (long long)n0 * A.d.n[1];
  auto xfc = [&](int uu, int ww) -> long long {   // ghost-layer cell of plane cell (uu, v past the face, ww)
    return gp.axis == 0 ? (long long)uu * n0 + ww : (long long)ww * n0 + uu;
  };

  for (int t = 0; t < Nw; ++t) {
    const int w = sa > 0 ? t : Nw - 1 - t;
    const int wp = w - sa;
    const bool wp_in = t > 0;
    const int wpm = wp_in ? wp : (perW ? (wp < 0 ? wp + Nw : wp - Nw) : w);
    T *cur = Ibuf + (t & 1) * bufstride;
    const T *prv = Ibuf + ((t + 1) & 1) * bufstride;
    const long long pbase = (long long)wpm * plane;
    for (int c = threadIdx.x; c < R * Nu; c += blockDim.x) {
      const int u = c % Nu;
      const int lv = c / Nu;
      const int v = v0 + lv;
      const long long pidx = ((long long)w * Nv + v) * Nu + u;
      const T chi0 = chiP[RT_IDX(pidx, cells, 1)];
      const T S0 = SP[RT_IDX(pidx, cells, 2)];
      const long long canon = (long long)(u) * csu + (long long)v * csv + (long long)w * csw;
      T Jacc = T(0);
      T Hm[3] = {T(0), T(0), T(0)};
      T Km[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < AMAX; ++a) {
        if (a < gp.na) {
          const AngleParam<T> &p = P[a];
          const int ua = u - p.su, vb = v - p.sv;
          const bool ua_in = (unsigned)ua < (unsigned)Nu;
          const bool vb_in = (unsigned)vb < (unsigned)Nv;
          const int um = ua_in ? ua : (perU ? (ua < 0 ? ua + Nu : ua - Nu) : u);
          const int vm = vb_in ? vb : (perV ? (vb < 0 ? vb + Nv : vb - Nv) : v);
          const long long iA = pbase + (long long)v * Nu + u;
          const long long iB = pbase + (long long)v * Nu + um;
          const long long iC = pbase + (long long)vm * Nu + u;
          const long long iD = pbase + (long long)vm * Nu + um;
          // the upwind face beyond a subdomain z face: the whole face (z sweeps at the
          // first plane) or its rows v - sv (x, y sweeps) read the ghost layer
          const bool xall = !wp_in && xw >= 0;
          const int xr = (!xall && zv && !vb_in && A.ext[vb < 0 ? 0 : 1]) ? (vb < 0 ? 0 : 1) : -1;
          T sA, sB, sC, sD;
          if (xall) {
            const T *X = A.xS[xw] + (long long)f * f2;
            sA = X[RT_IDX((long long)v * Nu + u, f2, 63)];
            sB = X[RT_IDX((long long)v * Nu + um, f2, 63)];
            sC = X[RT_IDX((long long)vm * Nu + u, f2, 63)];
            sD = X[RT_IDX((long long)vm * Nu + um, f2, 63)];
          } else {
            sA = SP[RT_IDX(iA, cells, 4)];
            sB = SP[RT_IDX(iB, cells, 4)];
            if (xr >= 0) {
              const T *X = A.xS[xr] + (long long)f * f2;
              sC = X[RT_IDX(xfc(u, wpm), f2, 64)];
              sD = X[RT_IDX(xfc(um, wpm), f2, 64)];
            } else {
              sC = SP[RT_IDX(iC, cells, 4)];
              sD = SP[RT_IDX(iD, cells, 4)];
            }
          }
          T IA, IB, IC, ID;
          if (wp_in) {
            const int rowA = (a * Rmax + lv) * Nu;
            IA = prv[RT_IDX(rowA + u, smem_n, 5)];
            IB = ua_in ? prv[RT_IDX(rowA + ua, smem_n, 5)]
                       : ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, ua, v, wp);
            if (vb_in) {
              const T *src = prv;
              int lvb = vb - v0;
              if (vb < v0 || vb >= v1) {
                const int rr = vb < v0 ? rank - 1 : rank + 1;
                const int rv0 = (int)(((long long)rr * Nv) / C);
                src = cluster.map_shared_rank(const_cast<T *>(prv), rr);
                lvb = vb - rv0;
              }
              const int rowC = (a * Rmax + lvb) * Nu;
              IC = src[RT_IDX(rowC + u, smem_n, 6)];
              ID = ua_in ? src[RT_IDX(rowC + ua, smem_n, 6)]
                         : ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, ua, vb, wp);
            } else {
              IC = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, u, vb, wp);
              ID = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, ua, vb, wp);
            }
          } else {
            IA = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, u, v, wp);
            IB = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, ua, v, wp);
            IC = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, u, vb, wp);
            ID = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, ua, vb, wp);
          }
          const T Sm = p.wa * sA + p.wb * sB + p.wc * sC + p.wd * sD;
          const T Im = p.wa * IA + p.wb * IB + p.wc * IC + p.wd * ID;
          T E, psi0;
          if (A.WE) {   // the medium's segment weights, tabulated once
            const long long wi = ((long long)(gp.a0 + a) * A.d.nf + f) * cells + pidx;
            E = A.WE[wi];
            psi0 = A.WP[wi];
          } else {
            T cA, cB, cC, cD;
            if (xall) {
              const T *X = A.xchi[xw] + (long long)f * f2;
              cA = X[(long long)v * Nu + u];
              cB = X[(long long)v * Nu + um];
              cC = X[(long long)vm * Nu + u];
              cD = X[(long long)vm * Nu + um];
            } else {
              cA = chiP[RT_IDX(iA, cells, 3)];
              cB = chiP[RT_IDX(iB, cells, 3)];
              if (xr >= 0) {
                const T *X = A.xchi[xr] + (long long)f * f2;
                cC = X[xfc(u, wpm)];
                cD = X[xfc(um, wpm)];
              } else {
                cC = chiP[RT_IDX(iC, cells, 3)];
                cD = chiP[RT_IDX(iD, cells, 3)];
              }
            }
            const T chim = p.wa * cA + p.wb * cB + p.wc * cC + p.wd * cD;
            const T dtau = (chim + chi0) * p.hs;
            T om;
            seg_weights(dtau, E, psi0, om);
          }
          const T I0 = Sm + E * (Im - Sm) + psi0 * (S0 - Sm);
          cur[RT_IDX((a * Rmax + lv) * Nu + u, smem_n, 7)] = I0;
          {   // intensities on the first / last z plane, for the neighbouring subdomains
            const int z = zw ? w : v;
            const int side = z == 0 ? 0 : (z == A.d.n[2] - 1 ? 1 : -1);
            if (side >= 0 && A.xout[side]) {
              const long long fc = zw ? (long long)v * Nu + u : xfc(u, w);
              A.xout[side][RT_IDX(((long long)f * A.na + p.angle) * f2 + fc, (long long)A.d.nf * A.na * f2, 65)] = I0;
            }
          }
          const T wI = p.wq * I0;
          Jacc += wI;
          if (MOM) {
            Hm[0] += wI * p.mu[0];
            Hm[1] += wI * p.mu[1];
            Hm[2] += wI * p.mu[2];
            Km[0] += wI * p.mu[0] * p.mu[0];
            Km[1] += wI * p.mu[1] * p.mu[1];
            Km[2] += wI * p.mu[2] * p.mu[2];
            Km[3] += wI * p.mu[0] * p.mu[1];
            Km[4] += wI * p.mu[0] * p.mu[2];
            Km[5] += wI * p.mu[1] * p.mu[2];
          }
          if (A.write_ghosts) {
            const long long gb = ((long long)f * A.na + p.angle) * A.d.gsize;
            const long long gn = (long long)A.d.nf * A.na * A.d.gsize;
            long long off = -1;
            if (perW && w == wlast) off = gb + (long long)v * Nu + u;
            if (off >= 0) ghost_store<T>(Gp, Gn, Gdn, RT_IDX(off, gn, 8), I0, inc, emit);
            off = -1;
            if (perU && u == (p.su > 0 ? Nu - 1 : 0)) off = gb + plane + (long long)w * Nv + v;
            if (off >= 0) ghost_store<T>(Gp, Gn, Gdn, RT_IDX(off, gn, 9), I0, inc, emit);
            off = -1;
            if (perV && v == (p.sv > 0 ? Nv - 1 : 0)) off = gb + plane + (long long)Nw * Nv + (long long)w * Nu + u;
            if (off >= 0) ghost_store<T>(Gp, Gn, Gdn, RT_IDX(off, gn, 10), I0, inc, emit);
          }
        }
      }
      Jout[RT_IDX(canon, cells, 13)] = Jacc;
      if (MOM) {
        T *M = A.Mpart + (long long)gi * 9 * A.d.nf * cells;
        const long long qs = (long long)A.d.nf * cells;
        const long long o = (long long)f * cells + canon;
#pragma unroll
        for (int q = 0; q < 3; ++q) M[q * qs + o] = Hm[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) M[(3 + q) * qs + o] = Km[q];
      }
    }
    if (C > 1) cluster.sync();
    else __syncthreads();
  }
}

// ------------------------------------------------------------- tiled sweep
// Same formal solution as sc_sweep_kernel, organised for throughput:
//  * the upwind plane's intensities, opacity and source function are staged in
//    shared memory with a one-cell halo (filled once per step from the
//    neighbouring strips over DSMEM, or from the ghost rules), so the per-ray
//    update reads shared memory only, without boundary tests;
//  * chi and S of the current plane are staged too (they are the next step's
//    upwind plane);
//  * a thread computes SEG consecutive cells of one row, reusing the staged
//    row values in registers, and each ray's signs (su, sv) are template
//    parameters of the update so all register indexing is static.

template <typename T, int SEG, bool MOM, int SU, int SV>
__device__ __forceinline__ void seg_update(const AngleParam<T> &p, const T *__restrict__ Ip,
                                           T *__restrict__ Ic, int row, int u0, int ncell, int W,
                                           const T (&cm)[SEG + 2], const T (&c0)[SEG + 2],
                                           const T (&cp)[SEG + 2], const T (&sm)[SEG + 2],
                                           const T (&s0)[SEG + 2], const T (&sp)[SEG + 2],
                                           const T (&chi0)[SEG], const T (&S0)[SEG], T (&out)[SEG]) {
  // intensities of the upwind plane on rows v and v - SV, columns covering the segment
  const int cb = u0 + (SU > 0 ? 0 : 1);
  T Ia[SEG + 1], Iv[SEG + 1];
#pragma unroll
  for (int k = 0; k < SEG + 1; ++k) {
    Ia[k] = Ip[row * W + cb + k];
    Iv[k] = Ip[(row - SV) * W + cb + k];
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int kA = j + (SU > 0 ? 1 : 0), kB = j + (SU > 0 ? 0 : 1);
    const int jA = j + 1, jB = j + 1 - SU;
    const T chiC = SV > 0 ? cm[jA] : cp[jA], chiD = SV > 0 ? cm[jB] : cp[jB];
    const T sC = SV > 0 ? sm[jA] : sp[jA], sD = SV > 0 ? sm[jB] : sp[jB];
    const T chim = p.wa * c0[jA] + p.wb * c0[jB] + p.wc * chiC + p.wd * chiD;
    const T Sm = p.wa * s0[jA] + p.wb * s0[jB] + p.wc * sC + p.wd * sD;
    const T Im = p.wa * Ia[kA] + p.wb * Ia[kB] + p.wc * Iv[kA] + p.wd * Iv[kB];
    const T dtau = (chim + chi0[j]) * p.hs;
    T E, psi0, om;
    seg_weights(dtau, E, psi0, om);
    const T I0 = Sm + E * (Im - Sm) + psi0 * (S0[j] - Sm);
    out[j] = I0;
    if (j < ncell) Ic[row * W + u0 + j + 1] = I0;
  }
}

template <typename T, int AMAX, bool MOM, int SEG>
__global__ void __launch_bounds__(sweep_max_threads<T>()) sc_sweep_tiled_kernel(const SweepArgs<T> A) {
  if (A.skip_if_done && A.st->done) return;
  const int C = A.cluster;
  const int rank = blockIdx.x % C;
  const int inst = blockIdx.x / C;
  const int gi = inst % A.ngroups;
  const int f = inst / A.ngroups;
  const GroupParam gp = A.grp[gi];
  if (A.gs_forward && gp.axis == A.gs_axis && gp.sa < 0) return;   // swept in the reverse phase
  if (gp.na > A.ray_slots) {   // plan inconsistent with the shared-memory layout: refuse to run
    if (threadIdx.x == 0) atomicCAS(&A.st->err, 0, 30);
    return;
  }
  int cax[3];
  plane_axes(gp.axis, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const int perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
            perW = pick3(A.d.periodic, cax[2]);
  const long long csu = canon_stride(A.d.n, cax[0]), csv = canon_stride(A.d.n, cax[1]),
                  csw = canon_stride(A.d.n, cax[2]);   // canonical strides of u, v, w
  const int v0 = (int)(((long long)rank * Nv) / C);
  const int v1 = (int)(((long long)(rank + 1) * Nv) / C);
  const int R = v1 - v0;
  const int Rmax = (Nv + C - 1) / C;
  const int W = Nu + 2 + SEG;          // staged row: halo, Nu cells, halo, padding
  const int RX = Rmax + 2;
  const int pb = RX * W;               // one staged plane
  const int ib = A.ray_slots * pb;     // one plane of every ray of the group
  const long long plane = (long long)Nu * Nv;
  const long long cells = A.d.cells;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ib = reinterpret_cast<T *>(smem_raw);   // [2][AMAX][RX][W]
  T *Cb = Ib + 2 * ib;                       // [2][RX][W]
  T *Sb = Cb + 2 * pb;                       // [2][RX][W]
#ifdef RT_DEBUG_BOUNDS
  const long long smem_n = 2LL * ib + 4LL * pb;
#endif
  __shared__ AngleParam<T> P[AMAX];
  if (threadIdx.x < gp.na) P[threadIdx.x] = A.ang[gp.a0 + threadIdx.x];
  __syncthreads();

  const int fs = A.st->fs_count + A.parity_offset;
  const int prev = fs & 1;
  const T *Gp = A.G[prev];
  T *Gn = A.G[prev ^ 1];
  const bool inc = A.incremental && A.st->iter > 0;
  const bool emit = A.incremental && A.st->iter == 0;
  const T *Gsrc = inc ? A.Gd[prev] : Gp;
  T *Gdn = A.incremental ? A.Gd[prev ^ 1] : nullptr;
  const T *chiP = A.chiP[gp.axis] + (long long)f * cells;
  const T *SP = A.SP[gp.axis] + (long long)f * cells;
  T *Jout = A.Jpart + ((long long)gi * A.d.nf + f) * cells;
  const int sa = gp.sa;
  const int wlast = sa > 0 ? Nw - 1 : 0;
  const int na = gp.na;
  const int nseg = (Nu + SEG - 1) / SEG;
  const int ext = (R + 2) * (Nu + 2);
  cg::cluster_group cluster = cg::this_cluster();

  auto stage_fields = [&](int wsrc, T *Cd, T *Sd) {
    for (int idx = threadIdx.x; idx < ext; idx += blockDim.x) {
      const int row = idx / (Nu + 2), col = idx - row * (Nu + 2);
      int uu = col - 1, vv = v0 - 1 + row;
      uu = uu < 0 ? (perU ? uu + Nu : 0) : (uu >= Nu ? (perU ? uu - Nu : Nu - 1) : uu);
      vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
      const long long o = (long long)wsrc * plane + (long long)vv * Nu + uu;
      Cd[RT_IDX(row * W + col, pb, 20)] = chiP[RT_IDX(o, cells, 21)];
      Sd[RT_IDX(row * W + col, pb, 20)] = SP[RT_IDX(o, cells, 21)];
    }
  };

  for (int t = 0; t < Nw; ++t) {
    const int w = sa > 0 ? t : Nw - 1 - t;
    const int wp = w - sa;
    const bool wp_in = t > 0;
    T *Icur = Ib + (t & 1) * ib;
    T *Iprv = Ib + ((t + 1) & 1) * ib;
    T *Ccur = Cb + (t & 1) * pb, *Cprv = Cb + ((t + 1) & 1) * pb;
    T *Scur = Sb + (t & 1) * pb, *Sprv = Sb + ((t + 1) & 1) * pb;

    // 1. chi, S of this plane (and of the upwind ghost plane on the first step)
    stage_fields(w, Ccur, Scur);
    if (!wp_in) stage_fields(perW ? (wp < 0 ? wp + Nw : wp - Nw) : w, Cprv, Sprv);
    // 2. intensities of the upwind plane outside this strip
    if (!wp_in) {
      for (int idx = threadIdx.x; idx < na * ext; idx += blockDim.x) {
        const int a = idx / ext, r2 = idx - a * ext;
        const int row = r2 / (Nu + 2), col = r2 - row * (Nu + 2);
        Iprv[RT_IDX(a * pb + row * W + col, 2LL * ib, 22)] =
            ghost_I<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, col - 1, v0 - 1 + row, wp);
      }
    } else {
      for (int idx = threadIdx.x; idx < na * 2 * Nu; idx += blockDim.x) {
        const int a = idx / (2 * Nu), r2 = idx - a * 2 * Nu;
        const int side = r2 / Nu, u = r2 - side * Nu;
        const int vv = side ? v1 : v0 - 1;
        const int row = side ? R + 1 : 0;
        T val;
        if (vv >= 0 && vv < Nv) {
          const int rr = side ? rank + 1 : rank - 1;
          const int rv0 = (int)(((long long)rr * Nv) / C);
          const T *src = cluster.map_shared_rank(Iprv, rr);
          val = src[RT_IDX(a * pb + (vv - rv0 + 1) * W + u + 1, 2LL * ib, 23)];
        } else {
          val = ghost_I<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, u, vv, wp);
        }
        Iprv[RT_IDX(a * pb + row * W + u + 1, 2LL * ib, 24)] = val;
      }
      for (int idx = threadIdx.x; idx < na * 2 * (R + 2); idx += blockDim.x) {
        const int a = idx / (2 * (R + 2)), r2 = idx - a * 2 * (R + 2);
        const int side = r2 / (R + 2), row = r2 - side * (R + 2);
        Iprv[RT_IDX(a * pb + row * W + (side ? Nu + 1 : 0), 2LL * ib, 25)] =
            ghost_I<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, side ? Nu : -1, v0 - 1 + row, wp);
      }
    }
    __syncthreads();

    // 3. the strip's cells, SEG per thread
    for (int sidx = threadIdx.x; sidx < R * nseg; sidx += blockDim.x) {
      const int lv = sidx / nseg, seg = sidx - lv * nseg;
      const int u0 = seg * SEG, v = v0 + lv, row = lv + 1;
      const int ncell = min(SEG, Nu - u0);
      T cm[SEG + 2], c0[SEG + 2], cp[SEG + 2], sm[SEG + 2], s0[SEG + 2], sp[SEG + 2];
#pragma unroll
      for (int j = 0; j < SEG + 2; ++j) {
        cm[j] = Cprv[(row - 1) * W + u0 + j];
        c0[j] = Cprv[row * W + u0 + j];
        cp[j] = Cprv[(row + 1) * W + u0 + j];
        sm[j] = Sprv[(row - 1) * W + u0 + j];
        s0[j] = Sprv[row * W + u0 + j];
        sp[j] = Sprv[(row + 1) * W + u0 + j];
      }
      T chi0[SEG], S0[SEG], Jacc[SEG];
      T Hm[MOM ? SEG : 1][3], Km[MOM ? SEG : 1][6];
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        chi0[j] = Ccur[row * W + u0 + j + 1];
        S0[j] = Scur[row * W + u0 + j + 1];
        Jacc[j] = T(0);
        if (MOM) {
#pragma unroll
          for (int q = 0; q < 3; ++q) Hm[MOM ? j : 0][q] = T(0);
#pragma unroll
          for (int q = 0; q < 6; ++q) Km[MOM ? j : 0][q] = T(0);
        }
      }
#pragma unroll
      for (int a = 0; a < AMAX; ++a) {
        if (a < na) {
          const AngleParam<T> &p = P[a];
          const T *Ip = Iprv + a * pb;
          T *Ic = Icur + a * pb;
          T I0[SEG];
          const int key = (p.su > 0 ? 1 : 0) | (p.sv > 0 ? 2 : 0);
          if (key == 3) seg_update<T, SEG, MOM, 1, 1>(p, Ip, Ic, row, u0, ncell, W, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
          else if (key == 2) seg_update<T, SEG, MOM, -1, 1>(p, Ip, Ic, row, u0, ncell, W, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
          else if (key == 1) seg_update<T, SEG, MOM, 1, -1>(p, Ip, Ic, row, u0, ncell, W, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
          else seg_update<T, SEG, MOM, -1, -1>(p, Ip, Ic, row, u0, ncell, W, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
#pragma unroll
          for (int j = 0; j < SEG; ++j) {
            const T wI = p.wq * I0[j];
            Jacc[j] += wI;
            if (MOM) {
              Hm[MOM ? j : 0][0] += wI * p.mu[0];
              Hm[MOM ? j : 0][1] += wI * p.mu[1];
              Hm[MOM ? j : 0][2] += wI * p.mu[2];
              Km[MOM ? j : 0][0] += wI * p.mu[0] * p.mu[0];
              Km[MOM ? j : 0][1] += wI * p.mu[1] * p.mu[1];
              Km[MOM ? j : 0][2] += wI * p.mu[2] * p.mu[2];
              Km[MOM ? j : 0][3] += wI * p.mu[0] * p.mu[1];
              Km[MOM ? j : 0][4] += wI * p.mu[0] * p.mu[2];
              Km[MOM ? j : 0][5] += wI * p.mu[1] * p.mu[2];
            }
          }
          if (A.write_ghosts) {
            const long long gb = ((long long)f * A.na + p.angle) * A.d.gsize;
            const long long gn = (long long)A.d.nf * A.na * A.d.gsize;
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
              if (j < ncell) {
                const int u = u0 + j;
                if (perW && w == wlast)
                  ghost_store<T>(Gp, Gn, Gdn, RT_IDX(gb + (long long)v * Nu + u, gn, 26), I0[j], inc, emit);
                if (perU && u == (p.su > 0 ? Nu - 1 : 0))
                  ghost_store<T>(Gp, Gn, Gdn, RT_IDX(gb + plane + (long long)w * Nv + v, gn, 27), I0[j], inc, emit);
                if (perV && v == (p.sv > 0 ? Nv - 1 : 0))
                  ghost_store<T>(Gp, Gn, Gdn, RT_IDX(gb + plane + (long long)Nw * Nv + (long long)w * Nu + u, gn, 28),
                                 I0[j], inc, emit);
              }
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        if (j < ncell) {
          const long long canon = (long long)(u0 + j) * csu + (long long)v * csv + (long long)w * csw;
          Jout[RT_IDX(canon, cells, 29)] = Jacc[j];
          if (MOM) {
            T *M = A.Mpart + (long long)gi * 9 * A.d.nf * cells;
            const long long qs = (long long)A.d.nf * cells;
            const long long o = (long long)f * cells + canon;
#pragma unroll
            for (int q = 0; q < 3; ++q) M[q * qs + o] = Hm[MOM ? j : 0][q];
#pragma unroll
            for (int q = 0; q < 6; ++q) M[(3 + q) * qs + o] = Km[MOM ? j : 0][q];
          }
        }
      }
    }
    if (C > 1) cluster.sync();
    else __syncthreads();
  }
}

// Segment weights of the one-cell-per-thread sweep, tabulated per medium: for
// each ray of group gi (slots gp.a0 ...) and cell (in the group's [w][v][u]
// layout) the E and Psi0 that sc_sweep_kernel would compute there -- the same
// upwind vertices (periodic image or the cell's own row/column/plane at a
// bounded face) and the same expressions.
template <typename T>
__global__ void __launch_bounds__(256) seg_table_kernel(const SweepArgs<T> A, int gi, T *WE, T *WP) {
  const GroupParam gp = A.grp[gi];
  int cax[3];
  plane_axes(gp.axis, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const int perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
            perW = pick3(A.d.periodic, cax[2]);
  const long long cells = A.d.cells, plane = (long long)Nu * Nv;
  const long long n = (long long)gp.na * A.d.nf * cells;
  const int sa = gp.sa;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(k / ((long long)A.d.nf * cells));
    const int f = (int)((k / cells) % A.d.nf);
    const long long pidx = k % cells;
    const int u = (int)(pidx % Nu), v = (int)((pidx / Nu) % Nv), w = (int)(pidx / plane);
    const AngleParam<T> p = A.ang[gp.a0 + a];
    const T *chiP = A.chiP[gp.axis] + (long long)f * cells;
    const int wp = w - sa;
    const bool wp_in = (unsigned)wp < (unsigned)Nw;
    const int wpm = wp_in ? wp : (perW ? (wp < 0 ? wp + Nw : wp - Nw) : w);
    const long long pbase = (long long)wpm * plane;
    const int ua = u - p.su, vb = v - p.sv;
    const bool ua_in = (unsigned)ua < (unsigned)Nu;
    const bool vb_in = (unsigned)vb < (unsigned)Nv;
    const int um = ua_in ? ua : (perU ? (ua < 0 ? ua + Nu : ua - Nu) : u);
    const int vm = vb_in ? vb : (perV ? (vb < 0 ? vb + Nv : vb - Nv) : v);
    const T cA = chiP[pbase + (long long)v * Nu + u], cB = chiP[pbase + (long long)v * Nu + um];
    const T cC = chiP[pbase + (long long)vm * Nu + u], cD = chiP[pbase + (long long)vm * Nu + um];
    const T chim = p.wa * cA + p.wb * cB + p.wc * cC + p.wd * cD;
    const T dtau = (chim + chiP[pidx]) * p.hs;
    T E, psi0, om;
    seg_weights(dtau, E, psi0, om);
    const long long wi = ((long long)(gp.a0 + a) * A.d.nf + f) * cells + pidx;
    WE[wi] = E;
    WP[wi] = psi0;
  }
}

template <typename T>
cudaError_t launch_seg_table(const SweepArgs<T> &A, int gi, int nslots, T *WE, T *WP, cudaStream_t s) {
  const long long n = (long long)nslots * A.d.nf * A.d.cells;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
  seg_table_kernel<T><<<grid, 256, 0, s>>>(A, gi, WE, WP);
  return cudaGetLastError();
}

// ------------------------------------------------------------ pipelined sweep
// The tiled organisation with the plane loads taken off the critical path:
//  * chi and S planes live in a three-deep ring in shared memory; while plane t
//    is computed, plane t+1 streams in with cp.async (16-byte copies when rows
//    are 16-byte aligned), so the only global-memory latency left is hidden;
//  * the halo intensities of the plane being computed (ghosts on the domain
//    faces) are fetched the same way for the next step;
//  * rows of neighbouring strips are read directly from their CTAs' shared
//    memory (DSMEM), so each plane costs one cluster barrier.


template <typename T, int SEG, int SU, int SV>
__device__ __forceinline__ void pipe_update(const AngleParam<T> &p, const T *__restrict__ Irow,
                                            const T *__restrict__ Ivrow, T *__restrict__ Iout, int ncell,
                                            const T (&cm)[SEG + 2], const T (&c0)[SEG + 2],
                                            const T (&cp)[SEG + 2], const T (&sm)[SEG + 2],
                                            const T (&s0)[SEG + 2], const T (&sp)[SEG + 2],
                                            const T (&chi0)[SEG], const T (&S0)[SEG], T (&out)[SEG]) {
  // Irow / Ivrow point at column X0 + u0 of rows v and v - SV of the upwind plane
  T Ia[SEG + 1], Iv[SEG + 1];
  const int cb = SU > 0 ? -1 : 0;
#pragma unroll
  for (int k = 0; k < SEG + 1; ++k) {
    Ia[k] = Irow[cb + k];
    Iv[k] = Ivrow[cb + k];
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int kA = j + (SU > 0 ? 1 : 0), kB = j + (SU > 0 ? 0 : 1);
    const int jA = j + 1, jB = j + 1 - SU;
    const T chiC = SV > 0 ? cm[jA] : cp[jA], chiD = SV > 0 ? cm[jB] : cp[jB];
    const T sC = SV > 0 ? sm[jA] : sp[jA], sD = SV > 0 ? sm[jB] : sp[jB];
    const T chim = p.wa * c0[jA] + p.wb * c0[jB] + p.wc * chiC + p.wd * chiD;
    const T Sm = p.wa * s0[jA] + p.wb * s0[jB] + p.wc * sC + p.wd * sD;
    const T Im = p.wa * Ia[kA] + p.wb * Ia[kB] + p.wc * Iv[kA] + p.wd * Iv[kB];
    const T dtau = (chim + chi0[j]) * p.hs;
    T E, psi0, om;
    seg_weights(dtau, E, psi0, om);
    out[j] = Sm + E * (Im - Sm) + psi0 * (S0[j] - Sm);
  }
  // a ragged last segment must not touch the halo column beyond the row
#pragma unroll
  for (int j = 0; j < SEG; ++j)
    if (j < ncell) Iout[j] = out[j];
}

// One staged row around a 4-cell segment, (u0-1 .. u0+4), without bank conflicts:
// one aligned 128-bit load per lane, neighbours by warp shuffle from the adjacent
// lanes (same row, adjacent segment) or, at row ends, by a scalar load.
__device__ __forceinline__ void vec_row(const float *rowp, bool haveL, bool haveR, float (&o)[6]) {
  const float4 q = *reinterpret_cast<const float4 *>(rowp);
  float l = __shfl_up_sync(0xffffffffu, q.w, 1);
  float r = __shfl_down_sync(0xffffffffu, q.x, 1);
  if (!haveL) l = rowp[-1];
  if (!haveR) r = rowp[4];
  o[0] = l; o[1] = q.x; o[2] = q.y; o[3] = q.z; o[4] = q.w; o[5] = r;
}

template <int SU, int SV>
__device__ __forceinline__ void vec_update(const AngleParam<float> &p, const float (&Ir)[6], const float (&Iw)[6],
                                           const float (&cm)[6], const float (&c0)[6], const float (&cp)[6],
                                           const float (&sm)[6], const float (&s0)[6], const float (&sp)[6],
                                           const float (&chi0)[4], const float (&S0)[4], float (&out)[4]) {
  // Ir, Iw: rows v and v - SV of the upwind plane, columns u0-1 .. u0+4
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int jA = j + 1, jB = j + 1 - SU;
    const float chiC = SV > 0 ? cm[jA] : cp[jA], chiD = SV > 0 ? cm[jB] : cp[jB];
    const float sC = SV > 0 ? sm[jA] : sp[jA], sD = SV > 0 ? sm[jB] : sp[jB];
    const float chim = p.wa * c0[jA] + p.wb * c0[jB] + p.wc * chiC + p.wd * chiD;
    const float Sm = p.wa * s0[jA] + p.wb * s0[jB] + p.wc * sC + p.wd * sD;
    const float Im = p.wa * Ir[jA] + p.wb * Ir[jB] + p.wc * Iw[jA] + p.wd * Iw[jB];
    const float dtau = (chim + chi0[j]) * p.hs;
    float E, psi0, om;
    seg_weights(dtau, E, psi0, om);
    out[j] = Sm + E * (Im - Sm) + psi0 * (S0[j] - Sm);
  }
}

// ------------------------------------------------ packed-pair update (float32)
// The vectorised pipelined sweep's formal-solution step without moments: a
// thread's four cells form two pairs, and every per-cell operation of Eq. 20
// (interpolants, dtau, segment weights, the intensity update, the J sum) runs
// on a pair with one packed-FP32 instruction (f32x2).  The pairs of the cell's
// own column on a row are aligned register pairs of the row's 128-bit load; the
// upwind-column values (offset by the sign of mu_u) enter by scalar FMAs.

// One staged row around a 4-cell segment: columns u0..u0+3 as two pairs, and
// the column before (l) or after (r) it, whichever the stencil needs.
struct Row4 {
  float2 a0, a1;
  float l, r;
};

template <int SU>
__device__ __forceinline__ void row4(unsigned addr, unsigned needL, unsigned needR, Row4 &o) {
  const float4 q = lds128(addr);
  o.a0 = make_float2(q.x, q.y);
  o.a1 = make_float2(q.z, q.w);
  if (SU > 0) {
    o.l = __shfl_up_sync(0xffffffffu, q.w, 1);
    lds32_if(o.l, addr - 4u, needL);   // first lane of a warp or first segment of a row
  } else {
    o.r = __shfl_down_sync(0xffffffffu, q.x, 1);
    lds32_if(o.r, addr + 16u, needR);
  }
}

// value of the upwind column (u - SU) for cell j of a segment (the row's cell
// j + 1 - SU in the order l, a0.x, a0.y, a1.x, a1.y, r)
template <int SU>
__device__ __forceinline__ float upcol(const Row4 &o, int j) {
  if (SU > 0) return j == 0 ? o.l : (j == 1 ? o.a0.x : (j == 2 ? o.a0.y : o.a1.x));
  return j == 0 ? o.a0.y : (j == 1 ? o.a1.x : (j == 2 ? o.a1.y : o.r));
}

// bilinear interpolant of one cell pair (cells 2h, 2h+1): w = {wa, wa, wb, wb},
// v = {wc, wc, wd, wd}; rows X (own row) and Y (row v - SV)
template <int SU>
__device__ __forceinline__ float2 bilin2(const float4 &w, const float4 &v, const Row4 &X, const Row4 &Y, int h) {
  const float2 xa = h ? X.a1 : X.a0, ya = h ? Y.a1 : Y.a0;
  float2 m = __fmul2_rn(make_float2(w.x, w.y), xa);
  m = __ffma2_rn(make_float2(v.x, v.y), ya, m);
  m.x = fmaf(w.z, upcol<SU>(X, 2 * h), m.x);
  m.y = fmaf(w.z, upcol<SU>(X, 2 * h + 1), m.y);
  m.x = fmaf(v.z, upcol<SU>(Y, 2 * h), m.x);
  m.y = fmaf(v.z, upcol<SU>(Y, 2 * h + 1), m.y);
  return m;
}

// E = e^-x and Psi0 = 1 - (1 - E)/x of a pair.  Below x = 1/2 Psi0 is
// x (c0 + c1 x + ... + c4 x^4), a polynomial fitted to Psi0/x on [0, 1/2] by
// minimising the largest error (about 6e-9 absolute in Psi0, under float32
// resolution; the Taylor series needs eight terms for the same); above it the
// direct form, whose error (that of the exponential over x) is then below 3e-7.
// Constants enter through scalar instructions (they take immediate operands,
// the packed ones do not).
__device__ __forceinline__ void seg_weights2(float2 x, float2 &E, float2 &psi0) {
  E.x = ex2_approx(x.x * -1.4426950408889634f);
  E.y = ex2_approx(x.y * -1.4426950408889634f);
  float px = fmaf(x.x, 0.0011282316f, -0.0081961248f), py = fmaf(x.y, 0.0011282316f, -0.0081961248f);
  px = fmaf(x.x, px, 0.041633245f); py = fmaf(x.y, py, 0.041633245f);
  px = fmaf(x.x, px, -0.16666308f); py = fmaf(x.y, py, -0.16666308f);
  px = fmaf(x.x, px, 0.49999988f); py = fmaf(x.y, py, 0.49999988f);
  const float2 small = __fmul2_rn(x, make_float2(px, py));
  const float2 e0 = make_float2(1.f - E.x, 1.f - E.y);
  const float2 q = __fmul2_rn(e0, make_float2(rcp_approx(x.x), rcp_approx(x.y)));
  psi0.x = x.x < 0.5f ? small.x : 1.f - q.x;
  psi0.y = x.y < 0.5f ? small.y : 1.f - q.y;
}

// One cluster's (group, frequency) instance `inst` of the grid described by A
// (blockIdx.x % A.cluster is the CTA's strip).
template <typename T, int AMAX, bool MOM, int SEG, bool VEC>
__device__ __forceinline__ void pipe_body(const SweepArgs<T> &A, const int inst) {
  if (A.skip_if_done && A.st->done) return;
  const int C = A.cluster;
  const int rank = blockIdx.x % C;
  const int gi = inst % A.ngroups;
  const int f = inst / A.ngroups;
  const GroupParam gp = A.grp[gi];
  if (A.gs_forward && gp.axis == A.gs_axis && gp.sa < 0) return;   // swept in the reverse phase
  if (gp.na > A.ray_slots) {
    if (threadIdx.x == 0) atomicCAS(&A.st->err, 0, 30);
    return;
  }
  int cax[3];
  plane_axes(gp.axis, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const int perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
            perW = pick3(A.d.periodic, cax[2]);
  const long long csu = canon_stride(A.d.n, cax[0]), csv = canon_stride(A.d.n, cax[1]),
                  csw = canon_stride(A.d.n, cax[2]);   // canonical strides of u, v, w
  const int v0 = (int)(((long long)rank * Nv) / C);
  const int v1 = (int)(((long long)(rank + 1) * Nv) / C);
  const int R = v1 - v0;
  const int Rmax = (Nv + C - 1) / C;
  const int W = pipe_row_len(Nu, SEG);
  const int RX = Rmax + 2;
  const int pb = RX * W;               // one staged plane
  const int ib = A.ray_slots * pb;     // one plane of every ray of the group
  const long long plane = (long long)Nu * Nv;
  const long long cells = A.d.cells;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ib = reinterpret_cast<T *>(smem_raw);   // [2][slots][RX][W]   intensities
  T *Cr = Ib + 2 * ib;                       // [3][RX][W]          chi ring
  T *Sr = Cr + 3 * pb;                       // [3][RX][W]          S ring
  T *Gpre = Sr + 3 * pb;                     // [2][slots][Rmax + Nu] lagged ghosts for the outflow pass
  const int gpl = Rmax + Nu;                 // one ray's prefetched u-face rows and v-face row
#ifdef RT_DEBUG_BOUNDS
  const long long smem_n = 2LL * ib + 6LL * pb;
#endif
  __shared__ AngleParam<T> P[AMAX];
  // the packed-pair path's ray constants: {wa, wa, wb, wb}, {wc, wc, wd, wd}, {hs, hs, wq, wq}
  __shared__ float4 P2[(VEC && !MOM) ? AMAX : 1][3];
  if (threadIdx.x < gp.na) {
    const AngleParam<T> q = A.ang[gp.a0 + threadIdx.x];
    P[threadIdx.x] = q;
    if constexpr (VEC && !MOM) {
      P2[threadIdx.x][0] = make_float4(q.wa, q.wa, q.wb, q.wb);
      P2[threadIdx.x][1] = make_float4(q.wc, q.wc, q.wd, q.wd);
      P2[threadIdx.x][2] = make_float4(q.hs, q.hs, q.wq, q.wq);
    }
  }

  const int fs = A.st->fs_count + A.parity_offset;
  const int prev = fs & 1;
  const T *Gp = A.G[prev];
  T *Gn = A.G[prev ^ 1];
  const bool inc = A.incremental && A.st->iter > 0;
  const bool emit = A.incremental && A.st->iter == 0;
  const T *Gsrc = inc ? A.Gd[prev] : Gp;
  T *Gdn = A.incremental ? A.Gd[prev ^ 1] : nullptr;
  const T *chiP = A.chiP[gp.axis] + (long long)f * cells;
  const T *SP = A.SP[gp.axis] + (long long)f * cells;
  T *Jout = A.Jpart + ((long long)gi * A.d.nf + f) * cells;
  const int sa = gp.sa;
  const int wlast = sa > 0 ? Nw - 1 : 0;
  const int na = gp.na;
  const int nseg = (Nu + SEG - 1) / SEG;
  const bool vec = (sizeof(T) == 4) && (Nu % 4 == 0);
  const bool top_edge = v0 == 0 && !perV;      // no strip and no periodic image below
  const bool bot_edge = v1 == Nv && !perV;
  cg::cluster_group cluster = cg::this_cluster();
  // intensity buffers of the strips above and below in the cluster (DSMEM); every
  // upwind read below is then a local shared-memory load
  T *Ntop0 = nullptr, *Nbot0 = nullptr;
  int top_row = 0;   // this strip's first row as the top neighbour's bottom halo row
  if (C > 1) {
    if (rank > 0) {
      Ntop0 = cluster.map_shared_rank(Ib, rank - 1);
      top_row = v0 - (int)(((long long)(rank - 1) * Nv) / C) + 1;
    }
    if (rank < C - 1) Nbot0 = cluster.map_shared_rank(Ib, rank + 1);
  }
  __syncthreads();

  // divisions of the per-plane work loops, by divisors fixed for the launch
  const FastDiv dq(vec ? Nu / 4 : Nu), dNu(Nu), drows(R + 2), d2rows(2 * (R + 2)), dR(R > 0 ? R : 1),
      dnrowNu((v0 == 0 ? 1 : 0) + (v1 == Nv ? 1 : 0) > 0 ? ((v0 == 0 ? 1 : 0) + (v1 == Nv ? 1 : 0)) * Nu : 1),
      dnseg(nseg);
  const bool vedge = v0 == 0 || v1 == Nv;   // this strip holds a v-face row of the domain

  // chi and S of plane wsrc (rows v0-1 .. v1, columns -1 .. Nu, wrapped or clamped) -> ring slot
  auto stage = [&](int wsrc, int slot) {
    T *Cd = Cr + slot * pb, *Sd = Sr + slot * pb;
    const int rows = R + 2;
    if (vec) {
      const int q = Nu / 4;
      for (int idx = threadIdx.x; idx < rows * q; idx += blockDim.x) {
        const int row = dq.div(idx), k = idx - row * q;
        int vv = v0 - 1 + row;
        vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
        const long long o = (long long)wsrc * plane + (long long)vv * Nu + 4 * k;
        cp_async16(Cd + RT_IDX(row * W + kPipeX0 + 4 * k, 6LL * pb, 43), chiP + o);
        cp_async16(Sd + RT_IDX(row * W + kPipeX0 + 4 * k, 6LL * pb, 43), SP + o);
      }
    } else {
      for (int idx = threadIdx.x; idx < rows * Nu; idx += blockDim.x) {
        const int row = dq.div(idx), u = idx - row * Nu;
        int vv = v0 - 1 + row;
        vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
        const long long o = (long long)wsrc * plane + (long long)vv * Nu + u;
        cp_async_elem(Cd + RT_IDX(row * W + kPipeX0 + u, 6LL * pb, 44), chiP + o);
        cp_async_elem(Sd + RT_IDX(row * W + kPipeX0 + u, 6LL * pb, 44), SP + o);
      }
    }
    for (int idx = threadIdx.x; idx < 2 * rows; idx += blockDim.x) {
      const int side = drows.div(idx), row = idx - side * rows;
      int vv = v0 - 1 + row;
      vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
      const int uu = side ? (perU ? 0 : Nu - 1) : (perU ? Nu - 1 : 0);
      const long long o = (long long)wsrc * plane + (long long)vv * Nu + uu;
      const int col = side ? kPipeX0 + Nu : kPipeX0 - 1;
      cp_async_elem(Cd + RT_IDX(row * W + col, 6LL * pb, 45), chiP + o);
      cp_async_elem(Sd + RT_IDX(row * W + col, 6LL * pb, 45), SP + o);
    }
  };
  // ghost intensities of plane wsrc around the strip: halo columns of every row,
  // and the halo rows on a domain face without a periodic image (whole plane if all)
  auto ghost_halo = [&](T *Ibuf, int wsrc, bool whole) {
    if (whole) {
      const int ext = (R + 2) * (Nu + 2);
      for (int idx = threadIdx.x; idx < na * ext; idx += blockDim.x) {
        const int a = idx / ext, r2 = idx - a * ext;
        const int row = r2 / (Nu + 2), col = r2 - row * (Nu + 2);
        ghost_async(Ibuf + RT_IDX(a * pb + row * W + kPipeX0 - 1 + col, 2LL * ib, 46),
                    ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, col - 1, v0 - 1 + row, wsrc));
      }
      return;
    }
    for (int idx = threadIdx.x; idx < na * 2 * (R + 2); idx += blockDim.x) {
      const int a = d2rows.div(idx), r2 = idx - a * 2 * (R + 2);
      const int side = drows.div(r2), row = r2 - side * (R + 2);
      const int vv = v0 - 1 + row;
      // a periodic u face with v inside the grid: the lagged ghost is the u-face
      // entry (w, v) of the ray's block (the general lookup gives the same address)
      const T *src = (perU && vv >= 0 && vv < Nv)
                         ? Gsrc + ((long long)f * A.na + P[a].angle) * A.d.gsize + plane + (long long)wsrc * Nv + vv
                         : ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, side ? Nu : -1, vv, wsrc);
      ghost_async(Ibuf + RT_IDX(a * pb + row * W + (side ? kPipeX0 + Nu : kPipeX0 - 1), 2LL * ib, 47), src);
    }
    const int nrow = (v0 == 0 ? 1 : 0) + (v1 == Nv ? 1 : 0);   // rows outside the domain in v
    for (int idx = threadIdx.x; idx < na * nrow * Nu; idx += blockDim.x) {
      const int a = dnrowNu.div(idx), r2 = idx - a * nrow * Nu;
      const int which = dNu.div(r2), u = r2 - which * Nu;
      const bool lo = (v0 == 0) && (which == 0);
      const int row = lo ? 0 : R + 1;
      // a periodic v face (u inside the grid): the v-face entry (w, u) of the ray's block
      const T *src = perV ? Gsrc + ((long long)f * A.na + P[a].angle) * A.d.gsize + plane + (long long)Nw * Nv +
                                (long long)wsrc * Nu + u
                          : ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gsrc, inc, u, lo ? -1 : Nv, wsrc);
      ghost_async(Ibuf + RT_IDX(a * pb + row * W + kPipeX0 + u, 2LL * ib, 48), src);
    }
  };

  // Outflow intensities of plane wp onto the periodic faces, for the next formal
  // solution (Sec. 3.5): the u face (one column per row), the v face (one row, in
  // the strip that holds it) and, at the last plane, the w face (the whole strip).
  // The incremental and increment-recording sweeps read the previous ghosts
  // where they write new ones; those values are fetched into shared memory one
  // plane step ahead (buffer buf), so the outflow pass does not wait on memory.
  const bool need_pre = A.write_ghosts && A.incremental;
  auto ghost_prefetch = [&](int wp, int buf) {
    if (!need_pre) return;
    T *dst = Gpre + (long long)buf * A.ray_slots * gpl;
    if (perU) {
      for (int idx = threadIdx.x; idx < na * R; idx += blockDim.x) {
        const int a = dR.div(idx), lv = idx - a * R;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        cp_async_elem(dst + a * gpl + lv, Gp + gb + plane + (long long)wp * Nv + v0 + lv);
      }
    }
    if (perV && vedge) {
      for (int idx = threadIdx.x; idx < na * Nu; idx += blockDim.x) {
        const int a = dNu.div(idx), u = idx - a * Nu;
        const int vr = P[a].sv > 0 ? Nv - 1 : 0;
        if (vr < v0 || vr >= v1) continue;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        cp_async_elem(dst + a * gpl + Rmax + u, Gp + gb + plane + (long long)Nw * Nv + (long long)wp * Nu + u);
      }
    }
  };
  // store with the previous ghost value taken from the prefetch buffer
  auto store_pre = [&](long long off, T I0, T pre) {
    if (inc) {
      Gdn[off] = I0;
      Gn[off] = pre + I0;
    } else {
      if (emit) Gdn[off] = I0 - pre;
      Gn[off] = I0;
    }
  };
  auto ghost_pass = [&](const T *Ibuf, int wp, int buf) {
    if (!A.write_ghosts) return;
    const long long gn = (long long)A.d.nf * A.na * A.d.gsize;
    const T *pre = Gpre + (long long)buf * A.ray_slots * gpl;
    if (perU) {
      for (int idx = threadIdx.x; idx < na * R; idx += blockDim.x) {
        const int a = dR.div(idx), lv = idx - a * R;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        const int col = P[a].su > 0 ? Nu - 1 : 0;
        const long long off = RT_IDX(gb + plane + (long long)wp * Nv + v0 + lv, gn, 54);
        const T I0 = Ibuf[RT_IDX(a * pb + (lv + 1) * W + kPipeX0 + col, 2LL * ib, 58)];
        if (need_pre) store_pre(off, I0, pre[a * gpl + lv]);
        else ghost_store<T>(Gp, Gn, Gdn, off, I0, inc, emit);
      }
    }
    if (perV && vedge) {
      for (int idx = threadIdx.x; idx < na * Nu; idx += blockDim.x) {
        const int a = dNu.div(idx), u = idx - a * Nu;
        const int vr = P[a].sv > 0 ? Nv - 1 : 0;
        if (vr < v0 || vr >= v1) continue;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        const long long off = RT_IDX(gb + plane + (long long)Nw * Nv + (long long)wp * Nu + u, gn, 55);
        const T I0 = Ibuf[RT_IDX(a * pb + (vr - v0 + 1) * W + kPipeX0 + u, 2LL * ib, 59)];
        if (need_pre) store_pre(off, I0, pre[a * gpl + Rmax + u]);
        else ghost_store<T>(Gp, Gn, Gdn, off, I0, inc, emit);
      }
    }
    if (perW && wp == wlast) {
      for (int idx = threadIdx.x; idx < na * R * Nu; idx += blockDim.x) {
        const int a = idx / (R * Nu), r2 = idx - a * R * Nu;
        const int lv = r2 / Nu, u = r2 - lv * Nu;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        ghost_store<T>(Gp, Gn, Gdn, RT_IDX(gb + (long long)(v0 + lv) * Nu + u, gn, 53),
                       Ibuf[RT_IDX(a * pb + (lv + 1) * W + kPipeX0 + u, 2LL * ib, 60)], inc, emit);
      }
    }
  };

  // prologue: the first plane, the upwind ghost plane, and its intensities
  const int w0 = sa > 0 ? 0 : Nw - 1;
  stage(w0, 0);
  stage(perW ? (sa > 0 ? Nw - 1 : 0) : w0, 2);
  ghost_halo(Ib + ib, w0 - sa, true);
  cp_async_commit();
  cp_async_wait_all();
  if (C > 1) cluster.sync();
  else __syncthreads();
  // asynchronous loads a plane step issues for later steps: the next plane's chi
  // and S, and the halo ghosts of this plane's intensities (the next upwind plane)
  auto issue = [&](int tt) {
    const int ww = sa > 0 ? tt : Nw - 1 - tt;
    if (tt + 1 < Nw) stage(ww + sa, (tt + 1) % 3);
    ghost_halo(Ib + (tt & 1) * ib, ww, false);
    ghost_prefetch(ww, tt & 1);   // for this plane's outflow pass, one step later
    cp_async_commit();
  };
  issue(0);

  // packed-pair path: each task's J partials are stored at the end of the
  // thread's next task, and its last task's of a plane after the plane's cluster
  // barrier, so that the barrier's release does not wait for their global
  // writes (they drain during the next task or plane)
  const bool defer = VEC && !MOM;
  const bool jxl = VEC && !MOM && A.jx && gp.axis == 0;   // partials in this group's plane layout
  float4 Jpend = make_float4(0.f, 0.f, 0.f, 0.f);
  long long cpend = -1;
  auto flush_J = [&]() {
    if (cpend < 0) return;
    float *Jf = reinterpret_cast<float *>(Jout);
    if (csu == 1 || jxl) {
      *reinterpret_cast<float4 *>(Jf + RT_IDX(cpend, cells, 56)) = Jpend;
    } else {
      Jf[RT_IDX(cpend, cells, 57)] = Jpend.x;
      Jf[RT_IDX(cpend + csu, cells, 57)] = Jpend.y;
      Jf[RT_IDX(cpend + 2 * csu, cells, 57)] = Jpend.z;
      Jf[RT_IDX(cpend + 3 * csu, cells, 57)] = Jpend.w;
    }
    cpend = -1;
  };

  for (int t = 0; t < Nw; ++t) {
    const int w = sa > 0 ? t : Nw - 1 - t;
    T *Icur = Ib + (t & 1) * ib;
    const T *Iprv = Ib + ((t + 1) & 1) * ib;
    const T *Cc = Cr + (t % 3) * pb, *Cp = Cr + ((t + 2) % 3) * pb;
    const T *Sc = Sr + (t % 3) * pb, *Sp = Sr + ((t + 2) % 3) * pb;
    // this plane's buffers of the neighbouring strips: the first and last rows of
    // the strip are also stored into their halo rows (read there as the upwind
    // plane of the next step, after the cluster barrier)
    T *Ntop = Ntop0 ? Ntop0 + (t & 1) * ib + top_row * W + kPipeX0 : nullptr;
    T *Nbot = Nbot0 ? Nbot0 + (t & 1) * ib + kPipeX0 : nullptr;
    if constexpr (VEC && !MOM) {
      // packed pairs, every shared-memory access by 32-bit address
      if (defer) {
        flush_J();                                   // the previous plane's J partials
        if (t > 0) ghost_pass(Iprv, w - sa, (t + 1) & 1);   // and its outflow ghosts
      }
      const int ntask = R * nseg;
      const int lane = threadIdx.x & 31;
      const unsigned sb = smem_addr(smem_raw);
      const unsigned pb4 = (unsigned)pb * 4u, W4 = (unsigned)W * 4u;
      const unsigned sIprv = sb + (unsigned)(((t + 1) & 1) * ib) * 4u;
      const unsigned sIcur = sb + (unsigned)((t & 1) * ib) * 4u;
      const unsigned sCp = sb + (unsigned)(2 * ib + ((t + 2) % 3) * pb) * 4u;
      const unsigned sCc = sb + (unsigned)(2 * ib + (t % 3) * pb) * 4u;
      const unsigned sSp = sb + (unsigned)(2 * ib + 3 * pb + ((t + 2) % 3) * pb) * 4u;
      const unsigned sSc = sb + (unsigned)(2 * ib + 3 * pb + (t % 3) * pb) * 4u;
      // this plane's halo rows of the neighbouring strips, in their shared memory
      const unsigned rTop = Ntop0 ? mapa_rank(sIcur + (unsigned)(top_row * W + kPipeX0) * 4u, rank - 1) : 0u;
      const unsigned rBot = Nbot0 ? mapa_rank(sIcur + (unsigned)kPipeX0 * 4u, rank + 1) : 0u;
      for (int base = threadIdx.x - lane; base < ntask; base += blockDim.x) {
        const int sidx = base + lane;
        const bool active = sidx < ntask;
        const int sc = active ? sidx : ntask - 1;
        const int lv = dnseg.div(sc), seg = sc - lv * nseg;
        const int u0 = seg * 4, v = v0 + lv, row = lv + 1;
        const unsigned needL = !(active && seg > 0 && lane > 0);
        const unsigned needR = !(active && seg < nseg - 1 && lane < 31 && sidx + 1 < ntask);
        const unsigned ro = (unsigned)(row * W + kPipeX0 + u0) * 4u;
        const bool pushTop = active && lv == 0 && Ntop0 != nullptr;
        const bool pushBot = active && lv == R - 1 && Nbot0 != nullptr;
        // chi and S of the upwind plane, rows v-1, v, v+1 (both stencil sides: the
        // rays' signs of mu_u differ within the group)
        Row4 cm, c0, cp, sm, s0, sp;
        {
          const float4 q = lds128(sCp + ro - W4);
          cm.a0 = make_float2(q.x, q.y); cm.a1 = make_float2(q.z, q.w);
          cm.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(cm.l, sCp + ro - W4 - 4u, needL);
          cm.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(cm.r, sCp + ro - W4 + 16u, needR);
        }
        {
          const float4 q = lds128(sCp + ro);
          c0.a0 = make_float2(q.x, q.y); c0.a1 = make_float2(q.z, q.w);
          c0.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(c0.l, sCp + ro - 4u, needL);
          c0.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(c0.r, sCp + ro + 16u, needR);
        }
        {
          const float4 q = lds128(sCp + ro + W4);
          cp.a0 = make_float2(q.x, q.y); cp.a1 = make_float2(q.z, q.w);
          cp.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(cp.l, sCp + ro + W4 - 4u, needL);
          cp.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(cp.r, sCp + ro + W4 + 16u, needR);
        }
        {
          const float4 q = lds128(sSp + ro - W4);
          sm.a0 = make_float2(q.x, q.y); sm.a1 = make_float2(q.z, q.w);
          sm.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(sm.l, sSp + ro - W4 - 4u, needL);
          sm.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(sm.r, sSp + ro - W4 + 16u, needR);
        }
        {
          const float4 q = lds128(sSp + ro);
          s0.a0 = make_float2(q.x, q.y); s0.a1 = make_float2(q.z, q.w);
          s0.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(s0.l, sSp + ro - 4u, needL);
          s0.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(s0.r, sSp + ro + 16u, needR);
        }
        {
          const float4 q = lds128(sSp + ro + W4);
          sp.a0 = make_float2(q.x, q.y); sp.a1 = make_float2(q.z, q.w);
          sp.l = __shfl_up_sync(0xffffffffu, q.w, 1); lds32_if(sp.l, sSp + ro + W4 - 4u, needL);
          sp.r = __shfl_down_sync(0xffffffffu, q.x, 1); lds32_if(sp.r, sSp + ro + W4 + 16u, needR);
        }
        const float4 q0 = lds128(sCc + ro), r0 = lds128(sSc + ro);
        const float2 chi0[2] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w)};
        const float2 S0[2] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w)};
        float2 Jp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        auto ray = [&](auto su_c, auto sv_c, int a) {
          constexpr int SU = decltype(su_c)::value, SV = decltype(sv_c)::value;
          const float4 wab = P2[a][0], wcd = P2[a][1], hq = P2[a][2];
          const unsigned ia = sIprv + (unsigned)a * pb4 + ro;
          Row4 Ir, Iw;
          row4<SU>(ia, needL, needR, Ir);
          row4<SU>(SV > 0 ? ia - W4 : ia + W4, needL, needR, Iw);   // halo rows hold the neighbours' rows
          const Row4 &cY = SV > 0 ? cm : cp;
          const Row4 &sY = SV > 0 ? sm : sp;
          float2 o[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 chim = bilin2<SU>(wab, wcd, c0, cY, h);
            const float2 Sm = bilin2<SU>(wab, wcd, s0, sY, h);
            const float2 Im = bilin2<SU>(wab, wcd, Ir, Iw, h);
            const float2 dtau = __fmul2_rn(__fadd2_rn(chim, chi0[h]), make_float2(hq.x, hq.y));
            float2 E, psi0;
            seg_weights2(dtau, E, psi0);
            // I0 = S- + E (I- - S-) + Psi0 (S0 - S-)
            const float2 d1 = make_float2(Im.x - Sm.x, Im.y - Sm.y);
            const float2 d2 = make_float2(S0[h].x - Sm.x, S0[h].y - Sm.y);
            float2 I0 = __ffma2_rn(E, d1, Sm);
            I0 = __ffma2_rn(psi0, d2, I0);
            o[h] = I0;
            Jp[h] = __ffma2_rn(make_float2(hq.z, hq.w), I0, Jp[h]);
          }
          const float4 o4 = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
          const unsigned ao = (unsigned)a * pb4;
          if (active) sts128(sIcur + ao + ro, o4);
          if (pushTop) stc128(rTop + ao + (unsigned)u0 * 4u, o4);
          if (pushBot) stc128(rBot + ao + (unsigned)u0 * 4u, o4);
        };
        auto block = [&](auto su_c, auto sv_c, int k0, int kn) {
#pragma unroll 2
          for (int q = 0; q < kn; ++q) ray(su_c, sv_c, k0 + q);
        };
        block(SignC<-1>{}, SignC<-1>{}, gp.kb[0], gp.kb[1] - gp.kb[0]);
        block(SignC<1>{}, SignC<-1>{}, gp.kb[1], gp.kb[2] - gp.kb[1]);
        block(SignC<-1>{}, SignC<1>{}, gp.kb[2], gp.kb[3] - gp.kb[2]);
        block(SignC<1>{}, SignC<1>{}, gp.kb[3], gp.kb[4] - gp.kb[3]);
        if (active) {
          flush_J();   // the thread's previous task of this plane, if any
          Jpend = make_float4(Jp[0].x, Jp[0].y, Jp[1].x, Jp[1].y);
          cpend = jxl ? (long long)u0 + (long long)v * Nu + (long long)w * plane
                      : (long long)(u0) * csu + (long long)v * csv + (long long)w * csw;
        }
      }
    } else if constexpr (VEC) {
      // float32 rows whose length is a multiple of 4: one segment per lane, a
      // warp-uniform trip count so every shuffle has the whole warp
      const int ntask = R * nseg;
      const int lane = threadIdx.x & 31;
      const long long ustride = csu;
      for (int base = threadIdx.x - lane; base < ntask; base += blockDim.x) {
        const int sidx = base + lane;
        const bool active = sidx < ntask;
        const int sc = active ? sidx : ntask - 1;
        const int lv = dnseg.div(sc), seg = sc - lv * nseg;
        const int u0 = seg * 4, v = v0 + lv, row = lv + 1;
        const bool haveL = active && seg > 0 && lane > 0;
        const bool haveR = active && seg < nseg - 1 && lane < 31 && sidx + 1 < ntask;
        float cm[6], c0[6], cp[6], sm[6], s0[6], sp[6];
        const float *Cpr = reinterpret_cast<const float *>(Cp) + row * W + kPipeX0 + u0;
        const float *Spr = reinterpret_cast<const float *>(Sp) + row * W + kPipeX0 + u0;
        vec_row(Cpr - W, haveL, haveR, cm);
        vec_row(Cpr, haveL, haveR, c0);
        vec_row(Cpr + W, haveL, haveR, cp);
        vec_row(Spr - W, haveL, haveR, sm);
        vec_row(Spr, haveL, haveR, s0);
        vec_row(Spr + W, haveL, haveR, sp);
        const float4 q0 = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(Cc) + row * W + kPipeX0 + u0);
        const float4 r0 = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(Sc) + row * W + kPipeX0 + u0);
        const float chi0[4] = {q0.x, q0.y, q0.z, q0.w};
        const float S0[4] = {r0.x, r0.y, r0.z, r0.w};
        float Jacc[4] = {0.f, 0.f, 0.f, 0.f};
        float Hm[MOM ? 4 : 1][3], Km[MOM ? 4 : 1][6];
        if (MOM) {
#pragma unroll
          for (int j = 0; j < (MOM ? 4 : 1); ++j) {
#pragma unroll
            for (int q = 0; q < 3; ++q) Hm[j][q] = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) Km[j][q] = 0.f;
          }
        }
        // one ray of the group; the signs of mu_u, mu_v are compile-time, so a block
        // of rays with the same signs is straight-line code
        auto ray = [&](auto su_c, auto sv_c, int a) {
          constexpr int SU = decltype(su_c)::value, SV = decltype(sv_c)::value;
          // the ray's constants in three 128-bit shared loads
          AngleParam<float> p;
          {
            const float4 *pv = reinterpret_cast<const float4 *>(&P[a]);
            const float4 x0 = pv[0], x1 = pv[1], x2 = pv[2];
            p.wa = x0.x; p.wb = x0.y; p.wc = x0.z; p.wd = x0.w;
            p.hs = x1.x; p.wq = x1.y; p.mu[0] = x1.z; p.mu[1] = x1.w;
            p.mu[2] = x2.x;
          }
          const float *Ia = reinterpret_cast<const float *>(Iprv) + a * pb + row * W + kPipeX0 + u0;
          const float *Iv = SV > 0 ? Ia - W : Ia + W;   // halo rows hold the neighbours' rows
          float Ir[6], Iw[6], I0[4];
          vec_row(Ia, haveL, haveR, Ir);
          vec_row(Iv, haveL, haveR, Iw);
          vec_update<SU, SV>(p, Ir, Iw, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
          if (active) {
            const float4 o4 = make_float4(I0[0], I0[1], I0[2], I0[3]);
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(Icur) + a * pb + row * W + kPipeX0 + u0) = o4;
            if (lv == 0 && Ntop) *reinterpret_cast<float4 *>(reinterpret_cast<float *>(Ntop) + a * pb + u0) = o4;
            if (lv == R - 1 && Nbot) *reinterpret_cast<float4 *>(reinterpret_cast<float *>(Nbot) + a * pb + u0) = o4;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float wI = p.wq * I0[j];
            Jacc[j] += wI;
            if (MOM) {
              Hm[MOM ? j : 0][0] += wI * p.mu[0];
              Hm[MOM ? j : 0][1] += wI * p.mu[1];
              Hm[MOM ? j : 0][2] += wI * p.mu[2];
              Km[MOM ? j : 0][0] += wI * p.mu[0] * p.mu[0];
              Km[MOM ? j : 0][1] += wI * p.mu[1] * p.mu[1];
              Km[MOM ? j : 0][2] += wI * p.mu[2] * p.mu[2];
              Km[MOM ? j : 0][3] += wI * p.mu[0] * p.mu[1];
              Km[MOM ? j : 0][4] += wI * p.mu[0] * p.mu[2];
              Km[MOM ? j : 0][5] += wI * p.mu[1] * p.mu[2];
            }
          }
        };
        // a short unroll: fully unrolled blocks (4 x AMAX ray bodies) overflow the
        // instruction cache; two bodies per trip keep some overlap between rays
        auto block = [&](auto su_c, auto sv_c, int k0, int kn) {
#pragma unroll 2
          for (int q = 0; q < kn; ++q) ray(su_c, sv_c, k0 + q);
        };
        block(SignC<-1>{}, SignC<-1>{}, gp.kb[0], gp.kb[1] - gp.kb[0]);
        block(SignC<1>{}, SignC<-1>{}, gp.kb[1], gp.kb[2] - gp.kb[1]);
        block(SignC<-1>{}, SignC<1>{}, gp.kb[2], gp.kb[3] - gp.kb[2]);
        block(SignC<1>{}, SignC<1>{}, gp.kb[3], gp.kb[4] - gp.kb[3]);
        if (active) {
          const long long canon = (long long)(u0) * csu + (long long)v * csv + (long long)w * csw;
          float *Jf = reinterpret_cast<float *>(Jout);
          if (ustride == 1) {
            *reinterpret_cast<float4 *>(Jf + RT_IDX(canon, cells, 56)) = make_float4(Jacc[0], Jacc[1], Jacc[2], Jacc[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) Jf[RT_IDX(canon + (long long)j * ustride, cells, 57)] = Jacc[j];
          }
          if (MOM) {
            T *M = A.Mpart + (long long)gi * 9 * A.d.nf * cells;
            const long long qs = (long long)A.d.nf * cells;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const long long o = (long long)f * cells + canon + (long long)j * ustride;
#pragma unroll
              for (int q = 0; q < 3; ++q) M[q * qs + o] = (T)Hm[MOM ? j : 0][q];
#pragma unroll
              for (int q = 0; q < 6; ++q) M[(3 + q) * qs + o] = (T)Km[MOM ? j : 0][q];
            }
          }
        }
      }
    } else {
      for (int sidx = threadIdx.x; sidx < R * nseg; sidx += blockDim.x) {
        const int lv = dnseg.div(sidx), seg = sidx - lv * nseg;
        const int u0 = seg * SEG, v = v0 + lv, row = lv + 1;
        const int ncell = min(SEG, Nu - u0);
        T cm[SEG + 2], c0[SEG + 2], cp[SEG + 2], sm[SEG + 2], s0[SEG + 2], sp[SEG + 2];
  #pragma unroll
        for (int j = 0; j < SEG + 2; ++j) {
          const int col = kPipeX0 - 1 + u0 + j;
          cm[j] = Cp[(row - 1) * W + col];
          c0[j] = Cp[row * W + col];
          cp[j] = Cp[(row + 1) * W + col];
          sm[j] = Sp[(row - 1) * W + col];
          s0[j] = Sp[row * W + col];
          sp[j] = Sp[(row + 1) * W + col];
        }
        T chi0[SEG], S0[SEG], Jacc[SEG];
        T Hm[MOM ? SEG : 1][3], Km[MOM ? SEG : 1][6];
  #pragma unroll
        for (int j = 0; j < SEG; ++j) {
          chi0[j] = Cc[row * W + kPipeX0 + u0 + j];
          S0[j] = Sc[row * W + kPipeX0 + u0 + j];
          Jacc[j] = T(0);
          if (MOM) {
  #pragma unroll
            for (int q = 0; q < 3; ++q) Hm[MOM ? j : 0][q] = T(0);
  #pragma unroll
            for (int q = 0; q < 6; ++q) Km[MOM ? j : 0][q] = T(0);
          }
        }
        auto ray = [&](auto su_c, auto sv_c, int a) {
          constexpr int SU = decltype(su_c)::value, SV = decltype(sv_c)::value;
          const AngleParam<T> &p = P[a];
          const T *Ia = Iprv + a * pb + row * W + kPipeX0 + u0;
          T *Io = Icur + a * pb + row * W + kPipeX0 + u0;
          const T *Iv = SV > 0 ? Ia - W : Ia + W;   // halo rows hold the neighbours' rows
          T I0[SEG];
          pipe_update<T, SEG, SU, SV>(p, Ia, Iv, Io, ncell, cm, c0, cp, sm, s0, sp, chi0, S0, I0);
          if (lv == 0 && Ntop) {
  #pragma unroll
            for (int j = 0; j < SEG; ++j)
              if (j < ncell) Ntop[a * pb + u0 + j] = I0[j];
          }
          if (lv == R - 1 && Nbot) {
  #pragma unroll
            for (int j = 0; j < SEG; ++j)
              if (j < ncell) Nbot[a * pb + u0 + j] = I0[j];
          }
  #pragma unroll
          for (int j = 0; j < SEG; ++j) {
            const T wI = p.wq * I0[j];
            Jacc[j] += wI;
            if (MOM) {
              Hm[MOM ? j : 0][0] += wI * p.mu[0];
              Hm[MOM ? j : 0][1] += wI * p.mu[1];
              Hm[MOM ? j : 0][2] += wI * p.mu[2];
              Km[MOM ? j : 0][0] += wI * p.mu[0] * p.mu[0];
              Km[MOM ? j : 0][1] += wI * p.mu[1] * p.mu[1];
              Km[MOM ? j : 0][2] += wI * p.mu[2] * p.mu[2];
              Km[MOM ? j : 0][3] += wI * p.mu[0] * p.mu[1];
              Km[MOM ? j : 0][4] += wI * p.mu[0] * p.mu[2];
              Km[MOM ? j : 0][5] += wI * p.mu[1] * p.mu[2];
            }
          }
        };
        auto block = [&](auto su_c, auto sv_c, int k0, int kn) {
  #pragma unroll 2
          for (int q = 0; q < kn; ++q) ray(su_c, sv_c, k0 + q);
        };
        block(SignC<-1>{}, SignC<-1>{}, gp.kb[0], gp.kb[1] - gp.kb[0]);
        block(SignC<1>{}, SignC<-1>{}, gp.kb[1], gp.kb[2] - gp.kb[1]);
        block(SignC<-1>{}, SignC<1>{}, gp.kb[2], gp.kb[3] - gp.kb[2]);
        block(SignC<1>{}, SignC<1>{}, gp.kb[3], gp.kb[4] - gp.kb[3]);
  #pragma unroll
        for (int j = 0; j < SEG; ++j) {
          if (j < ncell) {
            const long long canon = (long long)(u0 + j) * csu + (long long)v * csv + (long long)w * csw;
            Jout[RT_IDX(canon, cells, 52)] = Jacc[j];
            if (MOM) {
              T *M = A.Mpart + (long long)gi * 9 * A.d.nf * cells;
              const long long qs = (long long)A.d.nf * cells;
              const long long o = (long long)f * cells + canon;
  #pragma unroll
              for (int q = 0; q < 3; ++q) M[q * qs + o] = Hm[MOM ? j : 0][q];
  #pragma unroll
              for (int q = 0; q < 6; ++q) M[(3 + q) * qs + o] = Km[MOM ? j : 0][q];
            }
          }
        }
      }
    }
    // outflow ghosts of the previous plane, read from its (still intact) buffer
    if (t > 0 && !defer) ghost_pass(Iprv, w - sa, (t + 1) & 1);
    cp_async_wait_all();
    // the CTA is done with the chi/S slot and the halo columns the next issue
    // refills; the cluster barrier (strip edges pushed to the neighbours) is
    // split around that issue so its latency overlaps the copies' set-up
    __syncthreads();
    if (C > 1) {
      cluster.barrier_arrive();
      if (t + 1 < Nw) issue(t + 1);
      cluster.barrier_wait();
    } else if (t + 1 < Nw) {
      issue(t + 1);
    }
  }
  flush_J();
  ghost_pass(Ib + ((Nw - 1) & 1) * ib, sa > 0 ? Nw - 1 : 0, (Nw - 1) & 1);
  (void)top_edge;
  (void)bot_edge;
}

template <typename T, int AMAX, bool MOM, int SEG, bool VEC>
__global__ void __launch_bounds__(sweep_max_threads<T>()) sc_sweep_pipe_kernel(const __grid_constant__ SweepArgs<T> A) {
  pipe_body<T, AMAX, MOM, SEG, VEC>(A, blockIdx.x / A.cluster);
}

// The sweeps of several grids in one launch (the request server's shared
// launches): clusters [base[k], base[k+1]) run grid k's instances.  Every grid
// has the same cluster size; the launch's CTA size and shared memory are the
// largest of the grids' (the per-plane loops stride by blockDim).
template <typename T, int AMAX, int SEG, bool VEC>
__global__ void __launch_bounds__(sweep_max_threads<T>()) sc_sweep_multi_kernel(const __grid_constant__ MultiSweep<T> M) {
  const int c = blockIdx.x / M.a[0].cluster;
  int k = 0;
  while (k + 1 < M.n && c >= M.base[k + 1]) ++k;
  pipe_body<T, AMAX, false, SEG, VEC>(M.a[k], c - M.base[k]);
}

// --------------------------------------------------------------------- ALI update

__device__ __forceinline__ double rel_change(double d, double x) {
  const double ad = fabs(d), ax = fabs(x);
  return ax > 0.0 ? ad / ax : (ad > 0.0 ? INFINITY : 0.0);
}

__device__ __forceinline__ void block_max_to(double r, unsigned long long *dst) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = r;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0 && r > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(r));
  }
}

__device__ __forceinline__ long long perm_index(const Dims &d, int a, long long cell) {
  const int x = (int)(cell % d.n[0]);
  const int y = (int)((cell / d.n[0]) % d.n[1]);
  const int z = (int)(cell / ((long long)d.n[0] * d.n[1]));
  if (a == 2) return cell;
  if (a == 1) return ((long long)y * d.n[2] + z) * d.n[0] + x;   // [y][z][x]
  return ((long long)x * d.n[2] + z) * d.n[1] + y;                 // [x][z][y]
}

// Jacobi ALI (Eq. 24): dS = [(1-eps) J + eps B - S] / [1 - (1-eps) Lambda*], with
// the denominator formed as eps + (1-eps)(1 - Lambda*) from the separately summed
// 1 - Lambda* (no cancellation in thick cells).  All of it in FP64.
// A block owns a tile of 32 x 32 cells (x, y) of one z plane and frequency; the
// sweep copies of the new S (or of dS) are written x-contiguous for the y and z
// sweeps and through a shared-memory transpose, y-contiguous, for the x sweep.
constexpr int kAliTile = 32;
constexpr int kAliRows = 8;

template <typename T>
__global__ void __launch_bounds__(kAliTile * kAliRows) ali_update_kernel(const AliArgs<T> A) {
  if (A.st->done) return;
  __shared__ T tile[kAliTile][kAliTile + 1];
  const int nx = A.d.n[0], ny = A.d.n[1], nz = A.d.n[2];
  const int tx = threadIdx.x % kAliTile, ty = threadIdx.x / kAliTile;
  const int tiles_x = (nx + kAliTile - 1) / kAliTile;
  const int x0 = (blockIdx.x % tiles_x) * kAliTile, y0 = (blockIdx.x / tiles_x) * kAliTile;
  const int z = blockIdx.y, f = blockIdx.z;
  const long long cells = A.d.cells;
  const long long fbase = (long long)f * cells;
  const bool first = A.st->iter == 0;
  const bool inc = A.incremental && !first;
  const int x = x0 + tx;
  double rmax = 0.0;
  float rmaxf = 0.f;   // float32 sweeps: the maximum of the quantities taken in float32
  // float32 partials are summed exactly into a float pair (TwoSum) in group
  // order; those of the first nxg groups (sweeps along x) are in the [x][z][y]
  // layout and come through a shared-memory transpose of the tile
  if (A.fmask && A.fmask[f]) {   // this frequency is solved by another grid
    block_max_to(0.0, &A.st->resid_bits);
    return;
  }
  constexpr int KR = kAliTile / kAliRows;
  float xhi[KR], xlo[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) xhi[k] = xlo[k] = 0.f;
  if (sizeof(T) == 4 && A.Jpart && A.nxg > 0) {
    __shared__ float tJ[kAliTile][kAliTile + 1];
    for (int p = 0; p < A.nxg; ++p) {
      const float *src = reinterpret_cast<const float *>(A.Jpart) + ((long long)p * A.d.nf + f) * cells;
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const int xx = x0 + ty + k * kAliRows, yy = y0 + tx;
        tJ[ty + k * kAliRows][tx] = (xx < nx && yy < ny) ? src[((long long)xx * nz + z) * ny + yy] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const float v = tJ[tx][ty + k * kAliRows];
        const float s2 = xhi[k] + v;
        const float bp = s2 - xhi[k];
        xlo[k] += (xhi[k] - (s2 - bp)) + (v - bp);
        xhi[k] = s2;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int y = y0 + ty + k * kAliRows;
    T snew = T(0);
    if (x < nx && y < ny) {
      const long long c = ((long long)z * ny + y) * nx + x;
      const long long i = fbase + c;
      double dJ;
      if (!A.Jpart) {
        // the formal solution was done elsewhere (a mixed grid's FP64 first one):
        // its J is already in J64
        dJ = A.J64[i];
      } else if (sizeof(T) == 4) {
        // float32 partials summed exactly into a float pair (TwoSum), then one FP64
        // add: the result is the FP64 sum to ~1e-14 at FP32 cost
        float hi = xhi[k], lo = xlo[k];
#pragma unroll 4
        for (int p = A.nxg; p < A.ngroups_per_f; ++p) {
          const float x = (float)A.Jpart[(long long)p * A.d.nf * cells + i];
          const float s2 = hi + x;
          const float bp = s2 - hi;
          lo += (hi - (s2 - bp)) + (x - bp);
          hi = s2;
        }
        dJ = (double)hi + (double)lo;
      } else {
        dJ = 0.0;
#pragma unroll 4
        for (int p = 0; p < A.ngroups_per_f; ++p) dJ += (double)A.Jpart[(long long)p * A.d.nf * cells + i];
      }
      // incremental solves accumulate J in FP64 from the swept increments (an
      // FP64 iteration's J replaces the accumulated one)
      const double J = (inc && A.Jpart) ? A.J64[i] + dJ : dJ;
      double r;
      bool r64 = true;   // r holds this cell's quantity (else it went into rmaxf)
      if (A.lte) {
        const double Jp = A.incremental ? A.J64[i] : A.Jprev[i];
        r = first ? INFINITY : rel_change(inc ? dJ : J - Jp, J);
        A.Jprev[i] = J;
        snew = A.incremental ? T(0) : (T)A.S64[i];
      } else if (sizeof(T) == 4 && A.ia && !A.Opart) {
        // float32 sweeps: FP64 throughput is scarce on this part, so the update
        // is two FMAs with the per-medium factors ia = (1-e) iden, ib = e B iden,
        // and the stopping quantity is taken in float32 (within 1e-7 of it,
        // relative) unless S is outside the float32 normal range
        const double S = A.S64[i];
        const double dS = fma(A.ia[i], J, fma(-S, A.iden[i], A.ib[i]));
        const double Sn = S + dS;
        A.S64[i] = Sn;
        A.Sfs[i] = S;
        const float df = (float)dS, sf = fabsf((float)Sn);
        if (sf > 1e-30f && sf < 1e30f && fabsf(df) < 1e30f) {
          rmaxf = fmaxf(rmaxf, __fdividef(fabsf(df), sf));   // the running maximum in float32 too
          r = 0.0;
          r64 = false;
        } else {
          r = rel_change(dS, Sn);
        }
        snew = (T)(A.incremental ? df : (float)Sn);
      } else {
        const double S = A.S64[i], e = A.eps[i];
        double iden;
        if (A.Opart) {   // second-order sweeps: 1 - Lambda* of this formal solution
          double om = 0.0;
          for (int p = 0; p < A.ngroups_per_f; ++p) om += (double)A.Opart[(long long)p * A.d.nf * cells + i];
          iden = 1.0 / (e + (1.0 - e) * om);
        } else {
          iden = A.iden[i];
        }
        const double dS = ((1.0 - e) * J + e * A.B[i] - S) * iden;
        const double Sn = S + dS;
        A.S64[i] = Sn;
        A.Sfs[i] = S;
        // the float32 path takes the stopping quantity in float32 (within 1e-7 of
        // it, relative) unless S is outside the float32 normal range
        r = (sizeof(T) == 4 && fabs(Sn) > 1e-30 && fabs(Sn) < 1e30 && fabs(dS) < 1e30)
                ? (double)__fdividef((float)fabs(dS), (float)fabs(Sn))
                : rel_change(dS, Sn);
        snew = (T)(A.incremental ? dS : Sn);
      }
      A.J64[i] = J;
      if (r64) rmax = fmax(rmax, r);
      if (A.SP[2]) A.SP[2][i] = snew;                                                 // [z][y][x]
      if (A.SP[1]) A.SP[1][fbase + ((long long)y * nz + z) * nx + x] = snew;          // [y][z][x]
    }
    tile[ty + k * kAliRows][tx] = snew;
  }
  if (A.SP[0]) {                                                                      // [x][z][y]
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kAliTile / kAliRows; ++k) {
      const int xx = x0 + ty + k * kAliRows, yy = y0 + tx;
      if (xx < nx && yy < ny) A.SP[0][fbase + ((long long)xx * nz + z) * ny + yy] = tile[tx][ty + k * kAliRows];
    }
  }
  block_max_to(fmax(rmax, (double)rmaxf), &A.st->resid_bits);
}

// Lagged ghosts after an FP64 formal solution done for a float32 grid: the
// outflow Gout and, for the incremental sweeps that follow, its change against
// the ghosts Gin the solution started from.
__global__ void ghosts_from64_kernel(long long n, const double *Gout, const double *Gin, float *G, float *Gd) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    G[i] = (float)Gout[i];
    Gd[i] = (float)(Gout[i] - Gin[i]);
  }
}

__global__ void f32_to_f64_kernel(long long n, const float *src, double *dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// Jacobi denominator of Eq. 24, inverted once per medium: the update then
// multiplies instead of dividing in FP64 every iteration.
__global__ void inv_denominator_kernel(long long n, const double *eps, const double *oml, double *iden,
                                       const double *B, double *ia, double *ib) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = 1.0 / (eps[i] + (1.0 - eps[i]) * oml[i]);
    iden[i] = d;
    if (ia) {
      ia[i] = (1.0 - eps[i]) * d;
      ib[i] = eps[i] * B[i] * d;
    }
  }
}

// Convergence decision after one ALI iteration (single thread).
__global__ void finish_kernel(SolveState *st) {
  if (st->done) return;
  const double r = __longlong_as_double((long long)st->resid_bits);
  st->resid_bits = 0ULL;
  st->fs_count += 1;
  st->iter += 1;
  st->last_resid = r;
  if (r <= st->tol) {
    st->done = 1;
    st->converged = 1;
  } else if (st->iter >= st->max_iter) {
    st->done = 1;
  }
}

// Small state edits, in stream order.
__global__ void state_op_kernel(SolveState *st, int op, int a, double b, int c) {
  if (op == 0) {           // reset for a new ALI solve (and its error word)
    st->err = 0;
    st->err_info = 0;
    st->fs_count = 0;
    st->iter = 0;
    st->done = 0;
    st->converged = 0;
    st->max_iter = a;
    st->tol = b;
    st->lte = c;
    st->resid_bits = 0ULL;
    st->last_resid = INFINITY;
  } else if (op == 1) {    // one formal solution completed outside an ALI loop
    st->fs_count += 1;
  } else if (op == 2) {    // reset the ghost parity (ghosts re-initialised)
    st->fs_count = 0;
    st->done = 0;
  }
}

// ------------------------------------------------------------------- Lambda*
// Lambda*_ii = sum_k w_k Psi0_k(i) and 1 - Lambda*_ii = sum_k w_k (1 - Psi0_k(i)),
// from chi alone, with the sweep's precision T for the segment weights; the sums
// are FP64 (float32 grids: exact float pairs).  The rays' constants are staged in
// shared memory; each thread owns one cell and frequency.
template <typename T>
struct LstarRay {
  T w4[4];            // weights of the four upwind face vertices
  T hs;               // half the path length, s/2
  double w;           // quadrature weight
  signed char off[4][3];   // canonical offsets (x, y, z) of the four vertices
};
constexpr int kLstarChunk = 64;   // rays staged in shared memory at a time

template <typename T>
__global__ void __launch_bounds__(256) lstar_kernel(Dims d, const double *chi, const RayGeom *rays,
                                                    int na, double *lstar, double *oml,
                                                    const double *xchi_lo, const double *xchi_hi) {
  __shared__ LstarRay<T> R[kLstarChunk];
  const long long cells = d.cells;
  const long long N = cells * d.nf;
  const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
  const int px = d.periodic[0], py = d.periodic[1], pz = d.periodic[2];
  // every block walks the same cell range in the same chunks, so the barriers match
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long nloop = (N + stride - 1) / stride;
  for (long long it = 0; it < nloop; ++it) {
    const long long i = it * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool live = i < N;
    const long long f = live ? i / cells : 0, c = live ? i - f * cells : 0;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
    const double *chf = chi + f * cells;
    const T chi0 = live ? (T)chf[c] : T(0);
    // float32 sums kept exact as a float pair (TwoSum); FP64 sums directly
    T Lh = T(0), Ll = T(0), Oh = T(0), Ol = T(0);
    for (int k0 = 0; k0 < na; k0 += kLstarChunk) {
      const int nk = min(kLstarChunk, na - k0);
      __syncthreads();
      if (threadIdx.x < nk) {
        const RayGeom r = rays[k0 + threadIdx.x];
        LstarRay<T> q;
        const int ax = r.axis, b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
        const double f1 = b1 == 0 ? r.frac[0] : (b1 == 1 ? r.frac[1] : r.frac[2]);
        const double f2 = b2 == 0 ? r.frac[0] : (b2 == 1 ? r.frac[1] : r.frac[2]);
        for (int v = 0; v < 4; ++v) {
          const int d1 = v >> 1, d2 = v & 1;
          q.w4[v] = (T)((d1 ? f1 : 1.0 - f1) * (d2 ? f2 : 1.0 - f2));
          int o[3] = {0, 0, 0};
          o[ax] = -r.sgn[ax];
          o[b1] = -d1 * r.sgn[b1];
          o[b2] = -d2 * r.sgn[b2];
          for (int a = 0; a < 3; ++a) q.off[v][a] = (signed char)o[a];
        }
        q.hs = (T)(0.5 * r.s);
        q.w = r.w;
        R[threadIdx.x] = q;
      }
      __syncthreads();
      if (!live) continue;
      for (int k = 0; k < nk; ++k) {
        const LstarRay<T> &q = R[k];
        T chim = T(0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          int xx = x + q.off[v][0], yy = y + q.off[v][1], zz = z + q.off[v][2];
          xx = xx < 0 ? (px ? nx - 1 : 0) : (xx >= nx ? (px ? 0 : nx - 1) : xx);
          yy = yy < 0 ? (py ? ny - 1 : 0) : (yy >= ny ? (py ? 0 : ny - 1) : yy);
          // beyond a subdomain z face: the ghost layer's chi
          const double *xc = zz < 0 ? xchi_lo : (zz >= nz ? xchi_hi : nullptr);
          zz = zz < 0 ? (pz ? nz - 1 : 0) : (zz >= nz ? (pz ? 0 : nz - 1) : zz);
          chim += q.w4[v] * (T)(xc ? xc[(f * ny + yy) * nx + xx] : chf[((long long)zz * ny + yy) * nx + xx]);
        }
        const T dtau = (chim + chi0) * q.hs;
        T E, psi0, om;
        seg_weights(dtau, E, psi0, om);
        const T wl = (T)q.w * psi0, wo = (T)q.w * om;
        if (sizeof(T) == 4) {
          T s2 = Lh + wl, bp = s2 - Lh;
          Ll += (Lh - (s2 - bp)) + (wl - bp);
          Lh = s2;
          s2 = Oh + wo;
          bp = s2 - Oh;
          Ol += (Oh - (s2 - bp)) + (wo - bp);
          Oh = s2;
        } else {
          Lh += q.w * (double)psi0;
          Oh += q.w * (double)om;
        }
      }
    }
    if (live) {
      lstar[i] = (double)Lh + (double)Ll;
      oml[i] = (double)Oh + (double)Ol;
    }
  }
}

// ------------------------------------------------------------------- set-up kernels

// Counts inputs outside chi >= 0, 0 < eps <= 1, B >= 0 (or non-finite), and eps != 1.
__global__ void validate_kernel(long long n, const double *chi, const double *eps, const double *B,
                                int *counts) {
  int bad = 0, non1 = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double c = chi[i], e = eps[i], b = B[i];
    if (!(c >= 0.0) || !isfinite(c) || !(e > 0.0) || !(e <= 1.0) || !(b >= 0.0) || !isfinite(b)) ++bad;
    if (e != 1.0) ++non1;
  }
  if (bad) atomicAdd(&counts[0], bad);
  if (non1) atomicAdd(&counts[1], non1);
}

// Sweep-precision copies of a canonical FP64 field in the three permuted layouts.
template <typename T>
__global__ void permute_kernel(Dims d, const double *src, T *dst0, T *dst1, T *dst2) {
  const long long cells = d.cells;
  const long long N = cells * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / cells, c = i - f * cells;
    const T v = (T)src[i];
    if (dst0) dst0[f * cells + perm_index(d, 0, c)] = v;
    if (dst1) dst1[f * cells + perm_index(d, 1, c)] = v;
    if (dst2) dst2[f * cells + perm_index(d, 2, c)] = v;
  }
}

// Lagged ghosts before the first formal solution: S of each ghost's periodic image.
template <typename T>
__global__ void init_ghosts_kernel(Dims d, int na, const RayGeom *rays, const double *S, T *G) {
  const long long per_f = (long long)na * d.gsize;
  const long long N = per_f * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / per_f;
    const long long r = i - f * per_f;
    const int k = (int)(r / d.gsize);
    long long j = r - (long long)k * d.gsize;
    const RayGeom g = rays[k];
    int cax[3];
    plane_axes(g.axis, cax);
    const int Nu = d.n[cax[0]], Nv = d.n[cax[1]], Nw = d.n[cax[2]];
    const int su = g.sgn[cax[0]], sv = g.sgn[cax[1]], sw = g.sgn[cax[2]];
    int u, v, w;
    if (j < (long long)Nu * Nv) {
      v = (int)(j / Nu); u = (int)(j % Nu); w = sw > 0 ? Nw - 1 : 0;
    } else if ((j -= (long long)Nu * Nv) < (long long)Nw * Nv) {
      w = (int)(j / Nv); v = (int)(j % Nv); u = su > 0 ? Nu - 1 : 0;
    } else {
      j -= (long long)Nw * Nv;
      w = (int)(j / Nu); u = (int)(j % Nu); v = sv > 0 ? Nv - 1 : 0;
    }
    int crd[3];
    crd[cax[0]] = u;
    crd[cax[1]] = v;
    crd[cax[2]] = w;
    G[i] = (T)S[f * d.cells + ((long long)crd[2] * d.n[1] + crd[1]) * d.n[0] + crd[0]];
  }
}

// Inflow intensities of one non-periodic face [nf][na][face cells]:
// mode VACUUM -> 0, THERMAL -> B of the adjacent layer, FIXED -> user values.
template <typename T>
__global__ void fill_bc_kernel(Dims d, int na, int face, int mode, const double *B,
                               const double *user, T *dst) {
  const int ax = face / 2, side = face % 2;
  const long long fc = d.face[ax];
  const long long N = (long long)d.nf * na * fc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    if (mode == BC_VACUUM) { dst[i] = T(0); continue; }
    if (mode == BC_FIXED) { dst[i] = user ? (T)user[i] : T(0); continue; }
    const long long f = i / ((long long)na * fc);
    const long long p = i % fc;
    int x, y, z;
    const int edge = side ? d.n[ax] - 1 : 0;
    if (ax == 0) { x = edge; z = (int)(p / d.n[1]); y = (int)(p % d.n[1]); }
    else if (ax == 1) { y = edge; z = (int)(p / d.n[0]); x = (int)(p % d.n[0]); }
    else { z = edge; y = (int)(p / d.n[0]); x = (int)(p % d.n[0]); }
    dst[i] = (T)B[f * d.cells + ((long long)z * d.n[1] + y) * d.n[0] + x];
  }
}

// J = sum of the sweep groups' partials (fixed group order), FP64.
template <typename T>
__global__ void reduce_J_kernel(Dims d, int ngroups, const T *Jpart, double *J) {
  const long long N = d.cells * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < ngroups; ++p) s += (double)Jpart[(long long)p * N + i];
    J[i] = s;
  }
}

// J, H, K from the moment partials; f = K/J; 2D drops moments odd in mu_z.
template <typename T>
__global__ void reduce_moments_kernel(Dims d, int ngroups, const T *Jpart, const T *Mpart,
                                      double *J, double *H, double *K, double *F, int two_d) {
  const long long cells = d.cells;
  const long long N = cells * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / cells, c = i - f * cells;
    double s = 0.0, m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < ngroups; ++p) {
      s += (double)Jpart[(long long)p * N + i];
      const T *M = Mpart + (long long)p * 9 * N;
      for (int q = 0; q < 9; ++q) m[q] += (double)M[q * N + i];
    }
    if (two_d) { m[2] = 0.0; m[7] = 0.0; m[8] = 0.0; }
    J[i] = s;
    for (int q = 0; q < 3; ++q) H[(f * 3 + q) * cells + c] = m[q];
    for (int q = 0; q < 6; ++q) {
      K[(f * 6 + q) * cells + c] = m[3 + q];
      F[(f * 6 + q) * cells + c] = m[3 + q] / s;
    }
  }
}

__global__ void eps_thick_min_kernel(Dims d, const double *eps, const double *oml,
                                     unsigned long long *out) {
  const long long N = d.cells * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    if (oml[i] < 0.5) atomicMin(&out[i / d.cells], (unsigned long long)__double_as_longlong(eps[i]));
  }
}

// Q = 4 pi sum_nu w_nu eps_nu chi_nu (J_nu - B_nu)  (integral form, Sec. 4).
// d/dx of one component of H at a cell (i along an axis of n cells, stride st):
// centred difference, wrapped on a periodic axis, one-sided at the ends of a
// bounded one, zero on an axis of one cell.
__device__ __forceinline__ double ddx(const double *F, long long c, int i, int n, long long st, int per,
                                      double h) {
  if (n == 1) return 0.0;
  if (per) {
    const long long cp = i + 1 < n ? c + st : c - (long long)(n - 1) * st;
    const long long cm = i > 0 ? c - st : c + (long long)(n - 1) * st;
    return (F[cp] - F[cm]) / (2.0 * h);
  }
  if (i == 0) return (F[c + st] - F[c]) / h;
  if (i == n - 1) return (F[c] - F[c - st]) / h;
  return (F[c + st] - F[c - st]) / (2.0 * h);
}

// Heating rate (Sec. 4): Q^int = 4 pi sum w chi_abs (J - B), Q^dif = -4 pi sum w div H,
// or per cell and frequency the integral form where chi dx <= 1 (form 2).
__global__ void heating_kernel(Dims d, const double *fw, const double *chi, const double *eps,
                               const double *J, const double *B, const double *H, double hx, double hy,
                               double hz, double width, int form, double *Q) {
  const long long sy = d.n[0], sz = (long long)d.n[0] * d.n[1];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.cells;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % d.n[0]);
    const int y = (int)((c / d.n[0]) % d.n[1]);
    const int z = (int)(c / sz);
    double q = 0.0;
    for (int f = 0; f < d.nf; ++f) {
      const long long i = (long long)f * d.cells + c;
      const bool integral = form == 0 || (form == 2 && chi[i] * width <= 1.0);
      double qf;
      if (integral) {
        qf = eps[i] * chi[i] * (J[i] - B[i]);
      } else {
        const double *Hf = H + (long long)f * 3 * d.cells;
        const double div = ddx(Hf, c, x, d.n[0], 1, d.periodic[0], hx) +
                           ddx(Hf + d.cells, c, y, d.n[1], sy, d.periodic[1], hy) +
                           ddx(Hf + 2 * d.cells, c, z, d.n[2], sz, d.periodic[2], hz);
        qf = -div;
      }
      q += fw[f] * qf;
    }
    Q[c] = 4.0 * M_PI * q;
  }
}

// ---------------------------------------------------------------- launchers

cudaError_t prepare_kernel(const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
  done.insert({fn, dev});
  return cudaSuccess;
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T, int AMAX, bool MOM>
static cudaError_t launch_sweep_t(const SweepArgs<T> &A, int threads, size_t smem, cudaStream_t s) {
  auto kern = sc_sweep_kernel<T, AMAX, MOM>;
  // set on every launch: occupancy queries for other plans change these attributes
  cudaError_t e = prepare_kernel((const void *)kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.cluster * A.ngroups * A.d.nf), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)A.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = A.cluster > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, A);
}

template <typename T, int AMAX, bool MOM>
static cudaError_t launch_tiled_t(const SweepArgs<T> &A, int threads, size_t smem, cudaStream_t s) {
  auto kern = sc_sweep_tiled_kernel<T, AMAX, MOM, kSweepSeg>;
  // set on every launch: occupancy queries for other plans change these attributes
  cudaError_t e = prepare_kernel((const void *)kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.cluster * A.ngroups * A.d.nf), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)A.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = A.cluster > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, A);
}

template <typename T>
static bool pipe_vec_ok(const Dims &d) {
  if (sizeof(T) != 4) return false;
  // rows of every sweep axis (u = y for x sweeps, x otherwise) hold a multiple of 4 cells
  return d.n[0] % 4 == 0 && d.n[1] % 4 == 0;
}

template <typename T, int AMAX, bool MOM>
static cudaError_t launch_pipe_t(const SweepArgs<T> &A, int threads, size_t smem, cudaStream_t s) {
  auto kern = pipe_vec_ok<T>(A.d) ? sc_sweep_pipe_kernel<T, AMAX, MOM, kSweepSeg, (sizeof(T) == 4)>
                                  : sc_sweep_pipe_kernel<T, AMAX, MOM, kSweepSeg, false>;
  cudaError_t e = prepare_kernel((const void *)kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.cluster * A.ngroups * A.d.nf), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)A.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = A.cluster > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, A);
}

template <typename T>
cudaError_t launch_sweep_pipe(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                              cudaStream_t s) {
  switch (amax) {
    case 1: return moments ? launch_pipe_t<T, 1, true>(A, threads, smem, s) : launch_pipe_t<T, 1, false>(A, threads, smem, s);
    case 2: return moments ? launch_pipe_t<T, 2, true>(A, threads, smem, s) : launch_pipe_t<T, 2, false>(A, threads, smem, s);
    case 4: return moments ? launch_pipe_t<T, 4, true>(A, threads, smem, s) : launch_pipe_t<T, 4, false>(A, threads, smem, s);
    case 8: return moments ? launch_pipe_t<T, 8, true>(A, threads, smem, s) : launch_pipe_t<T, 8, false>(A, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int AMAX, bool VEC>
static cudaError_t launch_multi_t(const MultiSweep<T> &M, int threads, size_t smem, cudaStream_t s) {
  auto kern = sc_sweep_multi_kernel<T, AMAX, kSweepSeg, VEC>;
  cudaError_t e = prepare_kernel((const void *)kern);
  if (e != cudaSuccess) return e;
  const int C = M.a[0].cluster;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * M.base[M.n]), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = C > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, M);
}

template <typename T>
cudaError_t launch_sweep_multi(const MultiSweep<T> &M, int amax, int threads, size_t smem, cudaStream_t s) {
  if (M.n < 1 || M.n > kMultiMax) return cudaErrorInvalidValue;
  for (int k = 0; k < M.n; ++k)
    if (M.a[k].cluster != M.a[0].cluster || pipe_vec_ok<T>(M.a[k].d) != pipe_vec_ok<T>(M.a[0].d))
      return cudaErrorInvalidValue;
  const bool vec = pipe_vec_ok<T>(M.a[0].d) && sizeof(T) == 4;
  switch (amax) {
    case 1: return vec ? launch_multi_t<T, 1, true>(M, threads, smem, s) : launch_multi_t<T, 1, false>(M, threads, smem, s);
    case 2: return vec ? launch_multi_t<T, 2, true>(M, threads, smem, s) : launch_multi_t<T, 2, false>(M, threads, smem, s);
    case 4: return vec ? launch_multi_t<T, 4, true>(M, threads, smem, s) : launch_multi_t<T, 4, false>(M, threads, smem, s);
    case 8: return vec ? launch_multi_t<T, 8, true>(M, threads, smem, s) : launch_multi_t<T, 8, false>(M, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_sweep_tiled(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                               cudaStream_t s) {
  switch (amax) {
    case 1: return moments ? launch_tiled_t<T, 1, true>(A, threads, smem, s) : launch_tiled_t<T, 1, false>(A, threads, smem, s);
    case 2: return moments ? launch_tiled_t<T, 2, true>(A, threads, smem, s) : launch_tiled_t<T, 2, false>(A, threads, smem, s);
    case 4: return moments ? launch_tiled_t<T, 4, true>(A, threads, smem, s) : launch_tiled_t<T, 4, false>(A, threads, smem, s);
    case 8: return moments ? launch_tiled_t<T, 8, true>(A, threads, smem, s) : launch_tiled_t<T, 8, false>(A, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                         cudaStream_t s) {
  switch (amax) {
    case 1: return moments ? launch_sweep_t<T, 1, true>(A, threads, smem, s) : launch_sweep_t<T, 1, false>(A, threads, smem, s);
    case 2: return moments ? launch_sweep_t<T, 2, true>(A, threads, smem, s) : launch_sweep_t<T, 2, false>(A, threads, smem, s);
    case 4: return moments ? launch_sweep_t<T, 4, true>(A, threads, smem, s) : launch_sweep_t<T, 4, false>(A, threads, smem, s);
    case 8: return moments ? launch_sweep_t<T, 8, true>(A, threads, smem, s) : launch_sweep_t<T, 8, false>(A, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int AMAX>
static int max_active_t(int tiled, int cluster, int threads, size_t smem) {
  const void *kern = tiled == 3 ? (const void *)sc_sweep_pipe_kernel<T, AMAX, false, kSweepSeg, false>
                    : (tiled ? (const void *)sc_sweep_tiled_kernel<T, AMAX, false, kSweepSeg>
                             : (const void *)sc_sweep_kernel<T, AMAX, false>);
  if (prepare_kernel((const void *)kern) != cudaSuccess) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cluster, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

template <typename T>
int sweep_max_active_clusters(int tiled, int amax, int cluster, int threads, size_t smem) {
  switch (amax) {
    case 1: return max_active_t<T, 1>(tiled, cluster, threads, smem);
    case 2: return max_active_t<T, 2>(tiled, cluster, threads, smem);
    case 4: return max_active_t<T, 4>(tiled, cluster, threads, smem);
    case 8: return max_active_t<T, 8>(tiled, cluster, threads, smem);
    default: return -1;
  }
}

template <typename T>
cudaError_t launch_ali(const AliArgs<T> &A, cudaStream_t s) {
  const dim3 grid((unsigned)(((A.d.n[0] + kAliTile - 1) / kAliTile) * ((A.d.n[1] + kAliTile - 1) / kAliTile)),
                  (unsigned)A.d.n[2], (unsigned)A.d.nf);
  ali_update_kernel<T><<<grid, kAliTile * kAliRows, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_ghosts_from64(long long n, const double *Gout, const double *Gin, float *G, float *Gd,
                                 cudaStream_t s) {
  ghosts_from64_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, Gout, Gin, G, Gd);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(long long n, const float *src, double *dst, cudaStream_t s) {
  f32_to_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_finish(SolveState *st, cudaStream_t s) {
  finish_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_state_op(SolveState *st, int op, int a, double b, int c, cudaStream_t s) {
  state_op_kernel<<<1, 1, 0, s>>>(st, op, a, b, c);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lstar(const Dims &d, const double *chi, const RayGeom *rays, int na, double *lstar,
                         double *oml, const double *const xchi[2], cudaStream_t s) {
  lstar_kernel<T><<<grid_for(d.cells * d.nf, 256), 256, 0, s>>>(d, chi, rays, na, lstar, oml,
                                                                 xchi ? xchi[0] : nullptr,
                                                                 xchi ? xchi[1] : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_validate(long long n, const double *chi, const double *eps, const double *B,
                            int *counts, cudaStream_t s) {
  validate_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, chi, eps, B, counts);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_permute(const Dims &d, const double *src, T *d0, T *d1, T *d2, cudaStream_t s) {
  permute_kernel<T><<<grid_for(d.cells * d.nf, 256), 256, 0, s>>>(d, src, d0, d1, d2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_ghosts(const Dims &d, int na, const RayGeom *rays, const double *S, T *G,
                               cudaStream_t s) {
  init_ghosts_kernel<T><<<grid_for((long long)na * d.gsize * d.nf, 256), 256, 0, s>>>(d, na, rays, S, G);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill_bc(const Dims &d, int na, int face, int mode, const double *B,
                           const double *user, T *dst, cudaStream_t s) {
  const long long n = (long long)d.nf * na * d.face[face / 2];
  fill_bc_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(d, na, face, mode, B, user, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_J(const Dims &d, int ngroups, const T *Jpart, double *J, cudaStream_t s) {
  reduce_J_kernel<T><<<grid_for(d.cells * d.nf, 256), 256, 0, s>>>(d, ngroups, Jpart, J);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_moments(const Dims &d, int ngroups, const T *Jpart, const T *Mpart,
                                  double *J, double *H, double *K, double *F, int two_d,
                                  cudaStream_t s) {
  reduce_moments_kernel<T><<<grid_for(d.cells * d.nf, 256), 256, 0, s>>>(d, ngroups, Jpart, Mpart, J, H, K, F, two_d);
  return cudaGetLastError();
}


cudaError_t launch_inv_denominator(long long n, const double *eps, const double *oml, double *iden,
                                   const double *B, double *ia, double *ib, cudaStream_t s) {
  inv_denominator_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, eps, oml, iden, B, ia, ib);
  return cudaGetLastError();
}

cudaError_t launch_eps_thick_min(const Dims &d, const double *eps, const double *oml,
                                 unsigned long long *out, cudaStream_t s) {
  eps_thick_min_kernel<<<grid_for(d.cells * d.nf, 256), 256, 0, s>>>(d, eps, oml, out);
  return cudaGetLastError();
}

cudaError_t launch_heating(const Dims &d, const double *fw, const double *chi, const double *eps,
                           const double *J, const double *B, const double *H, const double h[3],
                           int form, double *Q, cudaStream_t s) {
  double width = 0.0;   // largest spacing along axes of more than one cell
  for (int a = 0; a < 3; ++a)
    if (d.n[a] > 1) width = width > h[a] ? width : h[a];
  if (width == 0.0) width = h[0];
  heating_kernel<<<grid_for(d.cells, 256), 256, 0, s>>>(d, fw, chi, eps, J, B, H, h[0], h[1], h[2], width,
                                                        form, Q);
  return cudaGetLastError();
}

#define RT_INSTANTIATE(T)                                                                          \
  template cudaError_t launch_sweep<T>(const SweepArgs<T> &, int, bool, int, size_t, cudaStream_t); \
  template cudaError_t launch_seg_table<T>(const SweepArgs<T> &, int, int, T *, T *, cudaStream_t);   \
  template cudaError_t launch_sweep_tiled<T>(const SweepArgs<T> &, int, bool, int, size_t, cudaStream_t); \
  template cudaError_t launch_sweep_pipe<T>(const SweepArgs<T> &, int, bool, int, size_t, cudaStream_t); \
  template cudaError_t launch_sweep_multi<T>(const MultiSweep<T> &, int, int, size_t, cudaStream_t);   \
  template int sweep_max_active_clusters<T>(int, int, int, int, size_t);                          \
  template cudaError_t launch_ali<T>(const AliArgs<T> &, cudaStream_t);                             \
  template cudaError_t launch_lstar<T>(const Dims &, const double *, const RayGeom *, int, double *, \
                                       double *, const double *const[2], cudaStream_t);                                     \
  template cudaError_t launch_permute<T>(const Dims &, const double *, T *, T *, T *, cudaStream_t);  \
  template cudaError_t launch_init_ghosts<T>(const Dims &, int, const RayGeom *, const double *, T *, \
                                             cudaStream_t);                                         \
  template cudaError_t launch_fill_bc<T>(const Dims &, int, int, int, const double *, const double *, \
                                         T *, cudaStream_t);                                        \
  template cudaError_t launch_reduce_J<T>(const Dims &, int, const T *, double *, cudaStream_t);     \
  template cudaError_t launch_reduce_moments<T>(const Dims &, int, const T *, const T *, double *,   \
                                                double *, double *, double *, int, cudaStream_t);

RT_INSTANTIATE(float)
RT_INSTANTIATE(double)

}  // namespace rtk
