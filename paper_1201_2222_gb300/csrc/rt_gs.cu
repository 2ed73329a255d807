// Gauss-Seidel ALI kernels (Sec. 3.4, after Trujillo Bueno & Fabiani Bendicho
// 1995), in plane-wavefront form.
//
//   gs_weights_kernel  per cell, the first-order correction weights of the
//                      forward rays on the 3 x 3 cells of the plane above
//   gs_reverse_kernel  the reverse phase of one iteration: the reverse rays
//                      swept from the top plane of V down, each plane's S
//                      updated (Eq. 24) with the freshest J before the next
//                      plane is swept
//
// One Gauss-Seidel iteration is: the forward sweep (every group except those
// crossing the V face with mu_V < 0) with the old S, then gs_reverse_kernel.
// At plane k the reverse kernel forms
//   J = J_F + C + sum over reverse rays of w I,
// where J_F sums the forward groups' partials and C = sum over the 3 x 3 cells
// of plane k+1 of (weight) x dS corrects, to first order, the forward rays' use
// of the old S there.  dS = [(1 - eps) J + eps B - S] / [1 - (1 - eps) Lambda*];
// then the reverse rays' intensities at plane k take the change of the S they
// read from plane k (Psi0 dS of the cell; on the top plane of a bounded V axis
// also Psi- times the change of the ghost layer, a copy of that plane).
//
// The planes are separated by a grid barrier: the launch is cooperative (all
// blocks resident) and each wait gives up after a bounded number of polls,
// recording kGsBarrierTimeout in the solve state, after which every block
// returns.  Values that other blocks write during the kernel (S, dS, the
// reverse intensities) are read with L2 loads (ld.global.cg) after the barrier.
#include <cuda_runtime.h>

#include <cmath>

#include "rt_common.cuh"
#include "rt_device.cuh"
#include "rt_kernels.h"

namespace rtk {

namespace {

// In-plane axes of the reverse axis V, in the plane coordinates of its sweep
// groups: u = cax[0], v = cax[1] (V = z: x, y; V = y in 2D: x, z).
__host__ __device__ inline int slot_of(int ou, int ov) { return (ov + 1) * 3 + (ou + 1); }

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch: the n-th call returns once every block
// has made it.  Arrivals are counted in two levels (blocks in groups of
// kGsBarGroup on their own counters, bar[1 + group]; the last block of a group
// adds the group to bar[0]) so that no counter takes more than a few dozen
// atomics per barrier.  A wait gives up after `limit` polls (about 64 ns
// apart).  Returns false (and records the timeout) if a wait gave up or another
// block already did; the caller then returns.
__device__ bool grid_sync(unsigned *bar, unsigned epoch, SolveState *st, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned grp = blockIdx.x / kGsBarGroup, ngrp = (gridDim.x + kGsBarGroup - 1) / kGsBarGroup;
    const unsigned gsize = min((unsigned)kGsBarGroup, gridDim.x - grp * kGsBarGroup);
    __threadfence();
    if (atomicAdd(&bar[1 + grp], 1u) + 1 == epoch * gsize) {   // the group is complete
      __threadfence();
      atomicAdd(&bar[0], 1u);
    }
    const unsigned target = epoch * ngrp;
    long long polls = 0;
    while (ld_relaxed(bar) < target) {   // the fence below orders what follows
      if (*(volatile int *)&st->err == kGsBarrierTimeout || ++polls > limit) {
        atomicCAS(&st->err, 0, kGsBarrierTimeout);
        good = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) {
  return __ldcg(p);
}

// periodic wrap or clamp of one coordinate (the ghost-layer rule for chi and S)
__device__ __forceinline__ int map_coord(int c, int n, bool per) {
  return c < 0 ? (per ? c + n : 0) : (c >= n ? (per ? c - n : n - 1) : c);
}

}  // namespace

// --------------------------------------------------------------- correction weights
// One thread per cell and frequency.  For every forward ray with mu_V < 0, its
// upwind vertices on the plane above (offset +1 along V) add w Psi- (vertex
// weight) to the slot of their in-plane offset; Psi- = 1 - E - Psi0 in the
// sweep's precision T (the forward sweep's own weight of S-).
template <typename T>
__global__ void __launch_bounds__(256) gs_weights_kernel(Dims d, int V, const double *chi,
                                                          const RayGeom *rays, const int *fwd,
                                                          int nfwd, double *gsw) {
  const long long cells = d.cells;
  const long long N = cells * d.nf;
  int cax[3];
  plane_axes(V, cax);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / cells, c = i - f * cells;
    const int x = (int)(c % d.n[0]), y = (int)((c / d.n[0]) % d.n[1]), z = (int)(c / ((long long)d.n[0] * d.n[1]));
    const double *chf = chi + f * cells;
    const T chi0 = (T)chf[c];
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    for (int k = 0; k < nfwd; ++k) {
      const RayGeom r = rays[fwd[k]];
      const int ax = r.axis, b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
      const double f1 = b1 == 0 ? r.frac[0] : (b1 == 1 ? r.frac[1] : r.frac[2]);
      const double f2 = b2 == 0 ? r.frac[0] : (b2 == 1 ? r.frac[1] : r.frac[2]);
      T chim = T(0);
      double wv[4];
      int oo[4][3];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int d1 = v >> 1, d2 = v & 1;
        wv[v] = (d1 ? f1 : 1.0 - f1) * (d2 ? f2 : 1.0 - f2);
        int o[3] = {0, 0, 0};
        o[ax] = -r.sgn[ax];
        o[b1] = -d1 * r.sgn[b1];
        o[b2] = -d2 * r.sgn[b2];
        oo[v][0] = o[0];
        oo[v][1] = o[1];
        oo[v][2] = o[2];
        const int xx = map_coord(x + o[0], d.n[0], d.periodic[0]);
        const int yy = map_coord(y + o[1], d.n[1], d.periodic[1]);
        const int zz = map_coord(z + o[2], d.n[2], d.periodic[2]);
        chim += (T)wv[v] * (T)chf[((long long)zz * d.n[1] + yy) * d.n[0] + xx];
      }
      const T dtau = (chim + chi0) * (T)(0.5 * r.s);
      T E, psi0, om;
      seg_weights(dtau, E, psi0, om);
      const double psim = (double)(om - E);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (wv[v] == 0.0 || pick3(oo[v][0], oo[v][1], oo[v][2], V) != 1) continue;
        const int ou = pick3(oo[v][0], oo[v][1], oo[v][2], cax[0]);
        const int ov = pick3(oo[v][0], oo[v][1], oo[v][2], cax[1]);
        const int q = slot_of(ou, ov);
#pragma unroll
        for (int s9 = 0; s9 < 9; ++s9)
          if (s9 == q) acc[s9] += r.w * psim * wv[v];
      }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) gsw[(f * 9 + q) * cells + c] = acc[q];
  }
}

template <typename T>
cudaError_t launch_gs_weights(const Dims &d, int V, const double *chi, const RayGeom *rays,
                              const int *fwd, int nfwd, double *gsw, cudaStream_t s) {
  const long long N = d.cells * d.nf;
  const int grid = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
  gs_weights_kernel<T><<<grid, 256, 0, s>>>(d, V, chi, rays, fwd, nfwd, gsw);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reverse phase
// A block takes tiles of TC cells of one plane and frequency; its thread t
// sweeps reverse ray t / TC at cell t % TC (TC = kGsThreads / nrev).  Per tile:
// the cells' inputs that do not depend on this plane's rays, the rays'
// intensities (upwind plane above), the cells' updates (one thread per cell, the
// rays' J terms summed in ray order), then the rays' corrections.  The planes of
// all frequencies advance together, one grid barrier apart.
//
// Incremental solves (float32 grids after their first iteration) sweep changes:
// the reverse rays' intensities at plane k differ from the last iteration's
// corrected ones by the SC update of (the change of S on the plane above, this
// iteration's dS; of ghost S read elsewhere, none where the last top-plane
// correction covered it, else the last iteration's dS; of the lagged ghost
// intensities, their increments), with no change of S0 yet.  J of the forward
// and of the reverse rays is kept in FP64 and advanced by the swept changes, so
// float32 rounding scales with the change, not with J.
template <typename T>
__global__ void __launch_bounds__(kGsThreads, 3) gs_reverse_kernel(const GsArgs<T> G) {
  const SweepArgs<T> &A = G.A;
  SolveState *st = A.st;
  if (st->done) return;   // converged earlier in this batch: every block returns
  __shared__ AngleParam<T> P[kGsMaxRev];
  __shared__ T jr[kGsThreads];
  __shared__ T jp0[kGsThreads];
  __shared__ double dsm[kGsThreads];
  __shared__ double rmax_s[kGsThreads / 32];
  __shared__ int fgs[kMaxGroups];
  const int nrev = G.nrev;
  for (int k = threadIdx.x; k < nrev; k += blockDim.x) P[k] = A.ang[G.rev0 + k];
  for (int k = threadIdx.x; k < G.nfg; k += blockDim.x) fgs[k] = G.fgroups[k];
  int cax[3];
  plane_axes(G.V, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const bool perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
             perW = pick3(A.d.periodic, cax[2]);
  const long long csu = canon_stride(A.d.n, cax[0]), csv = canon_stride(A.d.n, cax[1]),
                  csw = canon_stride(A.d.n, cax[2]);
  const long long cells = A.d.cells, plane = (long long)Nu * Nv;
  const int nf = A.d.nf;
  const int TC = kGsThreads / nrev;
  const long long tiles_pf = (plane + TC - 1) / TC, tiles = tiles_pf * nf;
  const int ri = threadIdx.x / TC, cs = threadIdx.x % TC;
  const bool ray_thread = ri < nrev;
  const long long IrPlane = (long long)nf * nrev * plane;   // one of the four blocks of Ir
  unsigned nbar = 0;
  double rmax = 0.0;
  const bool inc = G.incremental && st->iter > 0;    // sweep changes
  const bool emit = G.incremental && st->iter == 0;  // full sweep that records ghost increments

  // S of the previous formal solution (the old S, read where a plane has not
  // been updated yet) -- every cell, before any update
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells * nf;
       i += (long long)gridDim.x * blockDim.x)
    G.Sfs[i] = G.S64[i];
  if (!grid_sync(G.bar, ++nbar, st, G.poll_limit)) return;

  const int fs = st->fs_count;
  const int prev = fs & 1;
  const T *Gp = A.G[prev];
  T *Gn = A.G[prev ^ 1];
  const T *Gsrc = inc ? A.Gd[prev] : Gp;     // inflow: ghost increments or ghosts
  T *Gdn = G.incremental ? A.Gd[prev ^ 1] : nullptr;
  const bool ghost_fix = !perW || Nw == 1;   // the top plane's ghost layer copies the top plane

  // outflow ghosts of reverse ray p at cell (u, v, w): value I (or its change)
  auto store_ghosts = [&](const AngleParam<T> &p, int f, int u, int v, int w, T I) {
    const long long gb = ((long long)f * A.na + p.angle) * A.d.gsize;
    if (perU && u == (p.su > 0 ? Nu - 1 : 0)) ghost_store(Gp, Gn, Gdn, gb + plane + (long long)w * Nv + v, I, inc, emit);
    if (perV && v == (p.sv > 0 ? Nv - 1 : 0))
      ghost_store(Gp, Gn, Gdn, gb + plane + (long long)Nw * Nv + (long long)w * Nu + u, I, inc, emit);
    if (perW && w == 0) ghost_store(Gp, Gn, Gdn, gb + (long long)v * Nu + u, I, inc, emit);
  };

  for (int t = 0; t < Nw; ++t) {
    const int w = Nw - 1 - t;
    const bool fix = t == 0 && ghost_fix;
    const T *Iprv = G.Ir + (long long)(t & 1) * IrPlane;        // plane w + 1 (corrected)
    T *Icur = G.Ir + (long long)((t + 1) & 1) * IrPlane;        // plane w
    T *Psz = G.Ir + 2 * IrPlane, *Psm = G.Ir + 3 * IrPlane;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int f = (int)(tile / tiles_pf);
      const long long pc = (tile - (long long)f * tiles_pf) * TC + cs;   // cell in the plane
      const bool live = pc < plane && !(G.fmask && G.fmask[f]);
      const int u = live ? (int)(pc % Nu) : 0, v = live ? (int)(pc / Nu) : 0;
      const long long c = (long long)u * csu + (long long)v * csv + (long long)w * csw;
      const long long fc = (long long)f * cells;
      // sweep-precision copies along V ([w][v][u]): chi, and S (dS) -- new on
      // the planes already updated, old elsewhere
      const T *chv = A.chiP[G.V] + fc;
      T *spv = G.SPV + fc;
      T I0 = T(0), psi0 = T(0), psim = T(0);
      // ---- 0. the cell's inputs that do not depend on this plane's rays (the
      // plane above's dS is final since the barrier), loaded before the rays'
      // work so that their latency overlaps it
      const long long i = fc + c;
      double JF = 0.0, JRp = 0.0, corr = 0.0, S = 0.0, e = 0.0, Bc = 0.0, idn = 0.0;
      if (threadIdx.x < TC && live) {
        S = G.Sfs[i];
        e = G.eps[i];
        Bc = G.B[i];
        idn = G.iden[i];
        if (inc) JRp = G.JR64[i];
        // the forward partials and the correction's 9 weights and changes: all
        // loads issued before any is used (latency, not bandwidth, bounds this)
        const T *jp = A.Jpart + (long long)f * cells + c;
        const long long gstride = (long long)nf * cells;
        if (sizeof(T) == 4) {   // float partials summed as an exact float pair (TwoSum)
          float hi = 0.f, lo = 0.f;
          for (int q0 = 0; q0 < G.nfg; q0 += 8) {
            float xs[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) xs[q] = q0 + q < G.nfg ? (float)jp[fgs[q0 + q] * gstride] : 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float x = xs[q];
              const float s2 = hi + x;
              const float bp = s2 - hi;
              lo += (hi - (s2 - bp)) + (x - bp);
              hi = s2;
            }
          }
          JF = (double)hi + (double)lo;
        } else {
          for (int q0 = 0; q0 < G.nfg; q0 += 8) {
            double xs[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) xs[q] = q0 + q < G.nfg ? (double)jp[fgs[q0 + q] * gstride] : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) JF += xs[q];
          }
        }
        if (inc) JF += G.JF64[i];
        if (G.JF64) G.JF64[i] = JF;
        if (w + 1 < Nw) {
          double cw[9], ds[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            const int ou = q % 3 - 1, ov = q / 3 - 1;
            const int mu_ = map_coord(u + ou, Nu, perU), mv_ = map_coord(v + ov, Nv, perV);
            cw[q] = G.gsw[((long long)f * 9 + q) * cells + c];
            ds[q] = ldcg(G.dS + fc + (long long)mu_ * csu + (long long)mv_ * csv + (long long)(w + 1) * csw);
          }
#pragma unroll
          for (int q = 0; q < 9; ++q) corr += cw[q] * ds[q];
        }
      }
      // ---- 1. reverse ray ri at cell (u, v, w)
      if (ray_thread) {
        T wj = T(0), wp0 = T(0);
        if (live) {
          const AngleParam<T> &p = P[ri];
          const T wts[4] = {p.wa, p.wb, p.wc, p.wd};
          T Im = T(0), Sm = T(0), chim = T(0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int uu = u - ((q & 1) ? p.su : 0), vv = v - ((q & 2) ? p.sv : 0), ww = w + 1;
            const int mu_ = map_coord(uu, Nu, perU), mv_ = map_coord(vv, Nv, perV), mw_ = map_coord(ww, Nw, perW);
            const long long mp = ((long long)mw_ * Nv + mv_) * Nu + mu_;
            const bool in = uu >= 0 && uu < Nu && vv >= 0 && vv < Nv && ww < Nw;
            T Iv;
            if (in) Iv = ldcg(Iprv + ((long long)f * nrev + ri) * plane + (long long)vv * Nu + uu);
            else Iv = ghost_I<T>(A, cax, Nu, Nv, Nw, f, p.angle, Gsrc, inc, uu, vv, ww);
            // S of the plane above is the new one.  A ghost mapped elsewhere
            // reads the old S: on the top plane itself (being updated now) from
            // the FP64 copy, whose change the last iteration's top-plane
            // correction already covered; on plane 0 (periodic V, updated last)
            // from the sweep copy, which still holds the last iteration's dS
            T Sv;
            if (mw_ != w) Sv = ldcg(spv + mp);
            else Sv = inc ? T(0) : (T)G.Sfs[fc + (long long)mu_ * csu + (long long)mv_ * csv + (long long)mw_ * csw];
            Im += wts[q] * Iv;
            Sm += wts[q] * Sv;
            if (!A.WE) chim += wts[q] * chv[mp];
          }
          const long long pown = ((long long)w * Nv + v) * Nu + u;
          const T S0 = inc ? T(0) : spv[pown];
          T E, om;
          if (A.WE) {   // the medium's segment weights (FP64 grids), tabulated once
            const long long wi = ((long long)(G.rev0 + ri) * nf + f) * cells + pown;
            E = A.WE[wi];
            psi0 = A.WP[wi];
            om = T(1) - psi0;
          } else {
            const T dtau = (chim + chv[pown]) * p.hs;
            seg_weights(dtau, E, psi0, om);
          }
          I0 = Sm + E * (Im - Sm) + psi0 * (S0 - Sm);
          psim = om - E;
          wj = p.wq * I0;
          wp0 = p.wq * psi0;
        }
        jr[threadIdx.x] = wj;
        jp0[threadIdx.x] = wp0;
      }
      __syncthreads();
      // ---- 2. the cell's update with the freshest J
      if (threadIdx.x < TC && live) {
        T jrs = T(0), wps = T(0);   // the reverse rays' J terms, in ray order
        for (int r = 0; r < nrev; ++r) {
          jrs += jr[r * TC + threadIdx.x];
          wps += jp0[r * TC + threadIdx.x];
        }
        const double JR = JRp + (double)jrs, WP = (double)wps;
        const double J = JF + corr + JR;
        const double dS = ((1.0 - e) * J + e * Bc - S) * idn;
        const double Sn = S + dS;
        G.S64[i] = Sn;
        G.J64[i] = J;
        G.dS[i] = dS;
        spv[((long long)w * Nv + v) * Nu + u] = (T)(inc ? dS : Sn);
        // the reverse rays' J once their intensities take this dS (the top plane
        // of a bounded V axis adds its ghost-layer term in the pass below)
        if (G.JR64) G.JR64[i] = JR + WP * dS;
        dsm[threadIdx.x] = dS;
        const double ad = fabs(dS), as = fabs(Sn);
        const double r = (sizeof(T) == 4 && as > 1e-30 && as < 1e30 && ad < 1e30)
                             ? (double)__fdividef((float)ad, (float)as)
                             : (as > 0.0 ? ad / as : (ad > 0.0 ? INFINITY : 0.0));
        rmax = fmax(rmax, r);
      }
      __syncthreads();
      // ---- 3. the ray's intensity takes the change of its own S0
      if (ray_thread && live) {
        const long long o = ((long long)f * nrev + ri) * plane + pc;
        if (fix) {   // finished after the barrier below, once the whole plane has its dS
          Icur[o] = I0;
          Psz[o] = psi0;
          Psm[o] = psim;
        } else {
          const T I = I0 + psi0 * (T)dsm[cs];
          Icur[o] = I;
          store_ghosts(P[ri], f, u, v, w, I);
        }
      }
      __syncthreads();
    }
    if (!grid_sync(G.bar, ++nbar, st, G.poll_limit)) return;
    if (fix) {
      // top plane of a bounded V axis: the upwind S of the ghost layer was this
      // plane's; add Psi- times its change, then store the outflow ghosts.  One
      // thread per cell, the rays in order (their J term in a fixed order).
      const long long n = (long long)nf * plane;
      for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
           j += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(j / plane);
        const long long pc = j % plane;
        if (G.fmask && G.fmask[f]) continue;
        const int u = (int)(pc % Nu), v = (int)(pc / Nu);
        const long long fc = (long long)f * cells;
        const long long c = (long long)u * csu + (long long)v * csv + (long long)w * csw;
        const T dSc = (T)ldcg(G.dS + fc + c);
        double extra = 0.0;   // the ghost-layer term of the reverse rays' J
        for (int r = 0; r < nrev; ++r) {
          const AngleParam<T> &p = P[r];
          const T wts[4] = {p.wa, p.wb, p.wc, p.wd};
          double gsum = 0.0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int uu = u - ((q & 1) ? p.su : 0), vv = v - ((q & 2) ? p.sv : 0), ww = w + 1;
            const int mw_ = map_coord(ww, Nw, perW);
            if (wts[q] == T(0) || mw_ != w) continue;
            const int mu_ = map_coord(uu, Nu, perU), mv_ = map_coord(vv, Nv, perV);
            gsum += (double)wts[q] * ldcg(G.dS + fc + (long long)mu_ * csu + (long long)mv_ * csv + (long long)w * csw);
          }
          const long long o = ((long long)f * nrev + r) * plane + pc;
          const T gterm = Psm[o] * (T)gsum;
          const T I = Icur[o] + Psz[o] * dSc + gterm;
          Icur[o] = I;
          extra += (double)(p.wq * gterm);
          store_ghosts(p, f, u, v, w, I);
        }
        if (G.JR64) G.JR64[fc + c] += extra;
      }
      if (!grid_sync(G.bar, ++nbar, st, G.poll_limit)) return;
    }
  }
  // residual: block maximum, then one atomic per block
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) rmax_s[threadIdx.x >> 5] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, rmax_s[q]);
    if (r > 0.0) atomicMax(&st->resid_bits, (unsigned long long)__double_as_longlong(r));
  }
}

template <typename T>
cudaError_t launch_gs_reverse(const GsArgs<T> &G, cudaStream_t s) {
  // resident blocks per SM of this instantiation (a thread-safe one-time query)
  static const int bps = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gs_reverse_kernel<T>, kGsThreads, 0) != cudaSuccess)
      return 1;
    return n > 0 ? n : 1;
  }();
  cudaError_t e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int cax[3];
  plane_axes(G.V, cax);
  const long long plane = (long long)G.A.d.n[cax[0]] * G.A.d.n[cax[1]];
  const int TC = kGsThreads / G.nrev;
  const long long tiles = (plane + TC - 1) / TC * G.A.d.nf;
  const long long cap = std::min<long long>((long long)bps * sms, (long long)(kGsBarWords - 1) * kGsBarGroup);
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, cap));
  if ((e = cudaMemsetAsync(G.bar, 0, kGsBarWords * sizeof(unsigned), s)) != cudaSuccess) return e;
  GsArgs<T> arg = G;
  void *params[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)gs_reverse_kernel<T>, dim3(grid), dim3(kGsThreads),
                                     params, 0, s);
}

template cudaError_t launch_gs_weights<float>(const Dims &, int, const double *, const RayGeom *, const int *,
                                              int, double *, cudaStream_t);
template cudaError_t launch_gs_weights<double>(const Dims &, int, const double *, const RayGeom *, const int *,
                                               int, double *, cudaStream_t);
template cudaError_t launch_gs_reverse<float>(const GsArgs<float> &, cudaStream_t);
template cudaError_t launch_gs_reverse<double>(const GsArgs<double> &, cudaStream_t);

}  // namespace rtk
