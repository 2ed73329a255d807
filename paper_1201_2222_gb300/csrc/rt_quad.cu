// Second-order formal solution (Sec. 3.3): monotonic quadratic interpolation on
// the crossed face and Bezier-controlled parabolic integration of S along the
// segment.  Same wavefront organisation as the pipelined linear sweep (one
// cluster per sweep group and frequency, the plane split into row strips, strip
// edges pushed to the neighbours' halo rows through distributed shared memory),
// with a four-plane chi/S ring so that the downwind plane (S+, chi+) is staged
// while a plane is computed.
//
// Per cell and ray, with (tu, tv) = -(sign(mu_u) f_u, sign(mu_v) f_v) the offsets
// of the upwind point on the previous plane (f the fractional crossing offsets):
//   X- = quad(X on the 3 x 3 vertices of the previous plane at (tu, tv)), X = I, S, chi
//   Y+ = quad(Y on the 3 x 3 vertices of the next plane at (-tu, -tv)),   Y = S, chi
// where quad interpolates along u (the lower canonical face axis) in each of the
// three rows, then along v, each time by the parabola through three values
// clamped to the two that bracket the point;
//   dtau- = (chi- + chi0) s/2, dtau+ = (chi0 + chi+) s/2,
//   Sc = S0 - dtau-/2 S'(tau0), S' from the parabola through (S-, S0, S+), clamped
//   to [min(S-, S0), max(S-, S0)],
//   I0 = I- e^{-dtau-} + a S- + b S0 + c Sc  (integrals of the quadratic Bezier
//   curve's Bernstein polynomials against e^{-(dtau- - t)}),
// and per ray the weight of S0, b + c dSc/dS0 with dSc/dS0 limited to [0, 1]
// (0 or 1 where Sc is clamped); its complement 1 - b - c dSc/dS0 =
// a + e^{-dtau-} + c (1 - dSc/dS0) is accumulated without cancellation for the
// Jacobi denominator.  The scheme is nonlinear in S (the clamps), so ALI solves
// take Lambda* from every formal solution and never sweep increments.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "rt_common.cuh"
#include "rt_device.cuh"
#include "rt_kernels.h"

namespace cg = cooperative_groups;

namespace rtk {

// parabola through f(-1), f(0), f(1) at t in [-1, 1], clamped to the range of the
// two values that bracket t
template <typename T>
__device__ __forceinline__ T quad1(T fm, T f0, T fp, T t) {
  if (t == T(0)) return f0;
  T v = f0 + T(0.5) * t * (fp - fm) + T(0.5) * t * t * (fp - T(2) * f0 + fm);
  const T fe = t < T(0) ? fm : fp;
  const T lo = fe < f0 ? fe : f0, hi = fe < f0 ? f0 : fe;
  v = v < lo ? lo : v;
  v = v > hi ? hi : v;
  return v;
}

// a, b, c of I0 = I- E + a S- + b S0 + c Sc for a segment of optical depth t, and
// E = e^{-t}: with m_n = int_0^t x^n e^{-x} dx / t^(n+1), a = t m2,
// b = t (m0 - 2 m1 + m2), c = 2 t (m1 - m2).  Below the threshold (1 in float32,
// 0.1 in FP64) m_n is the series sum_k (-t)^k / (k! (n+k+1)).
template <typename T>
__device__ __forceinline__ void bezier_weights(T t, T &a, T &b, T &c, T &E) {
  const bool f32 = sizeof(T) == 4;
  E = f32 ? (T)__expf(-(float)t) : (T)exp(-(double)t);
  T m0, m1, m2;
  if (t < (f32 ? T(1) : T(0.1))) {
    T p = T(1), fct = T(1);
    m0 = m1 = m2 = T(0);
    const int nt = f32 ? 13 : 14;
    for (int k = 0; k < nt; ++k) {
      m0 += p / (fct * T(k + 1));
      m1 += p / (fct * T(k + 2));
      m2 += p / (fct * T(k + 3));
      p *= -t;
      fct *= T(k + 1);
    }
  } else {
    const T E0 = T(1) - E;
    const T E1 = E0 - t * E;
    const T E2 = T(2) * E1 - t * t * E;
    m0 = E0 / t;
    m1 = E1 / (t * t);
    m2 = E2 / (t * t * t);
  }
  a = t * m2;
  b = t * (m0 - T(2) * m1 + m2);
  c = T(2) * t * (m1 - m2);
}

// one cell, one ray: the second-order update.  Iu[r][k], Su, Cu: rows v-1, v, v+1
// (r = 0, 1, 2) and columns u-1, u, u+1 (k) of the previous plane; Sd, Cd the same
// on the next plane.  Returns I0; lam = dI0/dS0 (limited), om = 1 - lam.
template <typename T>
__device__ __forceinline__ T quad_update(const T (&Iu)[3][3], const T (&Su)[3][3], const T (&Cu)[3][3],
                                         const T (&Sd)[3][3], const T (&Cd)[3][3], T S0, T chi0, T tu,
                                         T tv, T hs, T &lam, T &om) {
  T rI[3], rS[3], rC[3], rSd[3], rCd[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    rI[r] = quad1(Iu[r][0], Iu[r][1], Iu[r][2], tu);
    rS[r] = quad1(Su[r][0], Su[r][1], Su[r][2], tu);
    rC[r] = quad1(Cu[r][0], Cu[r][1], Cu[r][2], tu);
    rSd[r] = quad1(Sd[r][0], Sd[r][1], Sd[r][2], -tu);
    rCd[r] = quad1(Cd[r][0], Cd[r][1], Cd[r][2], -tu);
  }
  const T Im = quad1(rI[0], rI[1], rI[2], tv);
  const T Sm = quad1(rS[0], rS[1], rS[2], tv);
  const T chim = quad1(rC[0], rC[1], rC[2], tv);
  const T Sp = quad1(rSd[0], rSd[1], rSd[2], -tv);
  const T chip = quad1(rCd[0], rCd[1], rCd[2], -tv);
  const T hm = (chim + chi0) * hs, hp = (chi0 + chip) * hs;
  if (!(hm > T(0))) {   // no opacity along the segment
    lam = T(0);
    om = T(1);
    return Im;
  }
  const T dm = (S0 - Sm) / hm;
  T dS, ddS;
  if (hp > T(0)) {
    const T dp = (Sp - S0) / hp;
    dS = (hp * dm + hm * dp) / (hm + hp);
    ddS = (hp / hm - hm / hp) / (hm + hp);
  } else {
    dS = dm;
    ddS = T(1) / hm;
  }
  T Sc = S0 - T(0.5) * hm * dS;
  T dSc = T(1) - T(0.5) * hm * ddS;
  dSc = dSc < T(0) ? T(0) : (dSc > T(1) ? T(1) : dSc);
  const T lo = Sm < S0 ? Sm : S0, hi = Sm < S0 ? S0 : Sm;
  if (Sc < lo) {
    Sc = lo;
    dSc = lo == S0 ? T(1) : T(0);
  } else if (Sc > hi) {
    Sc = hi;
    dSc = hi == S0 ? T(1) : T(0);
  }
  T a, b, c, E;
  bezier_weights(hm, a, b, c, E);
  lam = b + c * dSc;
  om = a + E + c * (T(1) - dSc);
  return Im * E + a * Sm + b * S0 + c * Sc;
}

// Each thread takes segments of kQuadSeg = 2 cells: with 4-cell segments the 3 x 3
// stencils of chi, S and I for the upwind and downwind points needed more than
// the 128 registers a thread of a 512-thread CTA may hold and some spilled to
// local memory (and capping the CTA at 384 or 256 threads to avoid that was
// slower still: 12 or 8 warps per SM hide less latency); 2-cell segments fit in
// 113 registers.
template <typename T, int AMAX, bool MOM>
__global__ void __launch_bounds__(sweep_max_threads<T>()) sc_sweep_quad_kernel(const SweepArgs<T> A) {
  constexpr int SEG = kQuadSeg;
  if (A.skip_if_done && A.st->done) return;
  const int C = A.cluster;
  const int rank = blockIdx.x % C;
  const int inst = blockIdx.x / C;
  const int gi = inst % A.ngroups;
  const int f = inst / A.ngroups;
  const GroupParam gp = A.grp[gi];
  if (gp.na > A.ray_slots) {
    if (threadIdx.x == 0) atomicCAS(&A.st->err, 0, 31);
    return;
  }
  int cax[3];
  plane_axes(gp.axis, cax);
  const int Nu = pick3(A.d.n, cax[0]), Nv = pick3(A.d.n, cax[1]), Nw = pick3(A.d.n, cax[2]);
  const int perU = pick3(A.d.periodic, cax[0]), perV = pick3(A.d.periodic, cax[1]),
            perW = pick3(A.d.periodic, cax[2]);
  const long long csu = canon_stride(A.d.n, cax[0]), csv = canon_stride(A.d.n, cax[1]),
                  csw = canon_stride(A.d.n, cax[2]);
  const int v0 = (int)(((long long)rank * Nv) / C);
  const int v1 = (int)(((long long)(rank + 1) * Nv) / C);
  const int R = v1 - v0;
  const int Rmax = (Nv + C - 1) / C;
  const int W = pipe_row_len(Nu, SEG);
  const int RX = Rmax + 2;
  const int pb = RX * W;
  const int ib = A.ray_slots * pb;
  const long long plane = (long long)Nu * Nv;
  const long long cells = A.d.cells;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ib = reinterpret_cast<T *>(smem_raw);   // [2][slots][RX][W]   intensities
  T *Cr = Ib + 2 * ib;                       // [4][RX][W]          chi ring
  T *Sr = Cr + 4 * pb;                       // [4][RX][W]          S ring
  __shared__ AngleParam<T> P[AMAX];
  if (threadIdx.x < gp.na) P[threadIdx.x] = A.ang[gp.a0 + threadIdx.x];

  const int fs = A.st->fs_count + A.parity_offset;
  const int prev = fs & 1;
  const T *Gp = A.G[prev];
  T *Gn = A.G[prev ^ 1];
  const T *chiP = A.chiP[gp.axis] + (long long)f * cells;
  const T *SP = A.SP[gp.axis] + (long long)f * cells;
  T *Jout = A.Jpart + ((long long)gi * A.d.nf + f) * cells;
  T *Oout = A.Opart ? A.Opart + ((long long)gi * A.d.nf + f) * cells : nullptr;
  const int sa = gp.sa;
  const int wlast = sa > 0 ? Nw - 1 : 0;
  const int na = gp.na;
  const int nseg = (Nu + SEG - 1) / SEG;
  cg::cluster_group cluster = cg::this_cluster();
  T *Ntop0 = nullptr, *Nbot0 = nullptr;
  int top_row = 0;
  if (C > 1) {
    if (rank > 0) {
      Ntop0 = cluster.map_shared_rank(Ib, rank - 1);
      top_row = v0 - (int)(((long long)(rank - 1) * Nv) / C) + 1;
    }
    if (rank < C - 1) Nbot0 = cluster.map_shared_rank(Ib, rank + 1);
  }
  __syncthreads();

  // source plane of a sweep coordinate outside the grid: the periodic image, or
  // the boundary layer (ghost chi and S copy it)
  auto src_plane = [&](int wv) { return wv < 0 ? (perW ? wv + Nw : 0) : (wv >= Nw ? (perW ? wv - Nw : Nw - 1) : wv); };
  // chi and S of plane wsrc (rows v0-1 .. v1, columns -1 .. Nu, wrapped or clamped) -> ring slot
  auto stage = [&](int wsrc, int slot) {
    T *Cd = Cr + slot * pb, *Sd = Sr + slot * pb;
    const int rows = R + 2;
    for (int idx = threadIdx.x; idx < rows * Nu; idx += blockDim.x) {
      const int row = idx / Nu, u = idx - row * Nu;
      int vv = v0 - 1 + row;
      vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
      const long long o = (long long)wsrc * plane + (long long)vv * Nu + u;
      cp_async_elem(Cd + RT_IDX(row * W + kPipeX0 + u, 8LL * pb, 61), chiP + o);
      cp_async_elem(Sd + RT_IDX(row * W + kPipeX0 + u, 8LL * pb, 61), SP + o);
    }
    for (int idx = threadIdx.x; idx < 2 * rows; idx += blockDim.x) {
      const int side = idx / rows, row = idx - side * rows;
      int vv = v0 - 1 + row;
      vv = vv < 0 ? (perV ? vv + Nv : 0) : (vv >= Nv ? (perV ? vv - Nv : Nv - 1) : vv);
      const int uu = side ? (perU ? 0 : Nu - 1) : (perU ? Nu - 1 : 0);
      const long long o = (long long)wsrc * plane + (long long)vv * Nu + uu;
      const int col = side ? kPipeX0 + Nu : kPipeX0 - 1;
      cp_async_elem(Cd + RT_IDX(row * W + col, 8LL * pb, 62), chiP + o);
      cp_async_elem(Sd + RT_IDX(row * W + col, 8LL * pb, 62), SP + o);
    }
  };
  // ghost intensities of plane wsrc around the strip (as in the linear sweep)
  auto ghost_halo = [&](T *Ibuf, int wsrc, bool whole) {
    if (whole) {
      const int ext = (R + 2) * (Nu + 2);
      for (int idx = threadIdx.x; idx < na * ext; idx += blockDim.x) {
        const int a = idx / ext, r2 = idx - a * ext;
        const int row = r2 / (Nu + 2), col = r2 - row * (Nu + 2);
        ghost_async(Ibuf + RT_IDX(a * pb + row * W + kPipeX0 - 1 + col, 2LL * ib, 63),
                    ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gp, false, col - 1, v0 - 1 + row, wsrc));
      }
      return;
    }
    for (int idx = threadIdx.x; idx < na * 2 * (R + 2); idx += blockDim.x) {
      const int a = idx / (2 * (R + 2)), r2 = idx - a * 2 * (R + 2);
      const int side = r2 / (R + 2), row = r2 - side * (R + 2);
      const int vv = v0 - 1 + row;
      // a periodic u face with v inside the grid: the lagged ghost is the u-face
      // entry (w, v) of the ray's block (the general lookup gives the same address)
      const T *src = (perU && vv >= 0 && vv < Nv)
                         ? Gp + ((long long)f * A.na + P[a].angle) * A.d.gsize + plane + (long long)wsrc * Nv + vv
                         : ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gp, false, side ? Nu : -1, vv, wsrc);
      ghost_async(Ibuf + RT_IDX(a * pb + row * W + (side ? kPipeX0 + Nu : kPipeX0 - 1), 2LL * ib, 64), src);
    }
    const int nrow = (v0 == 0 ? 1 : 0) + (v1 == Nv ? 1 : 0);
    for (int idx = threadIdx.x; idx < na * nrow * Nu; idx += blockDim.x) {
      const int a = idx / (nrow * Nu), r2 = idx - a * nrow * Nu;
      const int which = r2 / Nu, u = r2 - which * Nu;
      const bool lo = (v0 == 0) && (which == 0);
      const int row = lo ? 0 : R + 1;
      // a periodic v face (u inside the grid): the v-face entry (w, u) of the ray's block
      const T *src = perV ? Gp + ((long long)f * A.na + P[a].angle) * A.d.gsize + plane + (long long)Nw * Nv +
                                (long long)wsrc * Nu + u
                          : ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, P[a].angle, Gp, false, u, lo ? -1 : Nv, wsrc);
      ghost_async(Ibuf + RT_IDX(a * pb + row * W + kPipeX0 + u, 2LL * ib, 65), src);
    }
  };
  // outflow intensities of plane wp onto the periodic faces (as in the linear sweep)
  auto ghost_pass = [&](const T *Ibuf, int wp) {
    if (!A.write_ghosts) return;
    const long long gn = (long long)A.d.nf * A.na * A.d.gsize;
    if (perU) {
      for (int idx = threadIdx.x; idx < na * R; idx += blockDim.x) {
        const int a = idx / R, lv = idx - a * R;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        const int col = P[a].su > 0 ? Nu - 1 : 0;
        ghost_store<T>(Gp, Gn, nullptr, RT_IDX(gb + plane + (long long)wp * Nv + v0 + lv, gn, 66),
                       Ibuf[RT_IDX(a * pb + (lv + 1) * W + kPipeX0 + col, 2LL * ib, 67)], false, false);
      }
    }
    if (perV) {
      for (int idx = threadIdx.x; idx < na * Nu; idx += blockDim.x) {
        const int a = idx / Nu, u = idx - a * Nu;
        const int vr = P[a].sv > 0 ? Nv - 1 : 0;
        if (vr < v0 || vr >= v1) continue;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        ghost_store<T>(Gp, Gn, nullptr, RT_IDX(gb + plane + (long long)Nw * Nv + (long long)wp * Nu + u, gn, 68),
                       Ibuf[RT_IDX(a * pb + (vr - v0 + 1) * W + kPipeX0 + u, 2LL * ib, 69)], false, false);
      }
    }
    if (perW && wp == wlast) {
      for (int idx = threadIdx.x; idx < na * R * Nu; idx += blockDim.x) {
        const int a = idx / (R * Nu), r2 = idx - a * R * Nu;
        const int lv = r2 / Nu, u = r2 - lv * Nu;
        const long long gb = ((long long)f * A.na + P[a].angle) * A.d.gsize;
        ghost_store<T>(Gp, Gn, nullptr, RT_IDX(gb + (long long)(v0 + lv) * Nu + u, gn, 70),
                       Ibuf[RT_IDX(a * pb + (lv + 1) * W + kPipeX0 + u, 2LL * ib, 71)], false, false);
      }
    }
  };

  // prologue: planes t = 0 and 1 (or the downwind ghost plane), the upwind ghost
  // plane (slot 3), and the upwind plane's intensities
  const int w0 = sa > 0 ? 0 : Nw - 1;
  stage(w0, 0);
  stage(src_plane(w0 + sa), 1);
  stage(src_plane(w0 - sa), 3);
  ghost_halo(Ib + ib, w0 - sa, true);
  cp_async_commit();
  cp_async_wait_all();
  if (C > 1) cluster.sync();
  else __syncthreads();

  for (int t = 0; t < Nw; ++t) {
    const int w = sa > 0 ? t : Nw - 1 - t;
    T *Icur = Ib + (t & 1) * ib;
    const T *Iprv = Ib + ((t + 1) & 1) * ib;
    const T *Cc = Cr + (t & 3) * pb, *Cu = Cr + ((t + 3) & 3) * pb, *Cn = Cr + ((t + 1) & 3) * pb;
    const T *Sc = Sr + (t & 3) * pb, *Su = Sr + ((t + 3) & 3) * pb, *Sn = Sr + ((t + 1) & 3) * pb;
    // the plane after next (or the downwind ghost plane of the last plane)
    if (t + 2 <= Nw) stage(src_plane(w + 2 * sa), (t + 2) & 3);
    ghost_halo(Icur, w, false);
    cp_async_commit();
    T *Ntop = Ntop0 ? Ntop0 + (t & 1) * ib + top_row * W + kPipeX0 : nullptr;
    T *Nbot = Nbot0 ? Nbot0 + (t & 1) * ib + kPipeX0 : nullptr;
    for (int sidx = threadIdx.x; sidx < R * nseg; sidx += blockDim.x) {
      const int lv = sidx / nseg, seg = sidx - lv * nseg;
      const int u0 = seg * SEG, v = v0 + lv, row = lv + 1;
      const int ncell = min(SEG, Nu - u0);
      // rows v-1, v, v+1, columns u0-1 .. u0+SEG of the previous and next planes
      T cu[3][SEG + 2], su[3][SEG + 2], cn[3][SEG + 2], sn[3][SEG + 2];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int k = 0; k < SEG + 2; ++k) {
          const int o = (row - 1 + r) * W + kPipeX0 - 1 + u0 + k;
          cu[r][k] = Cu[o];
          su[r][k] = Su[o];
          cn[r][k] = Cn[o];
          sn[r][k] = Sn[o];
        }
      }
      T chi0[SEG], S0[SEG], Jacc[SEG], Oacc[SEG];
      T Hm[MOM ? SEG : 1][3], Km[MOM ? SEG : 1][6];
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        chi0[j] = Cc[row * W + kPipeX0 + u0 + j];
        S0[j] = Sc[row * W + kPipeX0 + u0 + j];
        Jacc[j] = T(0);
        Oacc[j] = T(0);
        if (MOM) {
#pragma unroll
          for (int q = 0; q < 3; ++q) Hm[MOM ? j : 0][q] = T(0);
#pragma unroll
          for (int q = 0; q < 6; ++q) Km[MOM ? j : 0][q] = T(0);
        }
      }
      for (int a = 0; a < na; ++a) {
        const AngleParam<T> &p = P[a];
        const T fu = p.wb + p.wd, fv = p.wc + p.wd;   // fractional crossing offsets
        const T tu = p.su > 0 ? -fu : fu, tv = p.sv > 0 ? -fv : fv;
        const T *Ia = Iprv + a * pb + (row - 1) * W + kPipeX0 - 1 + u0;
        T iu[3][SEG + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
          for (int k = 0; k < SEG + 2; ++k) iu[r][k] = Ia[r * W + k];
        }
        T I0[SEG];
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
          T Iq[3][3], Sq[3][3], Cq[3][3], Sdq[3][3], Cdq[3][3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              Iq[r][k] = iu[r][j + k];
              Sq[r][k] = su[r][j + k];
              Cq[r][k] = cu[r][j + k];
              Sdq[r][k] = sn[r][j + k];
              Cdq[r][k] = cn[r][j + k];
            }
          }
          T lam, om;
          I0[j] = quad_update<T>(Iq, Sq, Cq, Sdq, Cdq, S0[j], chi0[j], tu, tv, p.hs, lam, om);
          const T wI = p.wq * I0[j];
          Jacc[j] += wI;
          Oacc[j] += p.wq * om;
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
        T *Io = Icur + a * pb + row * W + kPipeX0 + u0;
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
          if (j < ncell) {
            Io[j] = I0[j];
            if (lv == 0 && Ntop) Ntop[a * pb + u0 + j] = I0[j];
            if (lv == R - 1 && Nbot) Nbot[a * pb + u0 + j] = I0[j];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        if (j < ncell) {
          const long long canon = (long long)(u0 + j) * csu + (long long)v * csv + (long long)w * csw;
          Jout[RT_IDX(canon, cells, 72)] = Jacc[j];
          if (Oout) Oout[RT_IDX(canon, cells, 73)] = Oacc[j];
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
    if (t > 0) ghost_pass(Iprv, w - sa);
    cp_async_wait_all();
    if (C > 1) cluster.sync();
    else __syncthreads();
  }
  ghost_pass(Ib + ((Nw - 1) & 1) * ib, sa > 0 ? Nw - 1 : 0);
}

template <typename T, int AMAX, bool MOM>
static cudaError_t launch_quad_t(const SweepArgs<T> &A, int threads, size_t smem, cudaStream_t s) {
  auto kern = sc_sweep_quad_kernel<T, AMAX, MOM>;
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
cudaError_t launch_sweep_quad(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                              cudaStream_t s) {
  switch (amax) {
    case 1: return moments ? launch_quad_t<T, 1, true>(A, threads, smem, s) : launch_quad_t<T, 1, false>(A, threads, smem, s);
    case 2: return moments ? launch_quad_t<T, 2, true>(A, threads, smem, s) : launch_quad_t<T, 2, false>(A, threads, smem, s);
    case 4: return moments ? launch_quad_t<T, 4, true>(A, threads, smem, s) : launch_quad_t<T, 4, false>(A, threads, smem, s);
    case 8: return moments ? launch_quad_t<T, 8, true>(A, threads, smem, s) : launch_quad_t<T, 8, false>(A, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int AMAX>
static int quad_clusters_t(int cluster, int threads, size_t smem) {
  auto kern = sc_sweep_quad_kernel<T, AMAX, false>;
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
int quad_max_active_clusters(int amax, int cluster, int threads, size_t smem) {
  switch (amax) {
    case 1: return quad_clusters_t<T, 1>(cluster, threads, smem);
    case 2: return quad_clusters_t<T, 2>(cluster, threads, smem);
    case 4: return quad_clusters_t<T, 4>(cluster, threads, smem);
    case 8: return quad_clusters_t<T, 8>(cluster, threads, smem);
    default: return -1;
  }
}

template <typename T>
__global__ void quad_lstar_kernel(Dims d, int ngroups, const T *Opart, double *lstar) {
  const long long n = d.cells * d.nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double om = 0.0;
    for (int p = 0; p < ngroups; ++p) om += (double)Opart[(long long)p * n + i];
    lstar[i] = 1.0 - om;
  }
}

template <typename T>
cudaError_t launch_quad_lstar(const Dims &d, int ngroups, const T *Opart, double *lstar, cudaStream_t s) {
  const long long n = d.cells * d.nf;
  long long b = (n + 255) / 256;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  quad_lstar_kernel<T><<<(int)b, 256, 0, s>>>(d, ngroups, Opart, lstar);
  return cudaGetLastError();
}

template cudaError_t launch_quad_lstar<float>(const Dims &, int, const float *, double *, cudaStream_t);
template cudaError_t launch_quad_lstar<double>(const Dims &, int, const double *, double *, cudaStream_t);
template cudaError_t launch_sweep_quad<float>(const SweepArgs<float> &, int, bool, int, size_t, cudaStream_t);
template cudaError_t launch_sweep_quad<double>(const SweepArgs<double> &, int, bool, int, size_t, cudaStream_t);
template int quad_max_active_clusters<float>(int, int, int, size_t);
template int quad_max_active_clusters<double>(int, int, int, size_t);

}  // namespace rtk
