// Device helpers shared by the sweep kernels' translation units (rt_kernels.cu,
// rt_quad.cu, rt_gs.cu): checked indexing of debug builds, the ghost-intensity
// lookup and outflow store of the lagged boundary scheme (Sec. 3.5), the linear
// segment weights of Eq. 20, and the asynchronous shared-memory copies of the
// pipelined sweeps.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "rt_common.cuh"
#include "rt_kernels.h"

namespace rtk {

#ifdef RT_DEBUG_BOUNDS
// Debug builds: every indexed access is checked; a bad index is recorded in the
// solve state and replaced by 0 so that no access leaves its buffer.
__device__ __forceinline__ long long chk(long long i, long long n, SolveState *st, int code) {
  if (i < 0 || i >= n) {
    atomicCAS(&st->err, 0, code);
    st->err_info = (int)i;
    return 0;
  }
  return i;
}
#define RT_IDX(i, n, code) chk((i), (n), A.st, (code))
#else
#define RT_IDX(i, n, code) (i)
#endif

// Canonical axis a's entry of a 3-vector, by selects (a runtime index into a
// register array would put the array in local memory).
__device__ __forceinline__ int pick3(const int (&x)[3], int a) { return a == 0 ? x[0] : (a == 1 ? x[1] : x[2]); }
__device__ __forceinline__ int pick3(int x0, int x1, int x2, int a) { return a == 0 ? x0 : (a == 1 ? x1 : x2); }

// Address of the intensity at an upwind vertex outside the domain (plane
// coordinates u, v, w), or nullptr when it is zero (fixed inflow in an
// incremental sweep, whose inflow does not change between formal solutions).
// If any out-of-range axis is non-periodic: the inflow intensity of the first
// such face in the order z, y, x.  Otherwise the image cell's intensity from the
// previous formal solution (lagged periodic ghost), read from the face buffer of
// the first out-of-range axis in the same order.
template <typename T>
__device__ __forceinline__ const T *ghost_ptr(const SweepArgs<T> &A, const int cax[3], int Nu, int Nv,
                                              int Nw, int f, int angle, const T *Gp, bool inc, int u,
                                              int v, int w) {
  // canonical coordinates, picked from the plane coordinates by selects
  const int c0 = cax[0] == 0 ? u : (cax[1] == 0 ? v : w);
  const int c1 = cax[0] == 1 ? u : (cax[1] == 1 ? v : w);
  const int c2 = cax[0] == 2 ? u : (cax[1] == 2 ? v : w);
  const int n0 = A.d.n[0], n1 = A.d.n[1], n2 = A.d.n[2];
  const bool p0 = A.d.periodic[0], p1 = A.d.periodic[1], p2 = A.d.periodic[2];
  const bool o0 = c0 < 0 || c0 >= n0, o1 = c1 < 0 || c1 >= n1, o2 = c2 < 0 || c2 >= n2;
  const int m0 = !o0 ? c0 : (p0 ? (c0 < 0 ? c0 + n0 : c0 - n0) : (c0 < 0 ? 0 : n0 - 1));
  const int m1 = !o1 ? c1 : (p1 ? (c1 < 0 ? c1 + n1 : c1 - n1) : (c1 < 0 ? 0 : n1 - 1));
  const int m2 = !o2 ? c2 : (p2 ? (c2 < 0 ? c2 + n2 : c2 - n2) : (c2 < 0 ? 0 : n2 - 1));
  int fax = -1, fside = 0;   // first non-periodic out-of-range axis in the order z, y, x
  // a vertex past a subdomain (EXTERNAL) z face lies inside the undecomposed
  // domain's z range: there an out-of-range bounded x or y face decides (thermal:
  // B of the ghost layer), else the neighbour's lagged intensity
  const int xs = (o2 && !p2 && A.ext[c2 < 0 ? 0 : 1]) ? (c2 < 0 ? 0 : 1) : -1;
  if (o0 && !p0) { fax = 0; fside = c0 >= n0; }
  if (o1 && !p1) { fax = 1; fside = c1 >= n1; }
  if (o2 && !p2 && xs < 0) { fax = 2; fside = c2 >= n2; }
  if (xs >= 0) {
    const long long f2 = (long long)n0 * n1, fc = (long long)m1 * n0 + m0;
    if (fax >= 0) {
      if (inc || (fside ? A.d.bc_hi[fax] : A.d.bc_lo[fax]) != BC_THERMAL) return nullptr;
      return A.xB[xs] + RT_IDX((long long)f * f2 + fc, (long long)A.d.nf * f2, 61);
    }
    if (inc) return nullptr;
    return A.xI[xs] + RT_IDX(((long long)f * A.na + angle) * f2 + fc, (long long)A.d.nf * A.na * f2, 62);
  }
  if (fax >= 0) {
    if (inc) return nullptr;
    // face cell index: x face [z][y], y face [z][x], z face [y][x]
    const long long fc = fax == 0 ? (long long)m2 * n1 + m1
                                  : (fax == 1 ? (long long)m2 * n0 + m0 : (long long)m1 * n0 + m0);
    const long long fsz = fax == 0 ? A.d.face[0] : (fax == 1 ? A.d.face[1] : A.d.face[2]);
    const long long idx = ((long long)f * A.na + angle) * fsz + fc;
    const T *base = fax == 0 ? A.Ibc[fside] : (fax == 1 ? A.Ibc[2 + fside] : A.Ibc[4 + fside]);
    return base + RT_IDX(idx, (long long)A.d.nf * A.na * fsz, 41);
  }
  const int ax = o2 ? 2 : (o1 ? 1 : 0);
  const int mu_ = pick3(m0, m1, m2, cax[0]), mv_ = pick3(m0, m1, m2, cax[1]), mw_ = pick3(m0, m1, m2, cax[2]);
  const long long gb = ((long long)f * A.na + angle) * A.d.gsize;
  long long off;
  if (ax == cax[2]) off = (long long)mv_ * Nu + mu_;
  else if (ax == cax[0]) off = (long long)Nu * Nv + (long long)mw_ * Nv + mv_;
  else off = (long long)Nu * Nv + (long long)Nw * Nv + (long long)mw_ * Nu + mu_;
  return Gp + RT_IDX(gb + off, (long long)A.d.nf * A.na * A.d.gsize, 42);
}

// Value of the intensity at an out-of-domain upwind vertex (see ghost_ptr).
template <typename T>
__device__ __forceinline__ T ghost_I(const SweepArgs<T> &A, const int cax[3], int Nu, int Nv,
                                     int Nw, int f, int angle, const T *Gp, bool inc, int u, int v,
                                     int w) {
  const T *q = ghost_ptr<T>(A, cax, Nu, Nv, Nw, f, angle, Gp, inc, u, v, w);
  return q ? *q : T(0);
}

// Outflow intensity onto a periodic face for the next formal solution.  Full
// solutions store I; the first one of an incremental solve also stores its
// change against the ghost it replaces; incremental ones store the change and
// advance the full ghost by it.
template <typename T>
__device__ __forceinline__ void ghost_store(const T *Gp, T *Gn, T *Gdn, long long off, T I0, bool inc,
                                            bool emit) {
  if (inc) {
    Gdn[off] = I0;
    Gn[off] = Gp[off] + I0;
  } else {
    if (emit) Gdn[off] = I0 - Gp[off];
    Gn[off] = I0;
  }
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
  if (sizeof(T) == 4) cp_async4(dst, src);
  else cp_async8(dst, src);
}

template <typename T>
__device__ __forceinline__ void ghost_async(T *dst, const T *src) {
  if (src) cp_async_elem(dst, src);
  else *dst = T(0);
}

// ----------------------------------------------------------------- segment weights
// Linear short-characteristics weights for one segment of optical depth dtau:
// E = exp(-dtau), Psi0 = 1 - (1 - E)/dtau (weight of S at the cell), and
// om = 1 - Psi0, all without cancellation: below the threshold Psi0 is the
// Taylor series of 1 - (1 - e^-x)/x = sum_{n>=1} (-1)^(n+1) x^n/(n+1)!.

__device__ __forceinline__ void seg_weights(float dtau, float &E, float &psi0, float &om) {
  E = __expf(-dtau);
  const float q = __fdividef(1.0f - E, dtau);
  const float x = dtau;
  const float ser =
      x * (1.0f / 2 - x * (1.0f / 6 - x * (1.0f / 24 - x * (1.0f / 120 - x * (1.0f / 720 -
      x * (1.0f / 5040 - x * (1.0f / 40320 - x * (1.0f / 362880))))))));
  const bool small = dtau < 0.5f;
  psi0 = small ? ser : 1.0f - q;
  om = small ? 1.0f - ser : q;
}

__device__ __forceinline__ void seg_weights(double dtau, double &E, double &psi0, double &om) {
  E = exp(-dtau);
  if (dtau < 1e-2) {
    const double x = dtau;
    psi0 = x * (1.0 / 2 - x * (1.0 / 6 - x * (1.0 / 24 - x * (1.0 / 120 - x * (1.0 / 720 -
           x * (1.0 / 5040 - x * (1.0 / 40320)))))));
    om = 1.0 - psi0;
  } else {
    om = -expm1(-dtau) / dtau;
    psi0 = 1.0 - om;
  }
}

constexpr int kPipeX0 = 4;   // first interior column of a staged row (16-byte aligned)

// ------------------------------------------------- shared memory by 32-bit address
// Loads and stores with the shared state space spelled out, so that address
// arithmetic stays 32-bit and no access goes through generic addressing.
__device__ __forceinline__ float4 lds128(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
// v = shared word at a where `take` is non-zero (only those lanes access memory)
__device__ __forceinline__ void lds32_if(float &v, unsigned a, unsigned take) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p ld.shared.f32 %0, [%1];\n}"
               : "+f"(v)
               : "r"(a), "r"(take)
               : "memory");
}
__device__ __forceinline__ void sts128(unsigned a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
// address of the same shared-memory offset in cluster CTA `rank`
__device__ __forceinline__ unsigned mapa_rank(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void stc128(unsigned a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// Division by a divisor fixed for a kernel's lifetime, by one high multiply, an
// add and a shift (Granlund & Montgomery 1994): for 0 <= n < 2^31 and d >= 1,
// n / d = (umulhi(n, m) + n) >> l with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
  unsigned m, l, d;
  __host__ __device__ FastDiv() : m(1), l(0), d(1) {}
  __host__ __device__ explicit FastDiv(unsigned dv) : d(dv) {
    l = 0;
    while ((1u << l) < dv) ++l;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - dv)) / dv + 1);
  }
  __device__ __forceinline__ int div(int n) const { return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> l); }
};

// ------------------------------------------------ special-function approximations
// 2^x and 1/x by the special-function unit (flush-to-zero; about 2 ulp).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// A compile-time sign of mu_u or mu_v (selects the interpolation stencil).
template <int V>
using SignC = std::integral_constant<int, V>;

}  // namespace rtk
