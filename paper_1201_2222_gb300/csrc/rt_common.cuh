// Internal structures shared by the host side (rt_api.cu) and the kernels
// (rt_kernels.cu) of the short-characteristics library.
//
// Sweep geometry (Davis, Stone & Jiang 2012, Sec. 3.3).  On a uniform grid every
// cell crosses the same upwind face for a given ray: the face normal to the axis
// a minimising d_a/|mu_a|.  All four vertices of that face lie on the previous
// plane along a, so a ray's formal solution is a sequence of planes normal to a,
// each depending only on the one before it.  A sweep group is a set of rays
// sharing (a, sign(mu_a)); its planes are swept together.  Inside a group the
// plane coordinates are (u, v) and the sweep coordinate is w:
//     a = x: (u, v, w) = (y, z, x)     a = y: (x, z, y)     a = z: (x, y, z)
// Sweep-precision copies of chi and S are stored per axis in the permuted
// layout [nf][w][v][u] so that every plane is contiguous.
#pragma once

#include <cstdint>

namespace rtk {

enum { BC_PERIODIC = 0, BC_VACUUM = 1, BC_THERMAL = 2, BC_FIXED = 3, BC_EXTERNAL = 4 };

constexpr int kMaxGroups = 512;

// Per-ray constants in the plane coordinates of its group.
template <typename T>
struct alignas(4 * sizeof(T)) AngleParam {
  T wa, wb, wc, wd; // face weights of vertices (u,v), (u-su,v), (u,v-sv), (u-su,v-sv)
  T hs;             // half the path length to the upwind face, s/2
  T wq;             // quadrature weight w_k
  T mu[3];          // direction cosines (x, y, z) for H and K
  int su, sv;       // sign of mu along u and v
  int angle;        // index in the full angle table
};

static_assert(sizeof(AngleParam<float>) == 48, "AngleParam<float> is read as three float4");

struct GroupParam {
  int axis;   // sweep axis a
  int sa;     // sign of mu_a: +1 sweeps w ascending
  int a0;     // first AngleParam of the group
  int na;     // rays in the group
  // the group's rays are ordered by key = (mu_u > 0) + 2 (mu_v > 0); rays
  // kb[k] .. kb[k+1]-1 (relative to a0) have key k
  int kb[5];
};

// Canonical per-ray geometry (used by the Lambda* kernel).
struct RayGeom {
  double w;
  double s;          // path length to the crossed face
  double frac[3];    // fractional offset on the crossed face per axis (1 on the crossed axis)
  int axis;
  int sgn[3];
};

struct Dims {
  int n[3];          // nx, ny, nz
  int nf;
  long long cells;   // nx*ny*nz
  int periodic[3];   // per canonical axis
  int bc_lo[3], bc_hi[3];
  long long gsize;   // ghost block per (frequency, ray): nx*ny + ny*nz + nx*nz
  long long face[3]; // face cells per canonical axis: x: nz*ny, y: nz*nx, z: ny*nx
};

// Stride of canonical axis a in a [nz][ny][nx] array.
__host__ __device__ inline long long canon_stride(const int n[3], int a) {
  return a == 0 ? 1LL : (a == 1 ? (long long)n[0] : (long long)n[0] * n[1]);
}

// Roles of the canonical axes for a sweep along axis a.
__host__ __device__ inline void plane_axes(int a, int cax[3]) {
  // cax[0] = u, cax[1] = v, cax[2] = w
  if (a == 0) { cax[0] = 1; cax[1] = 2; cax[2] = 0; }
  else if (a == 1) { cax[0] = 0; cax[1] = 2; cax[2] = 1; }
  else { cax[0] = 0; cax[1] = 1; cax[2] = 2; }
}

// Device-resident solve control block.
struct SolveState {
  int fs_count;             // formal solutions since the ghosts were initialised (ghost parity)
  int iter;                 // formal solutions in the current ALI solve
  int done;                 // 1: later kernels of the enqueued batch do nothing
  int converged;            // 1: stopped on tol; 0: stopped on max_iter / running
  int max_iter;
  int lte;                  // all eps == 1: test uses the change of J
  double tol;
  double last_resid;
  unsigned long long resid_bits;   // running max of |dS|/S (non-negative double bits)
  int err;                  // device-side error word (bounds checks in debug builds)
  int err_info;
};

}  // namespace rtk
