// Argument blocks and launchers of the library's kernels (see rt_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "rt_common.cuh"

namespace rtk {

template <typename T>
struct SweepArgs {
  Dims d;
  int na;                    // rays in the full angle table
  const T *chiP[3];          // sweep-precision opacity, permuted per sweep axis, [nf][cells]
  const T *SP[3];            // sweep-precision source function, same layouts
  T *G[2];                   // lagged periodic ghosts [nf][na][gsize], selected by parity
  T *Gd[2];                  // their increments between formal solutions (incremental solves)
  const T *Ibc[6];           // inflow intensity of non-periodic faces [nf][na][face cells]
  const AngleParam<T> *ang;  // rays in group order
  const GroupParam *grp;
  int ngroups;               // groups per frequency
  T *Jpart;                  // [ngroups][nf][cells] canonical
  T *Opart;                  // second-order sweeps: sum_k w_k (1 - dI0/dS0) per group, same layout
  T *Mpart;                  // [ngroups][9][nf][cells] (moments launches only)
  SolveState *st;
  int parity_offset;         // ghost parity = (st->fs_count + parity_offset) & 1
  int write_ghosts;
  int skip_if_done;
  int cluster;               // CTAs per cluster = strips per plane
  int incremental;           // ALI solve sweeping increments after its first formal solution
  int ray_slots;             // shared-memory planes per ray slot (>= rays of any group)
  const T *WE, *WP;          // one-cell-per-thread sweep: E and Psi0 per ray slot and cell,
                             // [slot][nf][w][v][u] of the slot's group (NULL: computed)
  int gs_forward;            // 1: Gauss-Seidel forward phase -- groups crossing the
  int gs_axis;               //    gs_axis face with mu < 0 (the reverse rays) do nothing
  // subdomain (EXTERNAL) z faces, side 0 = low, 1 = high (one-cell-per-thread
  // sweep only): the ghost layer's chi, S and B [nf][ny][nx] and every ray's
  // lagged intensity there [nf][na][ny][nx]; the sweep writes its own
  // intensities on the first / last z plane into xout [nf][na][ny][nx]
  int ext[2];
  const T *xchi[2], *xS[2], *xB[2], *xI[2];
  T *xout[2];
  int jx;                    // 1: the float32 pipelined sweep writes the J partials of
                             //    groups sweeping along x in their plane layout [x][z][y]
                             //    (contiguous rows); consumers must read them so
};

template <typename T>
struct AliArgs {
  Dims d;
  int ngroups_per_f;
  const T *Jpart;            // NULL: J64 already holds this formal solution's J (first iteration)
  int nxg;                   // the first nxg groups' partials are in the [x][z][y] layout (jx)
  const double *eps, *B;
  const double *iden;        // 1 / [eps + (1 - eps)(1 - Lambda*)], fixed for a medium
  const double *ia, *ib;     // (1 - eps) iden and eps B iden (float32 sweeps; NULL = from eps, B)
  const T *Opart;            // second-order sweeps: group partials of 1 - Lambda* of this
                             // formal solution (used instead of iden; NULL = linear)
  double *S64, *Sfs, *J64, *Jprev;
  T *SP[3];                  // permuted sweep copies of S to refresh (NULL = axis unused)
  SolveState *st;
  int lte;
  int incremental;           // partials are increments of J; SP receives dS
  const unsigned char *fmask; // frequencies solved elsewhere (skipped; NULL = none)
};

// Reverse phase of the Gauss-Seidel ALI (rt_gs.cu, Sec. 3.4): the reverse rays
// (crossed face normal to the reverse axis V, mu_V < 0) swept plane by plane from
// the top of V down, each plane's S updated with the freshest J before the next
// plane is swept.  One cooperative launch; the planes are separated by a grid
// barrier whose waits are bounded (on expiry: st->err = kGsBarrierTimeout).
constexpr int kGsMaxRev = 64;          // reverse rays per frequency
constexpr int kGsThreads = 256;
constexpr int kGsBarrierTimeout = 60;
constexpr int kGsBarGroup = 16;         // blocks per first-level barrier counter
constexpr int kGsBarWords = 1 + 256;    // barrier counters (grids of up to 4096 blocks)

template <typename T>
struct GsArgs {
  SweepArgs<T> A;            // grid, ghosts, inflow faces, solve state
  int V;                     // reverse axis (2; 1 in 2D)
  int nrev;                  // reverse rays, A.ang[rev0 .. rev0 + nrev)
  int rev0;
  const int *fgroups;        // the forward groups (their J partials are summed)
  int nfg;
  const double *chi, *eps, *B, *iden;
  double *S64, *Sfs, *J64;
  double *dS;                // [nf][cells] this iteration's change of S
  const double *gsw;         // [nf][9][cells] first-order correction weights
  int incremental;           // after the first iteration, sweep increments (float32 grids):
  double *JF64, *JR64;       //   J of the forward rays and (corrected) of the reverse rays,
                             //   accumulated in FP64 from the swept increments
  T *SPV;                    // sweep copy of S (or dS) along V, [nf][w][v][u]: read for the
                             // plane above and rewritten plane by plane with the new values
  T *Ir;                     // [4][nf][nrev][plane]: intensities or their increments
                             // (2 planes), Psi0, Psi-
  const unsigned char *fmask;
  unsigned *bar;             // grid-barrier counter, zero at launch
  long long poll_limit;      // polls of a barrier wait before it gives up
};

// Correction weights of the forward rays: for each cell and each of the 3 x 3
// cells of the plane above (V + 1), sum over forward rays with an upwind vertex
// there of w Psi- (vertex weight).  `fwd` lists the forward rays with mu_V < 0.
template <typename T>
cudaError_t launch_gs_weights(const Dims &d, int V, const double *chi, const RayGeom *rays,
                              const int *fwd, int nfwd, double *gsw, cudaStream_t s);
template <typename T>
cudaError_t launch_gs_reverse(const GsArgs<T> &G, cudaStream_t s);

// Sets, once per kernel and device, the largest dynamic shared memory the kernel
// may request and permission for non-portable cluster sizes.  The values never
// change afterwards, so launches and occupancy queries from several host threads
// (the request server's workers) cannot race on them.
cudaError_t prepare_kernel(const void *fn);

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                         cudaStream_t s);
// E and Psi0 of every ray of group gi at every cell, as the one-cell-per-thread
// sweep computes them (they depend on chi only), into A.WE / A.WP
template <typename T>
cudaError_t launch_seg_table(const SweepArgs<T> &A, int gi, int nslots, T *WE, T *WP, cudaStream_t s);
// cells per thread of the tiled sweeps
constexpr int kSweepSeg = 4;
// threads per CTA of the tiled and pipelined sweeps: FP64 keeps 256 so that its
// stencils stay in registers
template <typename T>
constexpr int sweep_max_threads() { return sizeof(T) == 8 ? 256 : 512; }
// staged row length of the pipelined sweep: 4 leading columns (halo at 3), Nu
// cells, halo, segment padding, rounded to 16 bytes
__host__ __device__ inline int pipe_row_len(int Nu, int seg) { return ((4 + Nu + 1 + seg + 3) / 4) * 4; }
template <typename T>
cudaError_t launch_sweep_pipe(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                              cudaStream_t s);
// The pipelined sweeps of up to kMultiMax grids in one launch: grid k's
// (group, frequency) instances are clusters base[k] .. base[k+1] - 1.  All grids
// have the same cluster size and the same vectorisation (rows of a multiple of
// 4 cells, or not); passed by value as the kernel's parameter.
constexpr int kMultiMax = 24;
static_assert(sizeof(SweepArgs<double>) * kMultiMax + 4 * (kMultiMax + 2) <= 32764, "kernel parameter limit");
template <typename T>
struct MultiSweep {
  SweepArgs<T> a[kMultiMax];
  int base[kMultiMax + 1];
  int n;
};
template <typename T>
cudaError_t launch_sweep_multi(const MultiSweep<T> &M, int amax, int threads, size_t smem, cudaStream_t s);
// cells per thread of the second-order sweep
constexpr int kQuadSeg = 2;
// second-order sweep (rt_quad.cu): monotonic quadratic face interpolation and
// Bezier-controlled segment integration, chi/S staged in a four-plane ring
template <typename T>
cudaError_t launch_sweep_quad(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                              cudaStream_t s);
template <typename T>
int quad_max_active_clusters(int amax, int cluster, int threads, size_t smem);
// Lambda* of a second-order formal solution: 1 - sum over groups of Opart
template <typename T>
cudaError_t launch_quad_lstar(const Dims &d, int ngroups, const T *Opart, double *lstar, cudaStream_t s);
// clusters of one sweep configuration that can be resident at once (-1 on error)
template <typename T>
int sweep_max_active_clusters(int tiled, int amax, int cluster, int threads, size_t smem);
template <typename T>
cudaError_t launch_sweep_tiled(const SweepArgs<T> &A, int amax, bool moments, int threads, size_t smem,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_ali(const AliArgs<T> &A, cudaStream_t s);
cudaError_t launch_finish(SolveState *st, cudaStream_t s);
// G = (float) Gout, Gd = (float) (Gout - Gin) over n ghost entries
cudaError_t launch_ghosts_from64(long long n, const double *Gout, const double *Gin, float *G, float *Gd,
                                 cudaStream_t s);
cudaError_t launch_f32_to_f64(long long n, const float *src, double *dst, cudaStream_t s);
// iden = 1 / [eps + (1 - eps)(1 - Lambda*)] (the Jacobi denominator of Eq. 24)
// and, where ia is not NULL, the update's factors ia = (1 - eps) iden and
// ib = eps B iden (dS = ia J + ib - S iden)
cudaError_t launch_inv_denominator(long long n, const double *eps, const double *oml, double *iden,
                                   const double *B, double *ia, double *ib, cudaStream_t s);
cudaError_t launch_state_op(SolveState *st, int op, int a, double b, int c, cudaStream_t s);
// xchi[2]: the ghost layers' chi [nf][ny][nx] beyond EXTERNAL z faces (NULL elsewhere)
template <typename T>
cudaError_t launch_lstar(const Dims &d, const double *chi, const RayGeom *rays, int na, double *lstar,
                         double *oml, const double *const xchi[2], cudaStream_t s);
cudaError_t launch_validate(long long n, const double *chi, const double *eps, const double *B,
                            int *counts, cudaStream_t s);
template <typename T>
cudaError_t launch_permute(const Dims &d, const double *src, T *d0, T *d1, T *d2, cudaStream_t s);
template <typename T>
cudaError_t launch_init_ghosts(const Dims &d, int na, const RayGeom *rays, const double *S, T *G,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_fill_bc(const Dims &d, int na, int face, int mode, const double *B,
                           const double *user, T *dst, cudaStream_t s);
template <typename T>
cudaError_t launch_reduce_J(const Dims &d, int ngroups, const T *Jpart, double *J, cudaStream_t s);
template <typename T>
cudaError_t launch_reduce_moments(const Dims &d, int ngroups, const T *Jpart, const T *Mpart,
                                  double *J, double *H, double *K, double *F, int two_d,
                                  cudaStream_t s);
// per frequency: the smallest eps among optically thick cells (1 - Lambda* < 1/2),
// as the bits of a non-negative double (atomicMin); cells with none leave 1.0
cudaError_t launch_eps_thick_min(const Dims &d, const double *eps, const double *oml,
                                 unsigned long long *out, cudaStream_t s);
// heating rate in the integral (0), differential (1) or switched (2) form; H
// [nf][3][cells], h the cell spacings
cudaError_t launch_heating(const Dims &d, const double *fw, const double *chi, const double *eps,
                           const double *J, const double *B, const double *H, const double h[3],
                           int form, double *Q, cudaStream_t s);

}  // namespace rtk
