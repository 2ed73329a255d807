/*
 * TEST INFRASTRUCTURE ONLY -- plain FP64 CPU oracle for one short-characteristics
 * formal solution (Davis, Stone & Jiang 2012, Sec. 3.3).  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load this file's
 * library; the CUDA library never does.
 *
 * What it computes, for one frequency and every angle k of the quadrature:
 *   - cells are swept in the paper's order (Fig. 4): x fastest, then y, then z,
 *     each index running in the direction of the ray (mu_a > 0: ascending);
 *   - at each cell the ray is traced upwind to the face of the dual cell it
 *     crosses first (the axis a minimising d_a/|mu_a|, ties to z, then y, then x),
 *     path length s = d_a/|mu_a|;
 *   - I-, S- and chi- at the crossing point are linear (bilinear on the face)
 *     interpolants of the four face vertices (Sec. 3.3, linear interpolation);
 *   - dtau = (chi- + chi0) s / 2;  E = exp(-dtau);  e0 = 1 - E;
 *     Psi0 = (dtau - e0)/dtau (a Taylor series below dtau = 1e-3); Psi- = e0 - Psi0;
 *     I0 = I- E + Psi- S- + Psi0 S0  (Eq. 20 with the linear form, Psi+ = 0);
 *   - J = sum_k w_k I_k (Eq. 17), Lambda*_ii = sum_k w_k Psi0_k (Sec. 3.4),
 *     H_i = sum_k w_k I_k mu_ik (Eq. 18), K_ij = sum_k w_k I_k mu_ik mu_jk (Eq. 19).
 *
 * Boundaries (Sec. 3.5): a vertex outside the domain is a ghost vertex.  chi and S
 * there are those of the periodic image (periodic axis) or of the adjacent
 * boundary layer (other axes).  I there is, if any out-of-range axis is
 * non-periodic, the boundary value of the first such axis in the order z, y, x
 * (vacuum: 0; thermal: B of the adjacent layer; fixed: the user's array);
 * otherwise the intensity of the periodic image cell from the PREVIOUS formal
 * solution (the lagged ghost, held in G_prev).  The intensity this solution
 * leaves on each periodic outflow face is written to G_next.
 *
 * Array layouts (all double):
 *   cell fields     [nz][ny][nx]
 *   face arrays     x-face [nz][ny], y-face [nz][nx], z-face [ny][nx]
 *   G_prev, G_next  [na][ x-face | y-face | z-face ]
 *   I_fixed         [6 faces: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi][na][face of that axis]
 *   H [3][cells], K [6][cells] ordered xx, yy, zz, xy, xz, yz.
 *
 * In 2D (nz == 1) the z spacing is infinite: no ray crosses a z face and the
 * interpolation on the crossed face is linear in one direction.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { BC_PERIODIC = 0, BC_VACUUM = 1, BC_THERMAL = 2, BC_FIXED = 3 };

typedef struct {
  int n[3];
  double d[3];
  int bc_lo[3], bc_hi[3];
  int two_d;
  long cells;
  long face[3];     /* cells on a face normal to axis a */
  long goff[3];     /* offset of each face inside one angle's ghost block */
  long gsize;       /* ghost block per angle */
} geom;

static long cell_index(const geom *g, int i, int j, int k) {
  return ((long)k * g->n[1] + j) * g->n[0] + i;
}

/* position of cell (i,j,k) on the face normal to axis a */
static long face_index(const geom *g, int a, int i, int j, int k) {
  if (a == 0) return (long)k * g->n[1] + j;
  if (a == 1) return (long)k * g->n[0] + i;
  return (long)j * g->n[0] + i;
}

/* Ghost intensity at vertex c[] (some coordinate out of range). */
static double ghost_I(const geom *g, const int c[3], int angle, int na,
                      const double *B, const double *I_fixed, const double *G_prev) {
  int m[3];
  int oor[3];
  int fixed_axis = -1, fixed_side = 0;
  for (int a = 0; a < 3; ++a) {
    oor[a] = 0;
    m[a] = c[a];
    if (c[a] < 0 || c[a] >= g->n[a]) {
      int side = c[a] < 0 ? 0 : 1;
      int bc = side ? g->bc_hi[a] : g->bc_lo[a];
      oor[a] = 1;
      if (bc == BC_PERIODIC) {
        m[a] = c[a] < 0 ? c[a] + g->n[a] : c[a] - g->n[a];
      } else {
        m[a] = side ? g->n[a] - 1 : 0;
      }
    }
  }
  /* first non-periodic out-of-range axis in the order z, y, x */
  for (int a = 2; a >= 0; --a) {
    if (!oor[a]) continue;
    int side = c[a] < 0 ? 0 : 1;
    int bc = side ? g->bc_hi[a] : g->bc_lo[a];
    if (bc != BC_PERIODIC) { fixed_axis = a; fixed_side = side; break; }
  }
  if (fixed_axis >= 0) {
    int bc = fixed_side ? g->bc_hi[fixed_axis] : g->bc_lo[fixed_axis];
    if (bc == BC_VACUUM) return 0.0;
    if (bc == BC_THERMAL) return B[cell_index(g, m[0], m[1], m[2])];
    /* BC_FIXED */
    long off = 0;
    for (int f = 0; f < 2 * fixed_axis + fixed_side; ++f) off += (long)na * g->face[f / 2];
    return I_fixed[off + (long)angle * g->face[fixed_axis] +
                   face_index(g, fixed_axis, m[0], m[1], m[2])];
  }
  /* all out-of-range axes periodic: lagged intensity of the image cell, read
     from the face of the first out-of-range axis in the order z, y, x */
  for (int a = 2; a >= 0; --a) {
    if (oor[a]) {
      return G_prev[(long)angle * g->gsize + g->goff[a] + face_index(g, a, m[0], m[1], m[2])];
    }
  }
  return 0.0; /* not reached */
}

static int map_field(const geom *g, const int c[3]) {
  int m[3];
  for (int a = 0; a < 3; ++a) {
    m[a] = c[a];
    if (c[a] < 0) m[a] = (g->bc_lo[a] == BC_PERIODIC) ? c[a] + g->n[a] : 0;
    else if (c[a] >= g->n[a]) m[a] = (g->bc_hi[a] == BC_PERIODIC) ? c[a] - g->n[a] : g->n[a] - 1;
  }
  return (int)cell_index(g, m[0], m[1], m[2]);
}

/*
 * One formal solution for one frequency.  Returns 0 on success, -1 on bad input.
 * J, lstar, H, K are overwritten (lstar, H, K may be NULL).  G_next may be NULL.
 * nthreads > 1 splits the angles over OpenMP threads, each with its own
 * accumulators, summed afterwards in thread order.
 */
int orc_formal_solution(int nx, int ny, int nz, double dx, double dy, double dz,
                        const int *bc_lo, const int *bc_hi,
                        int na, const double *mu, const double *wq,
                        const double *chi, const double *S, const double *B,
                        const double *I_fixed, const double *G_prev, double *G_next,
                        double *J, double *lstar, double *H, double *K, int nthreads) {
  geom g;
  g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
  g.d[0] = dx; g.d[1] = dy; g.d[2] = dz;
  g.two_d = (nz == 1);
  for (int a = 0; a < 3; ++a) { g.bc_lo[a] = bc_lo[a]; g.bc_hi[a] = bc_hi[a]; }
  g.cells = (long)nx * ny * nz;
  g.face[0] = (long)nz * ny; g.face[1] = (long)nz * nx; g.face[2] = (long)ny * nx;
  g.goff[0] = 0; g.goff[1] = g.face[0]; g.goff[2] = g.face[0] + g.face[1];
  g.gsize = g.face[0] + g.face[1] + g.face[2];
  if (nx < 1 || ny < 1 || nz < 1 || na < 1) return -1;
  if (nthreads < 1) nthreads = 1;

  const long C = g.cells;
  const int want_mom = (H != NULL) || (K != NULL);
  const int nacc = want_mom ? 11 : 2;   /* J, Lambda* (+ H, K) per thread */
  double *acc = (double *)calloc((size_t)nthreads * C * nacc, sizeof(double));
  double *Iw = (double *)malloc((size_t)nthreads * C * sizeof(double));
  if (!acc || !Iw) { free(acc); free(Iw); return -2; }

#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
  for (int k = 0; k < na; ++k) {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *I = Iw + (long)t * C;
    double *accJ = acc + (long)t * C * nacc;
    double *accL = accJ + C;
    double *accH = accL + C;       /* 3 C */
    double *accK = accH + 3 * C;   /* 6 C */
    const double m[3] = {mu[3 * k], mu[3 * k + 1], mu[3 * k + 2]};
    const double w = wq[k];
    int sgn[3];
    double tpath[3];
    for (int a = 0; a < 3; ++a) {
      sgn[a] = m[a] >= 0.0 ? 1 : -1;
      tpath[a] = (a == 2 && g.two_d) ? INFINITY : g.d[a] / fabs(m[a]);
    }
    /* dominant (first crossed) face: ties go to z, then y, then x */
    int ax = 2;
    if (tpath[1] < tpath[ax]) ax = 1;
    if (tpath[0] < tpath[ax]) ax = 0;
    const double s = tpath[ax];
    /* fractional offsets of the crossing point on the face, per axis */
    double frac[3];
    for (int a = 0; a < 3; ++a) {
      if (a == ax) frac[a] = 1.0;
      else if (a == 2 && g.two_d) frac[a] = 0.0;
      else frac[a] = s * fabs(m[a]) / g.d[a];
    }
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;

    /* paper order: x fastest, then y, then z, each along the ray direction */
    for (int kk = 0; kk < nz; ++kk) {
      const int iz = sgn[2] > 0 ? kk : nz - 1 - kk;
      for (int jj = 0; jj < ny; ++jj) {
        const int iy = sgn[1] > 0 ? jj : ny - 1 - jj;
        for (int ii = 0; ii < nx; ++ii) {
          const int ix = sgn[0] > 0 ? ii : nx - 1 - ii;
          const int c0[3] = {ix, iy, iz};
          const long ci = cell_index(&g, ix, iy, iz);
          double chim = 0.0, Sm = 0.0, Im = 0.0;
          /* the four vertices of the crossed face */
          for (int d1 = 0; d1 < 2; ++d1) {
            for (int d2 = 0; d2 < 2; ++d2) {
              const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) *
                                (d2 ? frac[b2] : 1.0 - frac[b2]);
              if (wv == 0.0) continue;
              int c[3];
              c[ax] = c0[ax] - sgn[ax];
              c[b1] = c0[b1] - d1 * sgn[b1];
              c[b2] = c0[b2] - d2 * sgn[b2];
              const int inside = c[0] >= 0 && c[0] < nx && c[1] >= 0 && c[1] < ny &&
                                 c[2] >= 0 && c[2] < nz;
              const int fi = map_field(&g, c);
              chim += wv * chi[fi];
              Sm += wv * S[fi];
              Im += wv * (inside ? I[cell_index(&g, c[0], c[1], c[2])]
                                 : ghost_I(&g, c, k, na, B, I_fixed, G_prev));
            }
          }
          const double dtau = 0.5 * (chim + chi[ci]) * s;
          const double E = exp(-dtau);
          const double e0 = -expm1(-dtau);
          double psi0;
          if (dtau < 1e-3) {
            psi0 = dtau * (0.5 - dtau * (1.0 / 6.0 - dtau * (1.0 / 24.0 - dtau / 120.0)));
          } else {
            psi0 = (dtau - e0) / dtau;
          }
          const double psim = e0 - psi0;
          const double I0 = Im * E + psim * Sm + psi0 * S[ci];
          I[ci] = I0;
          accJ[ci] += w * I0;
          accL[ci] += w * psi0;
          if (want_mom) {
            for (int a = 0; a < 3; ++a) accH[a * C + ci] += w * I0 * m[a];
            accK[0 * C + ci] += w * I0 * m[0] * m[0];
            accK[1 * C + ci] += w * I0 * m[1] * m[1];
            accK[2 * C + ci] += w * I0 * m[2] * m[2];
            accK[3 * C + ci] += w * I0 * m[0] * m[1];
            accK[4 * C + ci] += w * I0 * m[0] * m[2];
            accK[5 * C + ci] += w * I0 * m[1] * m[2];
          }
          /* periodic outflow faces feed the next solution's ghosts */
          if (G_next) {
            for (int a = 0; a < 3; ++a) {
              if (g.bc_lo[a] != BC_PERIODIC) continue;
              const int out = sgn[a] > 0 ? g.n[a] - 1 : 0;
              if (c0[a] == out)
                G_next[(long)k * g.gsize + g.goff[a] + face_index(&g, a, ix, iy, iz)] = I0;
            }
          }
        }
      }
    }
  }

  /* fixed-order reduction of the per-thread accumulators */
  for (long i = 0; i < C; ++i) {
    double sJ = 0.0, sL = 0.0, sH[3] = {0, 0, 0}, sK[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < nthreads; ++t) {
      const double *a = acc + (long)t * C * nacc;
      sJ += a[i];
      sL += a[C + i];
      if (want_mom) {
        for (int q = 0; q < 3; ++q) sH[q] += a[(2 + q) * C + i];
        for (int q = 0; q < 6; ++q) sK[q] += a[(5 + q) * C + i];
      }
    }
    J[i] = sJ;
    if (lstar) lstar[i] = sL;
    if (H) for (int q = 0; q < 3; ++q) H[q * C + i] = sH[q];
    if (K) for (int q = 0; q < 6; ++q) K[q * C + i] = sK[q];
  }
  free(acc);
  free(Iw);
  return 0;
}

/* Number of OpenMP threads available (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
