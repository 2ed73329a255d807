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

enum { BC_PERIODIC = 0, BC_VACUUM = 1, BC_THERMAL = 2, BC_FIXED = 3, BC_EXTERNAL = 4 };

typedef struct {
  int n[3];
  double d[3];
  int bc_lo[3], bc_hi[3];
  int two_d;
  long cells;
  long face[3];     /* cells on a face normal to axis a */
  long goff[3];     /* offset of each face inside one angle's ghost block */
  long gsize;       /* ghost block per angle */
  /* z faces of kind BC_EXTERNAL (a subdomain face, Sec. 3.5): the ghost layer's
     chi, S and B [ny][nx] and each ray's intensity there [na][ny][nx], supplied
     by the caller (lo = 0, hi = 1); NULL elsewhere */
  const double *xchi[2], *xS[2], *xI[2], *xB[2];
  /* when set, S at a ghost vertex is read from this array (same layout as S)
     instead of S itself: the ghost layers of the start of a Gauss-Seidel
     iteration */
  const double *Sg;
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
  /* A vertex past a subdomain (EXTERNAL) z face lies inside the undecomposed
     domain's z range, so there the z axis does not decide: the x and y faces do
     (as they would in the undecomposed domain), and only when neither of them is
     an out-of-range non-periodic face does the neighbour's intensity apply. */
  int ext_side = -1;
  if (oor[2]) {
    int side = c[2] < 0 ? 0 : 1;
    if ((side ? g->bc_hi[2] : g->bc_lo[2]) == BC_EXTERNAL) ext_side = side;
  }
  /* first non-periodic out-of-range axis in the order z, y, x */
  for (int a = 2; a >= 0; --a) {
    if (!oor[a] || (a == 2 && ext_side >= 0)) continue;
    int side = c[a] < 0 ? 0 : 1;
    int bc = side ? g->bc_hi[a] : g->bc_lo[a];
    if (bc != BC_PERIODIC) { fixed_axis = a; fixed_side = side; break; }
  }
  if (fixed_axis < 0 && ext_side >= 0)
    return g->xI[ext_side][(long)angle * g->face[2] + face_index(g, 2, m[0], m[1], m[2])];
  if (fixed_axis >= 0) {
    int bc = fixed_side ? g->bc_hi[fixed_axis] : g->bc_lo[fixed_axis];
    if (bc == BC_VACUUM) return 0.0;
    if (bc == BC_THERMAL) {
      /* B of the adjacent layer: past an external z face, the neighbour's plane */
      if (ext_side >= 0) return g->xB[ext_side][face_index(g, 2, m[0], m[1], m[2])];
      return B[cell_index(g, m[0], m[1], m[2])];
    }
    /* BC_FIXED (rejected together with an external z face) */
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

/* chi (which = 0) or S (1) at vertex c[]: beyond an external z face, the
   supplied ghost layer at the mapped (x, y); elsewhere the field at map_field */
static double field_value(const geom *g, const int c[3], const double *f, int which) {
  for (int side = 0; side < 2; ++side) {
    const double *const *x = which ? g->xS : g->xchi;
    if (!x[side] || (side ? c[2] < g->n[2] : c[2] >= 0)) continue;
    int m[3] = {c[0], c[1], 0};
    for (int a = 0; a < 2; ++a) {
      if (c[a] < 0) m[a] = (g->bc_lo[a] == BC_PERIODIC) ? c[a] + g->n[a] : 0;
      else if (c[a] >= g->n[a]) m[a] = (g->bc_hi[a] == BC_PERIODIC) ? c[a] - g->n[a] : g->n[a] - 1;
    }
    return x[side][face_index(g, 2, m[0], m[1], 0)];
  }
  if (which && g->Sg) {
    const int inside = c[0] >= 0 && c[0] < g->n[0] && c[1] >= 0 && c[1] < g->n[1] && c[2] >= 0 &&
                       c[2] < g->n[2];
    if (!inside) return g->Sg[map_field(g, c)];
  }
  return f[map_field(g, c)];
}

/*
 * One formal solution for one frequency.  Returns 0 on success, -1 on bad input.
 * J, lstar, H, K are overwritten (lstar, H, K may be NULL).  G_next may be NULL.
 * nthreads > 1 splits the angles over OpenMP threads, each with its own
 * accumulators, summed afterwards in thread order.
 */
int orc_formal_solution_ext(int nx, int ny, int nz, double dx, double dy, double dz,
                            const int *bc_lo, const int *bc_hi,
                            int na, const double *mu, const double *wq,
                            const double *chi, const double *S, const double *B,
                            const double *I_fixed, const double *G_prev, double *G_next,
                            double *J, double *lstar, double *H, double *K, int nthreads,
                            const double *xchi_lo, const double *xS_lo, const double *xI_lo,
                            const double *xB_lo,
                            const double *xchi_hi, const double *xS_hi, const double *xI_hi,
                            const double *xB_hi,
                            double *I_zlo, double *I_zhi, const double *S_ghost) {
  geom g;
  memset(&g, 0, sizeof g);
  g.Sg = S_ghost;
  g.xchi[0] = xchi_lo; g.xS[0] = xS_lo; g.xI[0] = xI_lo; g.xB[0] = xB_lo;
  g.xchi[1] = xchi_hi; g.xS[1] = xS_hi; g.xI[1] = xI_hi; g.xB[1] = xB_hi;
  for (int side = 0; side < 2; ++side) {
    const int bc = side ? bc_hi[2] : bc_lo[2];
    if ((bc == BC_EXTERNAL) != (g.xchi[side] && g.xS[side] && g.xI[side] && g.xB[side])) return -1;
  }
  if (bc_lo[0] == BC_EXTERNAL || bc_hi[0] == BC_EXTERNAL || bc_lo[1] == BC_EXTERNAL ||
      bc_hi[1] == BC_EXTERNAL)
    return -1;   /* subdomain faces are z faces */
  if ((bc_lo[2] == BC_EXTERNAL || bc_hi[2] == BC_EXTERNAL) &&
      (bc_lo[0] == BC_FIXED || bc_hi[0] == BC_FIXED || bc_lo[1] == BC_FIXED || bc_hi[1] == BC_FIXED))
    return -1;   /* a fixed x/y face would need the neighbour's incident intensities */
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
              chim += wv * field_value(&g, c, chi, 0);
              Sm += wv * field_value(&g, c, S, 1);
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
          if (I_zlo && iz == 0) I_zlo[(long)k * g.face[2] + face_index(&g, 2, ix, iy, 0)] = I0;
          if (I_zhi && iz == nz - 1) I_zhi[(long)k * g.face[2] + face_index(&g, 2, ix, iy, 0)] = I0;
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

int orc_formal_solution(int nx, int ny, int nz, double dx, double dy, double dz,
                        const int *bc_lo, const int *bc_hi,
                        int na, const double *mu, const double *wq,
                        const double *chi, const double *S, const double *B,
                        const double *I_fixed, const double *G_prev, double *G_next,
                        double *J, double *lstar, double *H, double *K, int nthreads) {
  return orc_formal_solution_ext(nx, ny, nz, dx, dy, dz, bc_lo, bc_hi, na, mu, wq, chi, S, B,
                                 I_fixed, G_prev, G_next, J, lstar, H, K, nthreads,
                                 NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------
 * Second-order variant (Sec. 3.3): monotonic quadratic interpolation on the
 * crossed face and the second-order (Bezier-controlled parabolic) integration
 * of S along the segment.
 *
 *   - the ray's upwind and downwind points lie on the planes c[a] -/+ 1 of its
 *     crossed axis a, at the fractional offsets -/+ sgn*frac along the two face
 *     axes; each is interpolated from the 3 x 3 face vertices centred on the
 *     cell's own column, along the lower canonical face axis first, then the
 *     other (quad1: the parabola
 *     through three values clamped to the two bracketing ones -- no new
 *     extrema, positivity kept, exact for monotone quadratic data);
 *   - because that stencil reaches the vertex ahead of the ray on the upwind
 *     face, the sweep runs plane by plane along the crossed axis (the paper's
 *     reorientation of the sweep for shallow rays);
 *   - I-, S-, chi- at the upwind point; S+, chi+ at the downwind point (chi and
 *     S there follow the same ghost rules as the upwind side);
 *   - dtau- = (chi- + chi0) s / 2, dtau+ = (chi0 + chi+) s / 2;
 *   - S between the upwind point and the cell is the quadratic Bezier curve with
 *     end values S-, S0 and control value Sc = S0 - (dtau-/2) S'(tau0), S' the
 *     derivative at the cell of the parabola through (S-, S0, S+); Sc is
 *     clamped to [min(S-, S0), max(S-, S0)] (where the parabola would
 *     overshoot);
 *   - I0 = I- exp(-dtau-) + a S- + b S0 + c Sc, with a, b, c the integrals of
 *     the Bernstein polynomials against exp(-(dtau- - t)) (orc_bezier_weights);
 *   - Lambda*_ii = sum_k w_k (b + c dSc/dS0): the local dependence of I0 on S0,
 *     with dSc/dS0 that of the control point limited to [0, 1] (0 or 1 where it
 *     is clamped).  It depends on S through the clamps, so an ALI solve with this
 *     scheme takes Lambda* from each formal solution.
 * ---------------------------------------------------------------------- */

/* a, b, c of I0 = I- e^{-t} + a S- + b S0 + c Sc for a segment of optical depth t:
 * with x the optical distance back from the cell and u = 1 - x/t,
 * a = int (x/t)^2 e^{-x}, b = int (1 - x/t)^2 e^{-x}, c = int 2 (x/t)(1 - x/t) e^{-x},
 * over 0 <= x <= t.  Series in t below 0.1, closed forms above. */
void orc_bezier_weights(double t, double *w3) {
  if (t <= 0.0) { w3[0] = w3[1] = w3[2] = 0.0; return; }
  double m0, m1, m2;   /* m_n = int_0^t x^n e^{-x} dx / t^(n+1) */
  if (t < 0.1) {
    /* m_n = sum_k (-t)^k / (k! (n+k+1)) */
    double p = 1.0, f = 1.0;
    m0 = m1 = m2 = 0.0;
    for (int k = 0; k < 14; ++k) {
      m0 += p / (f * (k + 1));
      m1 += p / (f * (k + 2));
      m2 += p / (f * (k + 3));
      p *= -t;
      f *= (k + 1);
    }
  } else {
    const double E = exp(-t);
    const double E0 = -expm1(-t);
    const double E1 = E0 - t * E;
    const double E2 = 2.0 * E1 - t * t * E;
    m0 = E0 / t;
    m1 = E1 / (t * t);
    m2 = E2 / (t * t * t);
  }
  /* a = t m2, b = t (m0 - 2 m1 + m2), c = 2 t (m1 - m2) */
  w3[0] = t * m2;
  w3[1] = t * (m0 - 2.0 * m1 + m2);
  w3[2] = 2.0 * t * (m1 - m2);
}

/* Monotonic quadratic interpolation of f(-1), f(0), f(1) at t in [-1, 1]: the
 * parabola through the three values, clamped to the range of the two values
 * that bracket t.  No new extrema (positivity kept); exact for quadratic data
 * wherever the parabola is monotone between the bracketing vertices. */
static double quad1(double fm, double f0, double fp, double t) {
  if (t == 0.0) return f0;
  double v = f0 + 0.5 * t * (fp - fm) + 0.5 * t * t * (fp - 2.0 * f0 + fm);
  const double fe = t < 0.0 ? fm : fp;
  const double lo = fe < f0 ? fe : f0, hi = fe < f0 ? f0 : fe;
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}

int orc_formal_solution_quad(int nx, int ny, int nz, double dx, double dy, double dz,
                             const int *bc_lo, const int *bc_hi,
                             int na, const double *mu, const double *wq,
                             const double *chi, const double *S, const double *B,
                             const double *I_fixed, const double *G_prev, double *G_next,
                             double *J, double *lstar, double *H, double *K, int nthreads) {
  geom g;
  memset(&g, 0, sizeof g);
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
  const int nacc = want_mom ? 11 : 2;
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
    double *accH = accL + C;
    double *accK = accH + 3 * C;
    const double m[3] = {mu[3 * k], mu[3 * k + 1], mu[3 * k + 2]};
    const double w = wq[k];
    int sgn[3];
    double tpath[3];
    for (int a = 0; a < 3; ++a) {
      sgn[a] = m[a] >= 0.0 ? 1 : -1;
      tpath[a] = (a == 2 && g.two_d) ? INFINITY : g.d[a] / fabs(m[a]);
    }
    int ax = 2;
    if (tpath[1] < tpath[ax]) ax = 1;
    if (tpath[0] < tpath[ax]) ax = 0;
    const double s = tpath[ax];
    double frac[3];
    for (int a = 0; a < 3; ++a) {
      if (a == ax) frac[a] = 1.0;
      else if (a == 2 && g.two_d) frac[a] = 0.0;
      else frac[a] = s * fabs(m[a]) / g.d[a];
    }
    /* face axes: b1 the lower canonical axis (interpolated first), b2 the higher */
    const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
    /* offsets of the upwind point on its face, in cells along b1, b2 */
    const double t1 = -sgn[b1] * frac[b1], t2 = -sgn[b2] * frac[b2];

    /* planes along the crossed axis in the ray's direction; within a plane any order */
    for (int pa = 0; pa < g.n[ax]; ++pa) {
      const int ia = sgn[ax] > 0 ? pa : g.n[ax] - 1 - pa;
      for (int q2 = 0; q2 < g.n[b2]; ++q2) {
        for (int q1 = 0; q1 < g.n[b1]; ++q1) {
          int c0[3];
          c0[ax] = ia; c0[b1] = q1; c0[b2] = q2;
          const long ci = cell_index(&g, c0[0], c0[1], c0[2]);
          /* 3 x 3 values on the upwind and downwind faces */
          double Iu[3][3], Su[3][3], Cu[3][3], Sd[3][3], Cd[3][3];
          for (int e2 = -1; e2 <= 1; ++e2) {
            for (int e1 = -1; e1 <= 1; ++e1) {
              int c[3];
              c[b1] = c0[b1] + e1;
              c[b2] = c0[b2] + e2;
              c[ax] = c0[ax] - sgn[ax];
              int inside = c[0] >= 0 && c[0] < nx && c[1] >= 0 && c[1] < ny && c[2] >= 0 && c[2] < nz;
              int fi = map_field(&g, c);
              Cu[e2 + 1][e1 + 1] = chi[fi];
              Su[e2 + 1][e1 + 1] = S[fi];
              Iu[e2 + 1][e1 + 1] = inside ? I[cell_index(&g, c[0], c[1], c[2])]
                                          : ghost_I(&g, c, k, na, B, I_fixed, G_prev);
              c[ax] = c0[ax] + sgn[ax];
              fi = map_field(&g, c);
              Cd[e2 + 1][e1 + 1] = chi[fi];
              Sd[e2 + 1][e1 + 1] = S[fi];
            }
          }
          double rI[3], rS[3], rC[3], rSd[3], rCd[3];
          for (int r = 0; r < 3; ++r) {
            rI[r] = quad1(Iu[r][0], Iu[r][1], Iu[r][2], t1);
            rS[r] = quad1(Su[r][0], Su[r][1], Su[r][2], t1);
            rC[r] = quad1(Cu[r][0], Cu[r][1], Cu[r][2], t1);
            rSd[r] = quad1(Sd[r][0], Sd[r][1], Sd[r][2], -t1);
            rCd[r] = quad1(Cd[r][0], Cd[r][1], Cd[r][2], -t1);
          }
          const double Im = quad1(rI[0], rI[1], rI[2], t2);
          const double Sm = quad1(rS[0], rS[1], rS[2], t2);
          const double chim = quad1(rC[0], rC[1], rC[2], t2);
          const double Sp = quad1(rSd[0], rSd[1], rSd[2], -t2);
          const double chip = quad1(rCd[0], rCd[1], rCd[2], -t2);
          const double S0 = S[ci], chi0 = chi[ci];
          const double hm = 0.5 * (chim + chi0) * s, hp = 0.5 * (chi0 + chip) * s;
          double I0, dI0;
          if (hm <= 0.0) {
            I0 = Im;    /* no opacity along the segment */
            dI0 = 0.0;
          } else {
            /* derivative at the cell of the parabola through (-hm, S-), (0, S0), (hp, S+) */
            double dS, ddS;   /* S'(tau0) and its derivative with respect to S0 */
            const double dm = (S0 - Sm) / hm;
            if (hp > 0.0) {
              const double dp = (Sp - S0) / hp;
              dS = (hp * dm + hm * dp) / (hm + hp);
              ddS = (hp / hm - hm / hp) / (hm + hp);
            } else {
              dS = dm;
              ddS = 1.0 / hm;
            }
            double Sc = S0 - 0.5 * hm * dS;
            /* dSc/dS0 for Lambda*: the control point's dependence on S0, limited to
               [0, 1]; where the control point is clamped, that of the bound it took */
            double dSc = 1.0 - 0.5 * hm * ddS;
            if (dSc < 0.0) dSc = 0.0;
            if (dSc > 1.0) dSc = 1.0;
            const double lo = Sm < S0 ? Sm : S0, hi = Sm < S0 ? S0 : Sm;
            if (Sc < lo) { Sc = lo; dSc = (lo == S0) ? 1.0 : 0.0; }
            else if (Sc > hi) { Sc = hi; dSc = (hi == S0) ? 1.0 : 0.0; }
            double w3[3];
            orc_bezier_weights(hm, w3);
            I0 = Im * exp(-hm) + w3[0] * Sm + w3[1] * S0 + w3[2] * Sc;
            dI0 = w3[1] + w3[2] * dSc;
          }
          I[ci] = I0;
          accJ[ci] += w * I0;
          accL[ci] += w * dI0;
          if (want_mom) {
            for (int a = 0; a < 3; ++a) accH[a * C + ci] += w * I0 * m[a];
            accK[0 * C + ci] += w * I0 * m[0] * m[0];
            accK[1 * C + ci] += w * I0 * m[1] * m[1];
            accK[2 * C + ci] += w * I0 * m[2] * m[2];
            accK[3 * C + ci] += w * I0 * m[0] * m[1];
            accK[4 * C + ci] += w * I0 * m[0] * m[2];
            accK[5 * C + ci] += w * I0 * m[1] * m[2];
          }
          if (G_next) {
            for (int a = 0; a < 3; ++a) {
              if (g.bc_lo[a] != BC_PERIODIC) continue;
              const int out = sgn[a] > 0 ? g.n[a] - 1 : 0;
              if (c0[a] == out)
                G_next[(long)k * g.gsize + g.goff[a] + face_index(&g, a, c0[0], c0[1], c0[2])] = I0;
            }
          }
        }
      }
    }
  }

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

/* ------------------------------------------------------------------------
 * Gauss-Seidel ALI (Sec. 3.4, after Trujillo Bueno & Fabiani Bendicho 1995),
 * in its plane-wavefront form.
 *
 * The reverse axis V is z (y in 2D).  The reverse rays are those whose crossed
 * face is the V face (ties with V included) and whose mu_V < 0: their upwind
 * vertices all lie on the plane above.  Every other ray is a forward ray; its
 * formal solution is done beforehand with the old S (J_F below).  Then the
 * planes of V are visited from the top (index n_V - 1) down; at plane k:
 *   1. the reverse rays' intensities at plane k, from the plane above, whose S
 *      is already the new one and whose intensities are already corrected;
 *      S0 of the cell itself is still the old one;
 *   2. J = J_F + C + sum over reverse rays of w I, where C corrects, to first
 *      order, the forward rays' use of the old S of the plane above (its cells
 *      hold their new S now): C = sum over forward rays and over their upwind
 *      vertices on plane k+1 of w Psi- (vertex weight) dS(vertex cell);
 *   3. dS = [(1 - eps) J + eps B - S] / [1 - (1 - eps) Lambda*], S <- S + dS
 *      (Eq. 24 with the freshest J);
 *   4. the reverse rays' intensities at plane k take the change of every S
 *      they used from plane k: I += Psi0 dS(cell) + Psi- (sum of the weights
 *      of upwind vertices whose S is read from a cell of plane k times its dS)
 *      -- the second term only on the top plane of a bounded V axis, whose
 *      ghost layer copies plane k (they are the upwind values of plane k-1 and
 *      the outflow ghosts).
 * At convergence dS = 0, C = 0, and the fixed point is that of the Jacobi
 * iteration.
 *
 * rev      [na]    1 for a reverse ray (rays with rev == 0 are forward rays)
 * J_F      [cells] sum over forward rays of w I, from the old S
 * S        [cells] in: S^n; out: S^{n+1}
 * lstar    [cells] the full Lambda* (all rays)
 * G_prev   ghosts read by the reverse rays (as in orc_formal_solution)
 * G_next   outflow ghosts of the reverse rays are written (other rows untouched)
 * J_out    [cells] the J of step 2;  dS_out [cells];  C_out [cells] or NULL
 * ---------------------------------------------------------------------- */

/* crossed axis (ties to z, then y, then x), path length and face offsets */
static void ray_geometry(const geom *g, const double m[3], int *ax_out, double *s_out,
                         double frac[3], int sgn[3]) {
  double tpath[3];
  for (int a = 0; a < 3; ++a) {
    sgn[a] = m[a] >= 0.0 ? 1 : -1;
    tpath[a] = (a == 2 && g->two_d) ? INFINITY : g->d[a] / fabs(m[a]);
  }
  int ax = 2;
  if (tpath[1] < tpath[ax]) ax = 1;
  if (tpath[0] < tpath[ax]) ax = 0;
  const double s = tpath[ax];
  for (int a = 0; a < 3; ++a) {
    if (a == ax) frac[a] = 1.0;
    else if (a == 2 && g->two_d) frac[a] = 0.0;
    else frac[a] = s * fabs(m[a]) / g->d[a];
  }
  *ax_out = ax;
  *s_out = s;
}

/* the SC segment weights of Eq. 20 (linear): E, Psi0 and Psi- */
static void sc_weights(double dtau, double *E, double *psi0, double *psim) {
  *E = exp(-dtau);
  const double e0 = -expm1(-dtau);
  if (dtau < 1e-3) {
    *psi0 = dtau * (0.5 - dtau * (1.0 / 6.0 - dtau * (1.0 / 24.0 - dtau / 120.0)));
  } else {
    *psi0 = (dtau - e0) / dtau;
  }
  *psim = e0 - *psi0;
}

/* coordinate along axis V of the cell with index fi */
static int plane_of(const geom *g, long fi, int V) {
  if (V == 2) return (int)(fi / ((long)g->n[0] * g->n[1]));
  if (V == 1) return (int)((fi / g->n[0]) % g->n[1]);
  return (int)(fi % g->n[0]);
}

/* 1 if ray k is a reverse ray of the Gauss-Seidel iteration */
int orc_gs_is_reverse(int nz, const double *mu, int k, double dx, double dy, double dz) {
  geom g;
  memset(&g, 0, sizeof g);
  g.two_d = (nz == 1);
  g.d[0] = dx; g.d[1] = dy; g.d[2] = dz;
  const int V = g.two_d ? 1 : 2;
  int ax, sgn[3];
  double s, frac[3];
  ray_geometry(&g, &mu[3 * k], &ax, &s, frac, sgn);
  return ax == V && mu[3 * k + V] < 0.0;
}

int orc_gs_reverse(int nx, int ny, int nz, double dx, double dy, double dz,
                   const int *bc_lo, const int *bc_hi,
                   int na, const double *mu, const double *wq, const int *rev,
                   const double *chi, const double *B, const double *eps, const double *lstar,
                   const double *J_F, double *S, const double *I_fixed,
                   const double *G_prev, double *G_next,
                   double *J_out, double *dS_out, double *C_out) {
  geom g;
  memset(&g, 0, sizeof g);
  g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
  g.d[0] = dx; g.d[1] = dy; g.d[2] = dz;
  g.two_d = (nz == 1);
  for (int a = 0; a < 3; ++a) { g.bc_lo[a] = bc_lo[a]; g.bc_hi[a] = bc_hi[a]; }
  g.cells = (long)nx * ny * nz;
  g.face[0] = (long)nz * ny; g.face[1] = (long)nz * nx; g.face[2] = (long)ny * nx;
  g.goff[0] = 0; g.goff[1] = g.face[0]; g.goff[2] = g.face[0] + g.face[1];
  g.gsize = g.face[0] + g.face[1] + g.face[2];
  if (nx < 1 || ny < 1 || nz < 1 || na < 1) return -1;
  const int V = g.two_d ? 1 : 2;
  const int P0 = 0, P1 = V == 2 ? 1 : 2;   /* the two in-plane axes */
  const long C = g.cells;
  int nrev = 0;
  for (int k = 0; k < na; ++k) nrev += rev[k] != 0;
  double *Ir = (double *)malloc((size_t)(nrev ? nrev : 1) * C * sizeof(double));
  double *Pr = (double *)malloc((size_t)(nrev ? nrev : 1) * C * sizeof(double));
  double *Mr = (double *)malloc((size_t)(nrev ? nrev : 1) * C * sizeof(double));
  if (!Ir || !Pr || !Mr) { free(Ir); free(Pr); free(Mr); return -2; }
  for (long i = 0; i < C; ++i) dS_out[i] = 0.0;

  for (int kk = 0; kk < g.n[V]; ++kk) {
    const int kv = g.n[V] - 1 - kk;
    /* 1. reverse rays on plane kv */
    int r = 0;
    for (int k = 0; k < na; ++k) {
      if (!rev[k]) continue;
      const double *m = &mu[3 * k];
      int ax, sgn[3];
      double s, frac[3];
      ray_geometry(&g, m, &ax, &s, frac, sgn);
      const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
      double *I = Ir + (long)r * C;
      double *Pz = Pr + (long)r * C;
      double *Pm = Mr + (long)r * C;
      for (int q = 0; q < g.n[P1]; ++q) {
        for (int p = 0; p < g.n[P0]; ++p) {
          int c0[3];
          c0[V] = kv; c0[P0] = p; c0[P1] = q;
          const long ci = cell_index(&g, c0[0], c0[1], c0[2]);
          double chim = 0.0, Sm = 0.0, Im = 0.0;
          for (int d1 = 0; d1 < 2; ++d1) {
            for (int d2 = 0; d2 < 2; ++d2) {
              const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) * (d2 ? frac[b2] : 1.0 - frac[b2]);
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
          double E, psi0, psim;
          sc_weights(0.5 * (chim + chi[ci]) * s, &E, &psi0, &psim);
          I[ci] = Im * E + psim * Sm + psi0 * S[ci];
          Pz[ci] = psi0;
          Pm[ci] = psim;
        }
      }
      ++r;
    }
    /* 2.-3. J with the first-order correction, then the update, on plane kv */
    for (int q = 0; q < g.n[P1]; ++q) {
      for (int p = 0; p < g.n[P0]; ++p) {
        int c0[3];
        c0[V] = kv; c0[P0] = p; c0[P1] = q;
        const long ci = cell_index(&g, c0[0], c0[1], c0[2]);
        double corr = 0.0;
        if (kv + 1 < g.n[V]) {
          for (int k = 0; k < na; ++k) {
            if (rev[k]) continue;
            const double *m = &mu[3 * k];
            int ax, sgn[3];
            double s, frac[3];
            ray_geometry(&g, m, &ax, &s, frac, sgn);
            const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
            double chim = 0.0, part = 0.0;
            for (int d1 = 0; d1 < 2; ++d1) {
              for (int d2 = 0; d2 < 2; ++d2) {
                const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) * (d2 ? frac[b2] : 1.0 - frac[b2]);
                if (wv == 0.0) continue;
                int c[3];
                c[ax] = c0[ax] - sgn[ax];
                c[b1] = c0[b1] - d1 * sgn[b1];
                c[b2] = c0[b2] - d2 * sgn[b2];
                const int fi = map_field(&g, c);
                chim += wv * chi[fi];
                if (c[V] == kv + 1) part += wv * dS_out[fi];
              }
            }
            if (part != 0.0) {
              double E, psi0, psim;
              sc_weights(0.5 * (chim + chi[ci]) * s, &E, &psi0, &psim);
              corr += wq[k] * psim * part;
            }
          }
        }
        double JR = 0.0;
        r = 0;
        for (int k = 0; k < na; ++k) {
          if (!rev[k]) continue;
          JR += wq[k] * Ir[(long)r * C + ci];
          ++r;
        }
        const double J = J_F[ci] + corr + JR;
        const double e = eps[ci];
        const double dS = ((1.0 - e) * J + e * B[ci] - S[ci]) / (1.0 - (1.0 - e) * lstar[ci]);
        S[ci] += dS;
        dS_out[ci] = dS;
        J_out[ci] = J;
        if (C_out) C_out[ci] = corr;
      }
    }
    /* 4. the reverse rays' intensities take the changes of the S they read
       from this plane; outflow ghosts */
    r = 0;
    for (int k = 0; k < na; ++k) {
      if (!rev[k]) continue;
      const double *m = &mu[3 * k];
      int ax, sgn[3];
      double s, frac[3];
      ray_geometry(&g, m, &ax, &s, frac, sgn);
      const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
      for (int q = 0; q < g.n[P1]; ++q) {
        for (int p = 0; p < g.n[P0]; ++p) {
          int c0[3];
          c0[V] = kv; c0[P0] = p; c0[P1] = q;
          const long ci = cell_index(&g, c0[0], c0[1], c0[2]);
          double ghost = 0.0;   /* upwind vertices whose S comes from this plane */
          for (int d1 = 0; d1 < 2; ++d1) {
            for (int d2 = 0; d2 < 2; ++d2) {
              const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) * (d2 ? frac[b2] : 1.0 - frac[b2]);
              if (wv == 0.0) continue;
              int c[3];
              c[ax] = c0[ax] - sgn[ax];
              c[b1] = c0[b1] - d1 * sgn[b1];
              c[b2] = c0[b2] - d2 * sgn[b2];
              const int fi = map_field(&g, c);
              if (plane_of(&g, fi, V) == kv) ghost += wv * dS_out[fi];
            }
          }
          const double I0 = Ir[(long)r * C + ci] + Pr[(long)r * C + ci] * dS_out[ci] +
                            Mr[(long)r * C + ci] * ghost;
          Ir[(long)r * C + ci] = I0;
          for (int a = 0; a < 3; ++a) {
            if (g.bc_lo[a] != BC_PERIODIC) continue;
            const int out = sgn[a] > 0 ? g.n[a] - 1 : 0;
            if (c0[a] == out)
              G_next[(long)k * g.gsize + g.goff[a] + face_index(&g, a, c0[0], c0[1], c0[2])] = I0;
          }
        }
      }
      ++r;
    }
  }
  free(Ir);
  free(Pr);
  free(Mr);
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

/* ------------------------------------------------------------------------
 * Gauss-Seidel ALI in the paper's cell order (Sec. 3.4, after Trujillo Bueno
 * & Fabiani Bendicho 1995, generalised to 3D with linear interpolation).
 *
 * The reverse sweep visits the cells one at a time in the reverse of the
 * paper's sweep order: V (z; y in 2D) from the top down, within a plane y
 * descending, within a row x descending -- i.e. by decreasing cell index,
 * starting at the top corner cell (x_N, y_N[, z_N]).  Each visited cell's S is
 * updated at once with Eq. 24 and every later computation uses the new value.
 *
 * Rays split in two sets:
 *   reverse rays: every upwind vertex (of nonzero weight) of a cell has a larger
 *     cell index than the cell, i.e. is visited first.  These are the downward
 *     rays (mu_V < 0) that cross the V face, or cross a face of another axis
 *     while pointing to decreasing index along every axis they move in.  Their
 *     intensities are computed during the reverse sweep, at the visit of each
 *     cell, from the intensities and the current S of its upwind vertices;
 *   forward rays: all others (the upward rays, and downward rays swept against
 *     the reverse order).  Their formal solution is done beforehand with the
 *     old S (J_F).  When a cell m gets its new S, the forward rays' J of the
 *     cells that have m as an upwind vertex is corrected to first order with
 *     weights saved beforehand: for each such vertex, w * wv * [Psi-(n) dS(m)
 *     + E(n) Psi0(m) dS(m)], the change through the interpolated S and through
 *     the interpolated intensity (the outgoing intensity at m, which takes
 *     Psi0(m) dS(m)).  The correction is not transported further.
 * The ghost layers (chi, S and the intensities, lagged or prescribed) are those
 * of the start of the iteration: a ghost vertex's S does not change during the
 * sweep, so only interior vertices carry corrections.  After the update of a
 * cell every ray's intensity there takes Psi0 dS (the outgoing intensities are
 * updated): the reverse rays' downwind cells then see it, and so do the outflow
 * ghosts of the next iteration (periodic faces).
 *
 * At convergence dS = 0, every correction vanishes, and the fixed point is the
 * Jacobi one.
 * ---------------------------------------------------------------------- */

static int setup_geom(geom *g, int nx, int ny, int nz, double dx, double dy, double dz,
                      const int *bc_lo, const int *bc_hi) {
  memset(g, 0, sizeof *g);
  g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
  g->d[0] = dx; g->d[1] = dy; g->d[2] = dz;
  g->two_d = (nz == 1);
  for (int a = 0; a < 3; ++a) { g->bc_lo[a] = bc_lo[a]; g->bc_hi[a] = bc_hi[a]; }
  g->cells = (long)nx * ny * nz;
  g->face[0] = (long)nz * ny; g->face[1] = (long)nz * nx; g->face[2] = (long)ny * nx;
  g->goff[0] = 0; g->goff[1] = g->face[0]; g->goff[2] = g->face[0] + g->face[1];
  g->gsize = g->face[0] + g->face[1] + g->face[2];
  return (nx < 1 || ny < 1 || nz < 1) ? -1 : 0;
}

/* 1 if ray k is a reverse ray of the cell-order Gauss-Seidel sweep */
int orc_gs_cell_is_reverse(int nz, const double *mu, int k, double dx, double dy, double dz) {
  geom g;
  memset(&g, 0, sizeof g);
  g.two_d = (nz == 1);
  g.d[0] = dx; g.d[1] = dy; g.d[2] = dz;
  const int V = g.two_d ? 1 : 2;
  if (mu[3 * k + V] >= 0.0) return 0;
  int ax, sgn[3];
  double s, frac[3];
  ray_geometry(&g, &mu[3 * k], &ax, &s, frac, sgn);
  const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
  for (int d1 = 0; d1 < 2; ++d1) {
    for (int d2 = 0; d2 < 2; ++d2) {
      const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) * (d2 ? frac[b2] : 1.0 - frac[b2]);
      if (wv == 0.0) continue;
      int o[3];
      o[ax] = -sgn[ax];
      o[b1] = -d1 * sgn[b1];
      o[b2] = -d2 * sgn[b2];
      /* visited first: the first nonzero offset in the order z, y, x is positive */
      const int first = o[2] != 0 ? o[2] : (o[1] != 0 ? o[1] : o[0]);
      if (first <= 0) return 0;
    }
  }
  return 1;
}

/* offset slot of a vertex relative to its cell, (dx, dy, dz) in {-1, 0, 1}^3 */
static int off_slot(const int o[3]) { return (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1); }

/* Upwind-vertex data of ray (ax, sgn, frac) at cell c0: chi-, S- (from S), the
   dependence weight of the cell's own S through ghost copies (selfw), and per
   vertex its weight, slot, interior flag and field index. */
typedef struct {
  int nv;
  double wv[4];
  int slot[4], inside[4];
  long fi[4], ci[4];
  int c[4][3];
} upwind;

static void upwind_vertices(const geom *g, int ax, const int sgn[3], const double frac[3],
                            const int c0[3], upwind *u) {
  const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
  u->nv = 0;
  for (int d1 = 0; d1 < 2; ++d1) {
    for (int d2 = 0; d2 < 2; ++d2) {
      const double wv = (d1 ? frac[b1] : 1.0 - frac[b1]) * (d2 ? frac[b2] : 1.0 - frac[b2]);
      if (wv == 0.0) continue;
      int c[3], o[3];
      o[ax] = -sgn[ax];
      o[b1] = -d1 * sgn[b1];
      o[b2] = -d2 * sgn[b2];
      for (int a = 0; a < 3; ++a) c[a] = c0[a] + o[a];
      const int q = u->nv++;
      u->wv[q] = wv;
      u->slot[q] = off_slot(o);
      u->inside[q] = c[0] >= 0 && c[0] < g->n[0] && c[1] >= 0 && c[1] < g->n[1] && c[2] >= 0 &&
                     c[2] < g->n[2];
      u->fi[q] = map_field(g, c);
      u->ci[q] = u->inside[q] ? cell_index(g, c[0], c[1], c[2]) : -1;
      for (int a = 0; a < 3; ++a) u->c[q][a] = c[a];
    }
  }
}

/* Correction weights of the forward rays (fwd[k] != 0), once per medium:
   Wc [27][cells]: for cell n and upwind-vertex slot o, the sum over forward rays
   with an interior vertex there of w wv [Psi-(n) + E(n) Psi0(vertex)]; slots
   of ghost vertices stay 0. */
int orc_gs_cell_weights(int nx, int ny, int nz, double dx, double dy, double dz,
                        const int *bc_lo, const int *bc_hi, int na, const double *mu,
                        const double *wq, const int *fwd, const double *chi, double *Wc) {
  geom g;
  if (setup_geom(&g, nx, ny, nz, dx, dy, dz, bc_lo, bc_hi) != 0 || na < 1) return -1;
  const long C = g.cells;
  double *Dk = (double *)malloc((size_t)C * sizeof(double));
  if (!Dk) return -2;
  for (long i = 0; i < 27 * C; ++i) Wc[i] = 0.0;
  for (int k = 0; k < na; ++k) {
    if (!fwd[k]) continue;
    int ax, sgn[3];
    double s, frac[3];
    ray_geometry(&g, &mu[3 * k], &ax, &s, frac, sgn);
    /* pass 1: D of this ray at every cell; pass 2: the weights */
    for (int pass = 0; pass < 2; ++pass) {
      for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
          for (int ix = 0; ix < nx; ++ix) {
            const int c0[3] = {ix, iy, iz};
            const long ci = cell_index(&g, ix, iy, iz);
            upwind u;
            upwind_vertices(&g, ax, sgn, frac, c0, &u);
            double chim = 0.0;
            for (int q = 0; q < u.nv; ++q) chim += u.wv[q] * chi[u.fi[q]];
            double E, psi0, psim;
            sc_weights(0.5 * (chim + chi[ci]) * s, &E, &psi0, &psim);
            if (pass == 0) {
              Dk[ci] = psi0;
              continue;
            }
            for (int q = 0; q < u.nv; ++q) {
              if (!u.inside[q]) continue;
              Wc[(long)u.slot[q] * C + ci] += wq[k] * u.wv[q] * (psim + E * Dk[u.ci[q]]);
            }
          }
    }
  }
  free(Dk);
  return 0;
}

/*
 * One reverse sweep (one frequency).  rev[k] != 0 marks the reverse rays (the
 * others are forward rays, already solved into J_F and their rows of G_next).
 * S in: S^n, out: S^{n+1} (unchanged when update == 0, a dry run in which dS is
 * taken as 0).  G_next: the reverse rays' rows are written; the forward rays'
 * rows (their outflow from the old S) take D dS of the outflow cell.
 * Outputs per cell: J_out (the J it was updated with), dS_out, JR_out (the
 * reverse rays' part of J), C_out (the forward rays' correction); JR_out and
 * C_out may be NULL.
 */
int orc_gs_cell_reverse(int nx, int ny, int nz, double dx, double dy, double dz,
                        const int *bc_lo, const int *bc_hi,
                        int na, const double *mu, const double *wq, const int *rev,
                        const double *chi, const double *B, const double *eps, const double *lstar,
                        const double *J_F, const double *Wc, double *S, const double *I_fixed,
                        const double *G_prev, double *G_next, int update,
                        double *J_out, double *dS_out, double *JR_out, double *C_out) {
  geom g;
  if (setup_geom(&g, nx, ny, nz, dx, dy, dz, bc_lo, bc_hi) != 0 || na < 1) return -1;
  const long C = g.cells;
  int nrev = 0;
  for (int k = 0; k < na; ++k) nrev += rev[k] != 0;
  double *Ir = (double *)malloc((size_t)(nrev ? nrev : 1) * C * sizeof(double));
  int *rk = (int *)malloc((size_t)(nrev ? nrev : 1) * sizeof(int));
  int *rof = (int *)malloc((size_t)na * sizeof(int));          /* reverse slot of ray k, or -1 */
  double *Dr = (double *)malloc((size_t)(nrev ? nrev : 1) * sizeof(double));
  double *S0 = (double *)malloc((size_t)C * sizeof(double));   /* S of the ghost layers */
  if (!Ir || !rk || !rof || !Dr || !S0) {
    free(Ir); free(rk); free(rof); free(Dr); free(S0);
    return -2;
  }
  memcpy(S0, S, (size_t)C * sizeof(double));
  {
    int r = 0;
    for (int k = 0; k < na; ++k) {
      rof[k] = rev[k] ? r : -1;
      if (rev[k]) rk[r++] = k;
    }
  }
  for (long i = 0; i < C; ++i) dS_out[i] = 0.0;

  for (long ci = C - 1; ci >= 0; --ci) {
    const int c0[3] = {(int)(ci % nx), (int)((ci / nx) % ny), (int)(ci / ((long)nx * ny))};
    /* the reverse rays at this cell, from their upwind vertices (visited first) */
    double JR = 0.0;
    for (int r = 0; r < nrev; ++r) {
      const int k = rk[r];
      int ax, sgn[3];
      double s, frac[3];
      ray_geometry(&g, &mu[3 * k], &ax, &s, frac, sgn);
      upwind u;
      upwind_vertices(&g, ax, sgn, frac, c0, &u);
      double chim = 0.0, Sm = 0.0, Im = 0.0;
      for (int q = 0; q < u.nv; ++q) {
        chim += u.wv[q] * chi[u.fi[q]];
        Sm += u.wv[q] * (u.inside[q] ? S[u.fi[q]] : S0[u.fi[q]]);
        Im += u.wv[q] * (u.inside[q] ? Ir[(long)r * C + u.ci[q]]
                                     : ghost_I(&g, u.c[q], k, na, B, I_fixed, G_prev));
      }
      double E, psi0, psim;
      sc_weights(0.5 * (chim + chi[ci]) * s, &E, &psi0, &psim);
      const double I0 = Im * E + psim * Sm + psi0 * S[ci];
      Ir[(long)r * C + ci] = I0;
      Dr[r] = psi0;
      JR += wq[k] * I0;
    }
    /* the forward rays' first-order correction for the cells already updated */
    double corr = 0.0;
    for (int o = 0; o < 27; ++o) {
      const double wc = Wc[(long)o * C + ci];
      if (wc == 0.0) continue;
      const int c[3] = {c0[0] + o % 3 - 1, c0[1] + (o / 3) % 3 - 1, c0[2] + o / 9 - 1};
      corr += wc * dS_out[map_field(&g, c)];
    }
    const double J = J_F[ci] + corr + JR;
    const double e = eps[ci];
    const double dS = update ? ((1.0 - e) * J + e * B[ci] - S[ci]) / (1.0 - (1.0 - e) * lstar[ci]) : 0.0;
    S[ci] += dS;
    dS_out[ci] = dS;
    J_out[ci] = J;
    if (JR_out) JR_out[ci] = JR;
    if (C_out) C_out[ci] = corr;
    /* every ray's outgoing intensity at this cell takes D dS; outflow ghosts */
    for (int r = 0; r < nrev; ++r) Ir[(long)r * C + ci] += Dr[r] * dS;
    for (int k = 0; k < na; ++k) {
      int ax, sgn[3];
      double s, frac[3];
      ray_geometry(&g, &mu[3 * k], &ax, &s, frac, sgn);
      int on_face = 0;
      for (int a = 0; a < 3; ++a)
        if (g.bc_lo[a] == BC_PERIODIC && c0[a] == (sgn[a] > 0 ? g.n[a] - 1 : 0)) on_face = 1;
      if (!on_face) continue;
      const int r = rof[k];
      double dI = 0.0;
      if (r < 0 && dS != 0.0) {
        upwind u;
        upwind_vertices(&g, ax, sgn, frac, c0, &u);
        double chim = 0.0;
        for (int q = 0; q < u.nv; ++q) chim += u.wv[q] * chi[u.fi[q]];
        double E, psi0, psim;
        sc_weights(0.5 * (chim + chi[ci]) * s, &E, &psi0, &psim);
        dI = psi0 * dS;
      }
      for (int a = 0; a < 3; ++a) {
        if (g.bc_lo[a] != BC_PERIODIC) continue;
        if (c0[a] != (sgn[a] > 0 ? g.n[a] - 1 : 0)) continue;
        double *gp = &G_next[(long)k * g.gsize + g.goff[a] + face_index(&g, a, c0[0], c0[1], c0[2])];
        if (r >= 0) *gp = Ir[(long)r * C + ci];
        else *gp += dI;
      }
    }
  }
  free(Ir);
  free(rk);
  free(rof);
  free(Dr);
  free(S0);
  return 0;
}
