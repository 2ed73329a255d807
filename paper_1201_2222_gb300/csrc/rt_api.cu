// Host side of the C ABI declared in include/rt_sc.h.
//
// Owns the grid's device state, builds the angle quadrature and the sweep
// groups, and enqueues the kernels of rt_kernels.cu.  Every numerical step runs
// on the GPU; this file only plans, allocates, copies and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <climits>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "rt_common.cuh"
#include "rt_kernels.h"
#include "rt_lockstep.h"
#include "rt_sc.h"

using rtk::AngleParam;
using rtk::GroupParam;
using rtk::RayGeom;

namespace {

thread_local std::string g_err = "no error";

}  // namespace

// Records the calling thread's error message for rt_last_error (used by the
// request server's translation unit); returns st.
rt_status rt_internal_error(rt_status st, const char *msg) {
  g_err = msg;
  return st;
}

namespace {

rt_status fail(rt_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,         \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// ------------------------------------------------------------------ quadrature
// Level-symmetric LQ_n set (Sec. 3.2 constraints: octant-identical, invariant under
// 90-degree rotations).  Levels mu_i^2 = a + (i-1) 2(1-3a)/(n_mu-2); octant nodes
// (i, j, l) with i + j + l = n_mu/2 + 2; permutation classes share a weight; a and
// the class weights satisfy sum w = 1 and sum w mu_z^(2p) = 1/(2p+1),
// p = 2 .. n_classes + 1 (one more equation than weights: a is where they agree).

struct LQSystem {
  int nc;
  std::vector<std::array<int, 3>> nodes;
  std::vector<int> node_class;
};

LQSystem lq_structure(int n_mu) {
  LQSystem s;
  const int half = n_mu / 2;
  std::vector<std::array<int, 3>> classes;
  for (int i = 1; i <= half; ++i)
    for (int j = 1; j <= half; ++j) {
      const int l = half + 2 - i - j;
      if (l >= 1) s.nodes.push_back({i, j, l});
    }
  for (auto n : s.nodes) {
    std::array<int, 3> c = n;
    std::sort(c.begin(), c.end());
    if (std::find(classes.begin(), classes.end(), c) == classes.end()) classes.push_back(c);
  }
  std::sort(classes.begin(), classes.end());
  for (auto n : s.nodes) {
    std::array<int, 3> c = n;
    std::sort(c.begin(), c.end());
    s.node_class.push_back((int)(std::find(classes.begin(), classes.end(), c) - classes.begin()));
  }
  s.nc = (int)classes.size();
  return s;
}

// rows: [count | moments p = 2..nc+1], columns: classes, plus the right-hand side
void lq_rows(const LQSystem &s, int n_mu, double a, std::vector<double> &M, std::vector<double> &b) {
  const int nc = s.nc, half = n_mu / 2;
  std::vector<double> mu2(half);
  for (int i = 0; i < half; ++i) mu2[i] = a + i * 2.0 * (1.0 - 3.0 * a) / (n_mu - 2);
  M.assign((nc + 1) * nc, 0.0);
  b.assign(nc + 1, 0.0);
  for (size_t q = 0; q < s.nodes.size(); ++q) {
    const int c = s.node_class[q];
    M[0 * nc + c] += 1.0;
    for (int p = 2; p <= nc + 1; ++p) M[(p - 1) * nc + c] += std::pow(mu2[s.nodes[q][2] - 1], p);
  }
  b[0] = 1.0;
  for (int p = 2; p <= nc + 1; ++p) b[p - 1] = 1.0 / (2 * p + 1);
}

// determinant (and optional solve) by Gaussian elimination with partial pivoting
double gauss(std::vector<double> A, int n, std::vector<double> *rhs) {
  double det = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) return 0.0;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      if (rhs) std::swap((*rhs)[k], (*rhs)[piv]);
      det = -det;
    }
    det *= A[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double m = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
      if (rhs) (*rhs)[i] -= m * (*rhs)[k];
    }
  }
  if (rhs) {
    for (int i = n - 1; i >= 0; --i) {
      double s = (*rhs)[i];
      for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * (*rhs)[j];
      (*rhs)[i] = s / A[i * n + i];
    }
  }
  return det;
}

double lq_consistency(const LQSystem &s, int n_mu, double a) {
  std::vector<double> M, b;
  lq_rows(s, n_mu, a, M, b);
  const int n = s.nc + 1;
  std::vector<double> Aug(n * n);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < s.nc; ++j) Aug[i * n + j] = M[i * s.nc + j];
    Aug[i * n + s.nc] = b[i];
  }
  return gauss(Aug, n, nullptr);
}

// weights at a consistent a: the square subsystem (one row dropped) with the largest |det|
bool lq_weights(const LQSystem &s, int n_mu, double a, std::vector<double> &w) {
  std::vector<double> M, b;
  lq_rows(s, n_mu, a, M, b);
  const int nc = s.nc;
  double best = -1.0;
  for (int drop = 0; drop <= nc; ++drop) {
    std::vector<double> A, r;
    for (int i = 0; i <= nc; ++i) {
      if (i == drop) continue;
      for (int j = 0; j < nc; ++j) A.push_back(M[i * nc + j]);
      r.push_back(b[i]);
    }
    const double d = std::fabs(gauss(A, nc, nullptr));
    if (d > best) {
      best = d;
      gauss(A, nc, &r);
      w = r;
    }
  }
  for (int i = 0; i <= nc; ++i) {
    double s2 = 0.0;
    for (int j = 0; j < nc; ++j) s2 += M[i * nc + j] * w[j];
    if (std::fabs(s2 - b[i]) > 1e-12) return false;
  }
  for (double x : w)
    if (!(x > 0.0)) return false;
  return true;
}

bool level_symmetric(int n_mu, bool two_d, std::vector<double> &mu, std::vector<double> &wq) {
  std::vector<std::array<double, 3>> omu;
  std::vector<double> ow;
  if (n_mu == 2) {
    const double m = 1.0 / std::sqrt(3.0);
    omu.push_back({m, m, m});
    ow.push_back(1.0);
  } else {
    if (n_mu < 4 || n_mu > 12 || (n_mu & 1)) return false;
    const LQSystem s = lq_structure(n_mu);
    const int nscan = 4001;
    const double lo = 1e-6, hi = 1.0 / 3.0 - 1e-6;
    double a_prev = lo, f_prev = lq_consistency(s, n_mu, lo);
    bool found = false;
    double a_root = 0.0;
    std::vector<double> wcls;
    for (int k = 1; k < nscan && !found; ++k) {
      const double a = lo + (hi - lo) * k / (nscan - 1);
      const double fa = lq_consistency(s, n_mu, a);
      if (f_prev == 0.0 || f_prev * fa < 0.0) {
        double x0 = a_prev, x1 = a, f0 = f_prev;
        for (int it = 0; it < 200 && x1 - x0 > 0.0; ++it) {
          const double xm = 0.5 * (x0 + x1);
          if (xm <= x0 || xm >= x1) break;
          const double fm = lq_consistency(s, n_mu, xm);
          if ((fm < 0) == (f0 < 0) && fm != 0.0) { x0 = xm; f0 = fm; }
          else x1 = xm;
        }
        const double r = f0 == 0.0 ? x0 : 0.5 * (x0 + x1);
        std::vector<double> w;
        if (lq_weights(s, n_mu, r, w)) {
          bool pos = true;
          for (int i = 0; i < n_mu / 2; ++i)
            if (!(r + i * 2.0 * (1.0 - 3.0 * r) / (n_mu - 2) > 0.0)) pos = false;
          if (pos) { found = true; a_root = r; wcls = w; }
        }
      }
      a_prev = a;
      f_prev = fa;
    }
    if (!found) return false;
    const int half = n_mu / 2;
    std::vector<double> lev(half);
    for (int i = 0; i < half; ++i) lev[i] = std::sqrt(a_root + i * 2.0 * (1.0 - 3.0 * a_root) / (n_mu - 2));
    for (size_t q = 0; q < s.nodes.size(); ++q) {
      omu.push_back({lev[s.nodes[q][0] - 1], lev[s.nodes[q][1] - 1], lev[s.nodes[q][2] - 1]});
      ow.push_back(wcls[s.node_class[q]]);
    }
  }
  mu.clear();
  wq.clear();
  for (int o = 0; o < 8; ++o) {
    const double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
    if (two_d && sz < 0) continue;
    for (size_t q = 0; q < omu.size(); ++q) {
      mu.push_back(sx * omu[q][0]);
      mu.push_back(sy * omu[q][1]);
      mu.push_back(sz * omu[q][2]);
      wq.push_back(ow[q] / 8.0 * (two_d ? 2.0 : 1.0));
    }
  }
  return true;
}

}  // namespace

// ------------------------------------------------------------------------ grid

struct rt_grid_s {
  rt_grid_desc desc{};
  int device = 0;
  rtk::Dims d{};
  bool two_d = false;
  int na = 0;
  std::vector<double> mu, wq;
  std::vector<RayGeom> rays;
  int used_axis[3] = {0, 0, 0};
  size_t tsize = 8;

  // sweep plan
  int apg = 0, amax = 1, cluster = 1, threads = 256, slots = 1, variant = 1;
  size_t smem = 0;
  int req_apg = 0, req_cluster = 0, req_threads = 0, req_variant = 0;
  std::vector<GroupParam> groups;
  std::vector<int> group_angles;   // angle index per AngleParam slot

  // device buffers
  double *chi = nullptr, *eps = nullptr, *B = nullptr, *fw = nullptr;
  double *S = nullptr, *Sfs = nullptr, *J = nullptr, *Jprev = nullptr;
  double *lstar = nullptr, *oml = nullptr, *iden = nullptr;
  double *ia = nullptr, *ib = nullptr;   // mixed grids: (1 - eps) iden, eps B iden
  void *chiP[3] = {nullptr, nullptr, nullptr};
  void *SP[3] = {nullptr, nullptr, nullptr};
  void *G[2] = {nullptr, nullptr};
  void *Gd[2] = {nullptr, nullptr};   // ghost increments (mixed-precision incremental solves)
  void *Ibc[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *user_bc[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void *Jpart = nullptr;
  size_t jpart_groups = 0;
  void *Mpart = nullptr;
  size_t mpart_groups = 0;
  void *angp = nullptr;
  GroupParam *grp = nullptr;
  RayGeom *rays_d = nullptr;
  rtk::SolveState *st = nullptr;
  int *counts = nullptr;
  double *tmp = nullptr;           // scratch for host-side outputs
  size_t tmp_n = 0;
  cudaStream_t own = nullptr;

  bool have_medium = false;
  bool lte = false;
  int fs_total = 0;                // formal solutions since the ghosts were initialised
  bool last_fs_from_Sfs = false;   // the latest formal solution used Sfs (ALI) or S
  bool last_incremental = false;   // the latest solve accumulated J from swept increments
  bool sp_is_delta = false;        // the sweep copies of S hold the last increment

  bool timing = false;
  rt_stats stats{};
  long long launches = 0;

  // Mixed grids do the first formal solution of each Jacobi ALI solve in FP64,
  // on this internal FP64 grid of every bin (the shadow: same medium, no Lambda*
  // of its own); the later sweeps carry increments, whose float32 rounding
  // scales with the update, and J is accumulated in FP64
  rt_grid first64 = nullptr;
  bool fp64_first = false;
  // ... and, whenever the largest relative change of S has fallen by this factor
  // since the last FP64 formal solution, one more iteration in FP64 from the
  // current S, whose J replaces the accumulated one (0: none after the first)
  double anchor_drop = 1e-2;
  bool shadow = false;                // this grid is another grid's FP64 first-solution shadow
  bool stepped = false;               // an ALI solve begun by rt_ali_begin may be continued
  // Mixed grids: frequency bins too ill-conditioned for float32 even as
  // increments after an FP64 first formal solution (unit roundoff over the
  // smallest eps of optically thick cells above bin_limit) are solved by an
  // internal FP64 grid of those bins and masked out of this grid's ALI update
  rt_grid sub64 = nullptr;
  std::vector<int> bins64;
  unsigned char *fmask = nullptr;
  unsigned long long *epsmin = nullptr;
  double *tmp2 = nullptr;
  size_t tmp2_n = 0;
  double bin_limit = 5e-4;
  // Subdomain (RT_BC_EXTERNAL) z faces, FP64 grids, side 0 = low, 1 = high: the
  // ghost layers set by rt_set_external_face (chi, S, B [nf][ny][nx], every ray's
  // lagged intensity [nf][na][ny][nx]) and the intensities the sweeps leave on
  // the first / last z plane for the neighbours [nf][na][ny][nx]
  double *xchi[2] = {nullptr, nullptr}, *xS[2] = {nullptr, nullptr}, *xB[2] = {nullptr, nullptr};
  double *xI[2] = {nullptr, nullptr}, *xout[2] = {nullptr, nullptr};
  int heat_form = RT_HEAT_INTEGRAL;   // form of Q returned by rt_moments (Sec. 4)
  int interp = RT_INTERP_LINEAR;      // order of the face interpolation (Sec. 3.3)
  void *Opart = nullptr;              // second-order sweeps: group partials of 1 - Lambda*
  size_t opart_groups = 0;

  // Gauss-Seidel iteration (rt_set_iteration): correction weights [nf][9][cells],
  // the reverse kernel's intensity / weight planes, its barrier counter and the
  // forward group and ray lists
  int iteration = RT_ITER_JACOBI;
  double *gsw = nullptr;
  bool gs_ready = false;              // gsw matches the medium and the rays
  void *gsIr = nullptr;
  size_t gsIr_bytes = 0;
  unsigned *gs_bar = nullptr;
  int *gs_list = nullptr;             // forward groups, then forward rays with mu_V < 0
  size_t gs_list_n = 0;
  long long gs_polls = 1LL << 22;     // polls of a reverse-phase barrier wait before it gives up
  double *gs_acc = nullptr;           // incremental solves: J of the forward and of the reverse
                                      // rays [2][nf][cells]

  // CUDA graphs of ALI batches (the launches of m iterations, replayed as one
  // graph); keyed by m, the scheme and the generation of the captured arguments
  struct Graph {
    long long gen;
    int m, gs, inc;
    long long nlaunch;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  long long gen = 0;                  // bumped whenever a captured pointer or plan may change
  bool graphs_ok = true;              // false once a capture failed on this grid
  // FP64 grids, one-cell-per-thread sweep: E and Psi0 per ray slot and cell,
  // [2][slots][nf][cells], tabulated for the medium and plan of generation wt_gen
  void *wt = nullptr;
  size_t wt_bytes = 0;
  long long wt_gen = -1;
  bool wt_off = false;                // the table did not fit in device memory
  long long graph_launches = 0;
};

namespace {

cudaStream_t pick_stream(rt_grid g, const rt_solve_opts *o) {
  return (o && o->stream) ? (cudaStream_t)o->stream : g->own;
}

long long N_of(rt_grid g) { return g->d.cells * g->d.nf; }

void build_rays(rt_grid g) {
  const double *dd = &g->desc.dx;
  int count[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  g->rays.resize(g->na);
  for (int a = 0; a < 3; ++a) g->used_axis[a] = 0;
  std::vector<std::array<double, 3>> tt(g->na);
  std::vector<int> tied(g->na, 0);   // bit a: the ray may sweep along a
  const int V = g->two_d ? 1 : 2;
  auto cls = [&](int k, int a) -> int & { return count[a][g->rays[k].sgn[a] > 0 ? 0 : 1]; };
  for (int k = 0; k < g->na; ++k) {
    RayGeom r{};
    const double *m = &g->mu[3 * k];
    double *t = tt[k].data();
    for (int a = 0; a < 3; ++a) {
      r.sgn[a] = m[a] >= 0.0 ? 1 : -1;
      t[a] = (a == 2 && g->two_d) ? std::numeric_limits<double>::infinity() : dd[a] / std::fabs(m[a]);
    }
    g->rays[k] = r;
    const double tmin = std::min(t[0], std::min(t[1], t[2]));
    // first-crossed face; a tie (the ray leaves through an edge) gives identical
    // interpolants on either face, so tied rays go to the least-loaded sweep group
    // -- except under Gauss-Seidel, where a ray tied with the reverse axis V is a
    // V ray (its upwind vertices all lie on the plane of V it comes from)
    int best = -1;
    for (int a = 2; a >= 0; --a) {
      if (t[a] != tmin) continue;
      if (best < 0 || cls(k, a) < cls(k, best)) best = a;
    }
    if (g->iteration == RT_ITER_GAUSS_SEIDEL && t[V] == tmin) {
      best = V;
    } else {
      for (int a = 0; a < 3; ++a)
        if (t[a] == tmin) tied[k] |= 1 << a;
    }
    g->rays[k].axis = best;
    cls(k, best)++;
  }
  // the greedy choice in angle order can leave the classes uneven (and with odd
  // counts, whose groups then hold a ray fewer): move tied rays from a class to
  // one of their other classes holding at least two rays fewer, until none can
  // (each move lowers the sum of squared class sizes, so this ends)
  for (bool moved = true; moved;) {
    moved = false;
    for (int k = 0; k < g->na; ++k) {
      if (__builtin_popcount(tied[k]) < 2) continue;
      const int a = g->rays[k].axis;
      for (int b = 0; b < 3; ++b) {
        if (b == a || !(tied[k] >> b & 1) || cls(k, a) - cls(k, b) < 2) continue;
        cls(k, a)--;
        cls(k, b)++;
        g->rays[k].axis = b;
        moved = true;
        break;
      }
    }
  }
  for (int k = 0; k < g->na; ++k) {
    RayGeom &r = g->rays[k];
    const double *m = &g->mu[3 * k];
    const int best = r.axis;
    r.s = tt[k][best];
    r.w = g->wq[k];
    for (int a = 0; a < 3; ++a) {
      if (a == best) r.frac[a] = 1.0;
      else if (a == 2 && g->two_d) r.frac[a] = 0.0;
      else r.frac[a] = std::min(1.0, r.s * std::fabs(m[a]) / dd[a]);
    }
    g->used_axis[best] = 1;
  }
}

// Largest dynamic shared memory a sweep CTA may use.
constexpr size_t kSweepSmemBudget = 200 * 1024;
constexpr int kSMs = 152;

int amax_for(int apg) { return apg <= 1 ? 1 : (apg <= 2 ? 2 : (apg <= 4 ? 4 : 8)); }

// Largest CTA of a sweep variant in the grid's precision.
int sweep_thread_cap(rt_grid g, int variant) {
  if (variant == 1) return 512;
  return g->desc.prec == RT_PREC_FP64 ? rtk::sweep_max_threads<double>() : rtk::sweep_max_threads<float>();
}

// Shared memory and threads of one sweep CTA for `slots` rays and C strips.
void sweep_shape(rt_grid g, int variant, int slots, int C, size_t *smem, int *threads) {
  size_t sm = 0;
  int th = 0;
  for (int a = 0; a < 3; ++a) {
    if (!g->used_axis[a]) continue;
    int cax[3];
    rtk::plane_axes(a, cax);
    const int Nu = g->d.n[cax[0]];
    const int Rmax = (g->d.n[cax[1]] + C - 1) / C;
    if (variant == 3) {
      // two intensity planes per ray; chi and S rings of 3 planes (4 for the
      // second-order sweep, which also reads the downwind plane)
      const int seg = g->interp == RT_INTERP_QUADRATIC ? rtk::kQuadSeg : rtk::kSweepSeg;
      const size_t W = (size_t)rtk::pipe_row_len(Nu, seg);
      const size_t ring = g->interp == RT_INTERP_QUADRATIC ? 8 : 6;
      // plus, for the linear sweep, two buffers of prefetched ghosts per ray slot
      const size_t pre = g->interp == RT_INTERP_QUADRATIC ? 0 : (size_t)2 * slots * (Rmax + Nu);
      sm = std::max(sm, ((size_t)(2 * slots + ring) * (Rmax + 2) * W + pre) * g->tsize);
      th = std::max(th, Rmax * ((Nu + seg - 1) / seg));
    } else if (variant == 2) {
      const size_t W = (size_t)Nu + 2 + rtk::kSweepSeg;
      sm = std::max(sm, (size_t)(2 * slots + 4) * (Rmax + 2) * W * g->tsize);
      th = std::max(th, Rmax * ((Nu + rtk::kSweepSeg - 1) / rtk::kSweepSeg));
    } else {
      sm = std::max(sm, (size_t)2 * slots * Rmax * Nu * g->tsize);
      th = std::max(th, Rmax * Nu);
    }
  }
  *smem = sm;
  // tasks of a plane spread evenly: the fewest passes the thread cap allows, and
  // the fewest threads that finish the plane in that many passes
  const int cap = sweep_thread_cap(g, variant);
  const int passes = std::max(1, (th + cap - 1) / cap);
  const int per = (th + passes - 1) / passes;
  *threads = std::max(32, std::min(cap, ((per + 31) / 32) * 32));
}

// Split each (crossed axis, direction) class of rays into chunks of <= apg.
void make_groups(rt_grid g, int apg, std::vector<GroupParam> &groups, std::vector<int> &gang, int *namax) {
  std::vector<int> per_key[6];
  for (int k = 0; k < g->na; ++k) {
    const RayGeom &r = g->rays[k];
    per_key[2 * r.axis + (r.sgn[r.axis] > 0 ? 0 : 1)].push_back(k);
  }
  groups.clear();
  gang.clear();
  *namax = 0;
  for (int key = 0; key < 6; ++key) {
    auto &v = per_key[key];
    if (v.empty()) continue;
    // order by the signs of mu along the plane axes, so that each group holds
    // runs of rays sharing one interpolation stencil
    int cax[3];
    rtk::plane_axes(key / 2, cax);
    auto skey = [&](int k) {
      const RayGeom &r = g->rays[k];
      return (r.sgn[cax[0]] > 0 ? 1 : 0) + (r.sgn[cax[1]] > 0 ? 2 : 0);
    };
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return skey(x) < skey(y); });
    const int nchunk = ((int)v.size() + apg - 1) / apg;
    size_t pos = 0;
    for (int c = 0; c < nchunk; ++c) {
      const int sz = (int)(v.size() - pos) / (nchunk - c);
      GroupParam gp{};
      gp.axis = key / 2;
      gp.sa = (key % 2) ? -1 : 1;
      gp.a0 = (int)gang.size();
      gp.na = sz;
      for (int q = 0; q < sz; ++q) gang.push_back(v[pos + q]);
      for (int k = 0; k <= 4; ++k) {   // first ray with stencil key >= k
        int q = 0;
        while (q < sz && skey(v[pos + q]) < k) ++q;
        gp.kb[k] = q;
      }
      pos += sz;
      groups.push_back(gp);
      *namax = std::max(*namax, sz);
    }
  }
}

int resident_clusters(rt_grid g, int variant, int amax, int C, int threads, size_t smem) {
  if (g->interp == RT_INTERP_QUADRATIC) {
    if (g->desc.prec == RT_PREC_FP64) return rtk::quad_max_active_clusters<double>(amax, C, threads, smem);
    return rtk::quad_max_active_clusters<float>(amax, C, threads, smem);
  }
  const int kind = variant == 3 ? 3 : (variant == 2 ? 1 : 0);
  if (g->desc.prec == RT_PREC_FP64) return rtk::sweep_max_active_clusters<double>(kind, amax, C, threads, smem);
  return rtk::sweep_max_active_clusters<float>(kind, amax, C, threads, smem);
}

// A sweep launch whose group instances fill k waves of co-resident clusters and
// part of one more ends with that last part running alone, each of its clusters
// carrying a whole group.  Splitting s = (groups mod resident) groups into
// halves (when 2s clusters fit one wave) leaves k full waves and a last wave of
// 2s half groups, which ends sooner.  Only single-frequency Jacobi grids are
// changed; only groups sweeping along y or z are split (the x groups stay
// first: the float32 update reads their partials in their own layout), and the
// halves go last, since clusters start in launch order.
void split_last_wave(rt_grid g) {
  if (g->iteration != RT_ITER_JACOBI || g->d.nf != 1 || g->apg < 2 || g->groups.empty()) return;
  const int nres = resident_clusters(g, g->variant, g->amax, g->cluster, g->threads, g->smem);
  const int G = (int)g->groups.size();
  if (nres <= 0 || G <= nres) return;
  const int s = G % nres;
  if (s == 0 || 2 * s > nres) return;
  std::vector<int> pick;   // the last s groups of two rays or more off the x axis
  for (int gi = G - 1; gi >= 0 && (int)pick.size() < s; --gi)
    if (g->groups[gi].axis != 0 && g->groups[gi].na >= 2) pick.push_back(gi);
  if ((int)pick.size() < s) return;
  auto set_kb = [&](GroupParam &gp) {   // stencil-key boundaries of a group's rays
    int cax[3];
    rtk::plane_axes(gp.axis, cax);
    for (int k = 0; k <= 4; ++k) {
      int q = 0;
      while (q < gp.na) {
        const RayGeom &r = g->rays[g->group_angles[gp.a0 + q]];
        const int key = (r.sgn[cax[0]] > 0 ? 1 : 0) + (r.sgn[cax[1]] > 0 ? 2 : 0);
        if (key >= k) break;
        ++q;
      }
      gp.kb[k] = q;
    }
  };
  std::vector<GroupParam> keep, halves;
  for (int gi = 0; gi < G; ++gi) {
    GroupParam gp = g->groups[gi];
    if (std::find(pick.begin(), pick.end(), gi) == pick.end()) {
      keep.push_back(gp);
      continue;
    }
    GroupParam a = gp, b = gp;
    a.na = gp.na / 2;
    b.a0 = gp.a0 + a.na;
    b.na = gp.na - a.na;
    set_kb(a);
    set_kb(b);
    halves.push_back(a);
    halves.push_back(b);
  }
  keep.insert(keep.end(), halves.begin(), halves.end());
  g->groups.swap(keep);
}

// Choose rays per group and strips per plane: the estimated sweep time is
// (waves of resident clusters) x (rays per group) x (cells per strip) x
// (CTAs sharing an SM), from the runtime's count of co-resident clusters
// (clusters cannot straddle a GPC, so this is not simply SMs / C).
void plan_groups(rt_grid g) {
  int minNv = 1 << 30;
  for (int a = 0; a < 3; ++a) {
    if (!g->used_axis[a]) continue;
    int cax[3];
    rtk::plane_axes(a, cax);
    minNv = std::min(minNv, g->d.n[cax[1]]);
  }
  int variant = g->req_variant;
  if (variant == 0) variant = g->desc.prec == RT_PREC_FP64 ? 1 : 3;
  if (g->interp == RT_INTERP_QUADRATIC) variant = 3;   // the second-order sweep is pipelined only
  const int Cmax = std::min(16, minNv);
  double best = 1e300;
  int bapg = 1, bC = 1;
  for (int apg = 1; apg <= 8; ++apg) {
    if (g->req_apg > 0 && apg != g->req_apg) continue;
    std::vector<GroupParam> gr;
    std::vector<int> ga;
    int namax = 0;
    make_groups(g, apg, gr, ga, &namax);
    const long long clusters = (long long)gr.size() * g->d.nf;
    for (int C = 1; C <= Cmax; ++C) {
      if (g->req_cluster > 0 && C != g->req_cluster) continue;
      size_t smem;
      int threads;
      sweep_shape(g, variant, namax, C, &smem, &threads);
      if (g->req_threads > 0) threads = std::min(g->req_threads, sweep_thread_cap(g, variant));
      if (smem > kSweepSmemBudget) continue;
      int raw_threads = 0;
      for (int a = 0; a < 3; ++a) {
        if (!g->used_axis[a]) continue;
        int cax[3];
        rtk::plane_axes(a, cax);
        const int Rmax = (g->d.n[cax[1]] + C - 1) / C;
        const int Nu = g->d.n[cax[0]];
        const int seg = g->interp == RT_INTERP_QUADRATIC ? rtk::kQuadSeg : rtk::kSweepSeg;
        raw_threads = std::max(raw_threads, variant >= 2 ? Rmax * ((Nu + seg - 1) / seg) : Rmax * Nu);
      }
      int nres = resident_clusters(g, variant, amax_for(namax), C, threads, smem);
      if (nres <= 0) nres = 1;   // unknown occupancy: assume one resident cluster
      const double waves = std::ceil((double)clusters / nres);
      const double share = std::max(1.0, (double)std::min<long long>(clusters, nres) * C / kSMs);
      const double passes = std::ceil((double)raw_threads / threads);   // cells per thread per plane
      double work = 0.0;
      for (int a = 0; a < 3; ++a) {
        if (!g->used_axis[a]) continue;
        int cax[3];
        rtk::plane_axes(a, cax);
        const int Rmax = (g->d.n[cax[1]] + C - 1) / C;
        work = std::max(work, (double)Rmax * g->d.n[cax[0]]);
      }
      // per-step cost: the rays' cells per strip plus a per-ray and per-step staging
      // and barrier overhead (measured: groups of 7-8 rays beat small groups on
      // the 128^3 x 80-ray box, whose per-plane work is otherwise latency bound),
      // and the J partials every group writes
      const double per_step = namax * std::max(work, 64.0 * passes) + 4096.0 + 1024.0 * namax;
      const double partials = (double)gr.size() * g->d.nf * (double)g->d.cells / kSMs / 16.0;
      const double est = waves * share * per_step * (Cmax > 0 ? 1.0 : 1.0) + partials / std::max(1.0, (double)g->d.n[0]);
      if (est < best * 0.999) {
        best = est;
        bapg = apg;
        bC = C;
      }
    }
  }
  int namax = 0;
  make_groups(g, bapg, g->groups, g->group_angles, &namax);
  g->variant = variant;
  g->apg = bapg;
  g->slots = namax;
  g->amax = amax_for(namax);
  g->cluster = bC;
  sweep_shape(g, variant, namax, bC, &g->smem, &g->threads);
  if (g->req_threads > 0) g->threads = std::min(g->req_threads, sweep_thread_cap(g, variant));
  split_last_wave(g);
}

template <typename T>
rt_status upload_plan(rt_grid g) {
  g->gen++;
  std::vector<AngleParam<T>> ap(g->group_angles.size());
  for (size_t gi = 0; gi < g->groups.size(); ++gi) {
    const GroupParam &gp = g->groups[gi];
    int cax[3];
    rtk::plane_axes(gp.axis, cax);
    for (int q = 0; q < gp.na; ++q) {
      const int k = g->group_angles[gp.a0 + q];
      const RayGeom &r = g->rays[k];
      const double fu = r.frac[cax[0]], fv = r.frac[cax[1]];
      AngleParam<T> p{};
      p.wq = (T)r.w;
      p.hs = (T)(0.5 * r.s);
      p.wa = (T)((1.0 - fu) * (1.0 - fv));
      p.wb = (T)(fu * (1.0 - fv));
      p.wc = (T)((1.0 - fu) * fv);
      p.wd = (T)(fu * fv);
      for (int a = 0; a < 3; ++a) p.mu[a] = (T)g->mu[3 * k + a];
      p.su = r.sgn[cax[0]];
      p.sv = r.sgn[cax[1]];
      p.angle = k;
      ap[gp.a0 + q] = p;
    }
  }
  if (g->angp) cudaFree(g->angp);
  if (g->grp) cudaFree(g->grp);
  g->angp = nullptr;
  g->grp = nullptr;
  CU(cudaMalloc(&g->angp, std::max<size_t>(1, ap.size()) * sizeof(AngleParam<T>)));
  CU(cudaMalloc((void **)&g->grp, std::max<size_t>(1, g->groups.size()) * sizeof(GroupParam)));
  CU(cudaMemcpy(g->angp, ap.data(), ap.size() * sizeof(AngleParam<T>), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(g->grp, g->groups.data(), g->groups.size() * sizeof(GroupParam), cudaMemcpyHostToDevice));
  const size_t need = g->groups.size();
  if (need > g->jpart_groups) {
    if (g->Jpart) cudaFree(g->Jpart);
    g->Jpart = nullptr;
    CU(cudaMalloc(&g->Jpart, need * (size_t)N_of(g) * sizeof(T)));
    g->jpart_groups = need;
  }
  if (g->interp == RT_INTERP_QUADRATIC && need > g->opart_groups) {
    if (g->Opart) cudaFree(g->Opart);
    g->Opart = nullptr;
    CU(cudaMalloc(&g->Opart, need * (size_t)N_of(g) * sizeof(T)));
    g->opart_groups = need;
  }
  return RT_OK;
}

rt_status upload_plan_any(rt_grid g) {
  return g->desc.prec == RT_PREC_FP64 ? upload_plan<double>(g) : upload_plan<float>(g);
}

rt_status ensure_tmp(rt_grid g, size_t n) {
  if (n <= g->tmp_n) return RT_OK;
  if (g->tmp) cudaFree(g->tmp);
  g->tmp = nullptr;
  g->tmp_n = 0;
  CU(cudaMalloc((void **)&g->tmp, n * sizeof(double)));
  g->tmp_n = n;
  return RT_OK;
}

rt_status copy_in(rt_grid g, double *dst, const double *src, size_t n, int on_device, cudaStream_t s) {
  CU(cudaMemcpyAsync(dst, src, n * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  (void)g;
  return RT_OK;
}

rt_status copy_out(double *dst, const double *src, size_t n, int on_device, cudaStream_t s) {
  CU(cudaMemcpyAsync(dst, src, n * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return RT_OK;
}

template <typename T>
rt_status permute_into(rt_grid g, const double *src, void *const dst[3], cudaStream_t s) {
  T *d0 = g->used_axis[0] ? (T *)dst[0] : nullptr;
  T *d1 = g->used_axis[1] ? (T *)dst[1] : nullptr;
  T *d2 = g->used_axis[2] ? (T *)dst[2] : nullptr;
  CU(rtk::launch_permute<T>(g->d, src, d0, d1, d2, s));
  g->launches++;
  return RT_OK;
}

rt_status permute_any(rt_grid g, const double *src, void *const dst[3], cudaStream_t s) {
  return g->desc.prec == RT_PREC_FP64 ? permute_into<double>(g, src, dst, s)
                                      : permute_into<float>(g, src, dst, s);
}

template <typename T>
rt_status init_ghosts(rt_grid g, const double *S, cudaStream_t s) {
  CU(rtk::launch_init_ghosts<T>(g->d, g->na, g->rays_d, S, (T *)g->G[0], s));
  CU(rtk::launch_state_op(g->st, 2, 0, 0.0, 0, s));
  g->launches += 2;
  g->fs_total = 0;
  return RT_OK;
}

rt_status init_ghosts_any(rt_grid g, const double *S, cudaStream_t s) {
  return g->desc.prec == RT_PREC_FP64 ? init_ghosts<double>(g, S, s) : init_ghosts<float>(g, S, s);
}

template <typename T>
rt_status fill_bc(rt_grid g, int face, cudaStream_t s) {
  const int ax = face / 2, side = face % 2;
  const int bc = side ? g->desc.bc_hi[ax] : g->desc.bc_lo[ax];
  if (g->d.periodic[ax] || bc == RT_BC_EXTERNAL) return RT_OK;
  CU(rtk::launch_fill_bc<T>(g->d, g->na, face, bc, g->B, g->user_bc[face], (T *)g->Ibc[face], s));
  g->launches++;
  return RT_OK;
}

rt_status fill_bc_any(rt_grid g, int face, cudaStream_t s) {
  return g->desc.prec == RT_PREC_FP64 ? fill_bc<double>(g, face, s) : fill_bc<float>(g, face, s);
}

// Error word written by the bounds-checked debug build's kernels.
rt_status check_device_error(rt_grid g) {
  rtk::SolveState hs{};
  CU(cudaMemcpy(&hs, g->st, sizeof hs, cudaMemcpyDeviceToHost));
  if (hs.err) return fail(RT_ERR_CUDA, "device check failed (code %d, index %d)", hs.err, hs.err_info);
  return RT_OK;
}

template <typename T>
rtk::SweepArgs<T> sweep_args(rt_grid g) {
  rtk::SweepArgs<T> A{};
  A.d = g->d;
  A.na = g->na;
  for (int a = 0; a < 3; ++a) {
    A.chiP[a] = (const T *)g->chiP[a];
    A.SP[a] = (const T *)g->SP[a];
  }
  A.G[0] = (T *)g->G[0];
  A.G[1] = (T *)g->G[1];
  A.Gd[0] = (T *)g->Gd[0];
  A.Gd[1] = (T *)g->Gd[1];
  A.incremental = 0;
  A.ray_slots = g->slots;
  for (int f = 0; f < 6; ++f) A.Ibc[f] = (const T *)g->Ibc[f];
  A.ang = (const AngleParam<T> *)g->angp;
  A.grp = g->grp;
  A.ngroups = (int)g->groups.size();
  A.Jpart = (T *)g->Jpart;
  A.Opart = g->interp == RT_INTERP_QUADRATIC ? (T *)g->Opart : nullptr;
  A.Mpart = (T *)g->Mpart;
  A.st = g->st;
  A.parity_offset = 0;
  A.write_ghosts = 1;
  A.skip_if_done = 1;
  A.cluster = g->cluster;
  const bool wt = g->wt && g->wt_gen == g->gen && g->variant == 1 && g->interp == RT_INTERP_LINEAR;
  const size_t half = g->wt_bytes / 2;
  A.WE = wt ? (const T *)g->wt : nullptr;
  A.WP = wt ? (const T *)((const char *)g->wt + half) : nullptr;
  for (int side = 0; side < 2; ++side) {   // subdomain z faces (FP64 grids only)
    A.ext[side] = g->xI[side] != nullptr;
    A.xchi[side] = (const T *)g->xchi[side];
    A.xS[side] = (const T *)g->xS[side];
    A.xB[side] = (const T *)g->xB[side];
    A.xI[side] = (const T *)g->xI[side];
    A.xout[side] = (T *)g->xout[side];
  }
  return A;
}

// The one-cell-per-thread sweep of FP64 grids reads its segment weights E, Psi0
// (functions of chi alone) from a table filled once per medium and plan: the
// FP64 exponential and divide are then paid once, not every formal solution.
// Without the memory for it, the sweep computes them as before.
template <typename T>
rt_status ensure_seg_table(rt_grid g, cudaStream_t s) {
  if (sizeof(T) != 8 || g->variant != 1 || g->interp != RT_INTERP_LINEAR || g->wt_off) return RT_OK;
  if (g->wt && g->wt_gen == g->gen) return RT_OK;
  const size_t need = 2 * g->group_angles.size() * (size_t)N_of(g) * sizeof(T);
  if (need > g->wt_bytes) {
    if (g->wt) cudaFree(g->wt);
    g->wt = nullptr;
    g->wt_bytes = 0;
    if (cudaMalloc(&g->wt, need) != cudaSuccess) {
      cudaGetLastError();
      g->wt = nullptr;
      g->wt_off = true;
      return RT_OK;
    }
    g->wt_bytes = need;
    g->gen++;   // a new buffer: captured graphs must not replay the old pointers
  }
  rtk::SweepArgs<T> A = sweep_args<T>(g);
  T *WE = (T *)g->wt, *WP = (T *)((char *)g->wt + g->wt_bytes / 2);
  for (size_t gi = 0; gi < g->groups.size(); ++gi) {
    CU(rtk::launch_seg_table<T>(A, (int)gi, g->groups[gi].na, WE, WP, s));
    g->launches++;
  }
  g->wt_gen = g->gen;
  return RT_OK;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
};

template <typename T>
rt_status enqueue_sweep(rt_grid g, rtk::SweepArgs<T> &A, bool moments, cudaStream_t s,
                        std::vector<EventPair> *ev) {
  EventPair p;
  if (ev) {
    CU(cudaEventCreate(&p.a));
    CU(cudaEventCreate(&p.b));
    CU(cudaEventRecord(p.a, s));
  }
  if (g->interp == RT_INTERP_QUADRATIC) {
    CU(rtk::launch_sweep_quad<T>(A, g->amax, moments, g->threads, g->smem, s));
  } else if (g->variant == 3) {
    CU(rtk::launch_sweep_pipe<T>(A, g->amax, moments, g->threads, g->smem, s));
  } else if (g->variant == 2) {
    CU(rtk::launch_sweep_tiled<T>(A, g->amax, moments, g->threads, g->smem, s));
  } else {
    CU(rtk::launch_sweep<T>(A, g->amax, moments, g->threads, g->smem, s));
  }
  g->launches++;
  if (ev) {
    CU(cudaEventRecord(p.b, s));
    ev->push_back(p);
  }
  return RT_OK;
}

// Sums the first `first_n` recorded sweep durations (later ones were launches
// enqueued after convergence that returned at once) and releases all events.
rt_status collect_events(std::vector<EventPair> &ev, double *ms_out, int *n_out, size_t first_n) {
  double ms = 0.0;
  int n = 0;
  cudaError_t err = cudaSuccess;
  for (size_t i = 0; i < ev.size(); ++i) {
    if (i < first_n && err == cudaSuccess) {
      float t = 0.0f;
      err = cudaEventElapsedTime(&t, ev[i].a, ev[i].b);
      ms += t;
      ++n;
    }
    cudaEventDestroy(ev[i].a);
    cudaEventDestroy(ev[i].b);
  }
  ev.clear();
  CU(err);
  *ms_out = ms;
  *n_out = n;
  return RT_OK;
}

// Gauss-Seidel set-up: the reverse groups (crossed axis V, mu_V < 0), which
// make_groups leaves adjacent with their rays adjacent in the angle table; the
// forward groups and the forward rays with mu_V < 0 (device lists); the
// correction weights (once per medium and ray set); the reverse kernel's
// buffers.
template <typename T>
rt_status gs_setup(rt_grid g, cudaStream_t s, bool incremental, rtk::GsArgs<T> &G) {
  const int V = g->two_d ? 1 : 2;
  std::vector<int> fg, fr;
  int rev_first = -1, nrev = 0, rev0 = 0;
  for (size_t gi = 0; gi < g->groups.size(); ++gi) {
    const GroupParam &gp = g->groups[gi];
    if (gp.axis == V && gp.sa < 0) {
      if (rev_first < 0) {
        rev_first = (int)gi;
        rev0 = gp.a0;
      } else if (gp.a0 != rev0 + nrev) {
        return fail(RT_ERR_STATE, "reverse sweep groups are not adjacent in the angle table");
      }
      nrev += gp.na;
    } else {
      fg.push_back((int)gi);
    }
  }
  if (nrev < 1 || nrev > rtk::kGsMaxRev)
    return fail(RT_ERR_STATE, "Gauss-Seidel needs 1..%d reverse rays, the angle set gives %d", rtk::kGsMaxRev, nrev);
  for (int k = 0; k < g->na; ++k) {
    const RayGeom &r = g->rays[k];
    if (!(r.axis == V && r.sgn[V] < 0) && g->mu[3 * k + V] < 0.0) fr.push_back(k);
  }
  std::vector<int> list(fg);
  list.insert(list.end(), fr.begin(), fr.end());
  if (list.size() > g->gs_list_n) {
    g->gen++;
    if (g->gs_list) cudaFree(g->gs_list);
    g->gs_list = nullptr;
    g->gs_list_n = 0;
    CU(cudaMalloc((void **)&g->gs_list, list.size() * sizeof(int)));
    g->gs_list_n = list.size();
  }
  CU(cudaMemcpyAsync(g->gs_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const size_t N = (size_t)N_of(g);
  if (!g->gsw || !g->gs_bar) g->gen++;
  if (!g->gsw) CU(cudaMalloc((void **)&g->gsw, 9 * N * sizeof(double)));
  if (!g->gs_bar) CU(cudaMalloc((void **)&g->gs_bar, rtk::kGsBarWords * sizeof(unsigned)));
  int cax[3];
  rtk::plane_axes(V, cax);
  const size_t plane = (size_t)g->d.n[cax[0]] * g->d.n[cax[1]];
  const size_t irb = 4 * (size_t)g->d.nf * nrev * plane * sizeof(T);
  if (irb > g->gsIr_bytes) {
    g->gen++;
    if (g->gsIr) cudaFree(g->gsIr);
    g->gsIr = nullptr;
    g->gsIr_bytes = 0;
    CU(cudaMalloc(&g->gsIr, irb));
    g->gsIr_bytes = irb;
  }
  if (!g->gs_ready) {
    CU(rtk::launch_gs_weights<T>(g->d, V, g->chi, g->rays_d, g->gs_list + fg.size(), (int)fr.size(), g->gsw, s));
    g->launches++;
    g->gs_ready = true;
  }
  G.V = V;
  G.nrev = nrev;
  G.rev0 = rev0;
  G.fgroups = g->gs_list;
  G.nfg = (int)fg.size();
  G.chi = g->chi;
  G.eps = g->eps;
  G.B = g->B;
  G.iden = g->iden;
  G.S64 = g->S;
  G.Sfs = g->Sfs;
  G.J64 = g->J;
  G.dS = g->Jprev;   // Jprev serves only the eps = 1 test, which Gauss-Seidel leaves to Jacobi
  G.incremental = incremental ? 1 : 0;
  G.JF64 = G.JR64 = nullptr;
  if (incremental) {
    if (!g->gs_acc) {
      g->gen++;
      CU(cudaMalloc((void **)&g->gs_acc, 2 * N * sizeof(double)));
    }
    G.JF64 = g->gs_acc;
    G.JR64 = g->gs_acc + N;
  }
  G.gsw = g->gsw;
  G.SPV = (T *)g->SP[V];
  G.Ir = (T *)g->gsIr;
  G.fmask = g->fmask;
  G.poll_limit = g->gs_polls;
  G.bar = g->gs_bar;
  return RT_OK;
}

// Sweep and Jacobi-update arguments of an ALI solve of g with the pipelined or
// one-cell-per-thread sweep (the Gauss-Seidel forward-phase flags are set by the
// caller).  The float32 pipelined sweep writes the partials of the groups
// sweeping along x (the first groups) in their plane layout, which the Jacobi
// update reads.
template <typename T>
void solve_args(rt_grid g, int incremental, bool gs, rtk::SweepArgs<T> &A, rtk::AliArgs<T> &L) {
  A = sweep_args<T>(g);
  A.incremental = incremental;
  int nxg = 0;
  if (sizeof(T) == 4 && !gs && g->variant == 3 && g->interp == RT_INTERP_LINEAR && g->d.n[0] % 4 == 0 &&
      g->d.n[1] % 4 == 0) {
    while (nxg < (int)g->groups.size() && g->groups[nxg].axis == 0) ++nxg;
    A.jx = 1;
  }
  L = rtk::AliArgs<T>{};
  L.d = g->d;
  L.ngroups_per_f = (int)g->groups.size();
  L.Jpart = (const T *)g->Jpart;
  L.eps = g->eps;
  L.B = g->B;
  L.iden = g->iden;
  L.ia = g->ia;
  L.ib = g->ib;
  L.Opart = g->interp == RT_INTERP_QUADRATIC ? (const T *)g->Opart : nullptr;
  L.S64 = g->S;
  L.Sfs = g->Sfs;
  L.J64 = g->J;
  L.Jprev = g->Jprev;
  for (int a = 0; a < 3; ++a) L.SP[a] = g->used_axis[a] ? (T *)g->SP[a] : nullptr;
  L.st = g->st;
  L.lte = g->lte ? 1 : 0;
  L.incremental = incremental;
  L.fmask = g->fmask;
  L.nxg = nxg;
}

template <typename T>
rt_status formal_once(rt_grid g, cudaStream_t s);

// One Jacobi iteration of a mixed grid whose formal solution is done in FP64 by
// the internal FP64 grid, from the current S: the first iteration of a solve
// (ghosts from S, as for every first formal solution) or a later one (the lagged
// ghosts taken from this grid's current float32 ghosts, prev = their parity).
// J64 receives the FP64 J, this grid's next ghosts and their change the FP64
// outflow; then the update and the decision.  The float32 increments that
// follow start from this J: the rounding accumulated in J64 so far is dropped.
rt_status fp64_iteration(rt_grid g, const rtk::AliArgs<float> &L, int prev, bool first, cudaStream_t s) {
  rt_grid h = g->first64;
  const long long ng = (long long)g->d.nf * g->na * g->d.gsize;
  rt_status r;
  if (first) {
    rt_solve_opts o2{};
    o2.stream = (void *)s;
    if ((r = rt_formal_solve(h, g->S, g->J, nullptr, 1, &o2)) != RT_OK) return r;
  } else {
    const size_t N = (size_t)N_of(g);
    CU(cudaMemcpyAsync(h->S, g->S, N * 8, cudaMemcpyDeviceToDevice, s));
    if ((r = permute_any(h, h->S, h->SP, s)) != RT_OK) return r;
    CU(rtk::launch_f32_to_f64(ng, (const float *)g->G[prev], (double *)h->G[0], s));
    CU(rtk::launch_state_op(h->st, 2, 0, 0.0, 0, s));
    h->fs_total = 0;
    h->launches += 2;
    if ((r = formal_once<double>(h, s)) != RT_OK) return r;
    CU(cudaMemcpyAsync(g->J, h->J, N * 8, cudaMemcpyDeviceToDevice, s));
  }
  CU(rtk::launch_ghosts_from64(ng, (const double *)h->G[1], (const double *)h->G[0], (float *)g->G[prev ^ 1],
                               (float *)g->Gd[prev ^ 1], s));
  rtk::AliArgs<float> L0 = L;
  L0.Jpart = nullptr;
  CU(rtk::launch_ali<float>(L0, s));
  CU(rtk::launch_finish(g->st, s));
  g->launches += 3;
  return RT_OK;
}

template <typename T>
rt_status ali_loop(rt_grid g, const rt_solve_opts *opts, cudaStream_t s, int *iters, double *resid,
                   bool *converged) {
  const double tol = opts ? opts->tol : 1e-6;
  const int max_iter = opts && opts->max_iter > 0 ? opts->max_iter : 1000;
  CU(rtk::launch_state_op(g->st, 0, max_iter, tol, g->lte ? 1 : 0, s));
  g->launches++;
  // The mixed path sweeps increments after the first formal solution so that
  // float32 rounding scales with the update, not with S (J accumulated in FP64).
  // (the second-order sweep is nonlinear in S -- its clamps -- so it never
  // sweeps increments; it also brings its own Lambda* every iteration)
  const bool gs = g->iteration == RT_ITER_GAUSS_SEIDEL && !g->lte;
  const int incremental = (g->desc.prec == RT_PREC_MIXED && g->interp == RT_INTERP_LINEAR) ? 1 : 0;
  rtk::GsArgs<T> GA{};
  if (gs) {
    rt_status r = gs_setup<T>(g, s, incremental != 0, GA);
    if (r != RT_OK) return r;
  }
  {
    rt_status r = ensure_seg_table<T>(g, s);
    if (r != RT_OK) return r;
  }
  rtk::SweepArgs<T> A;
  rtk::AliArgs<T> L;
  solve_args<T>(g, incremental, gs, A, L);
  if (gs) {
    A.gs_forward = 1;
    A.gs_axis = GA.V;
    GA.A = A;
  }
  std::vector<EventPair> ev;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (g->timing) {
    CU(cudaEventCreate(&t0));
    CU(cudaEventCreate(&t1));
    CU(cudaEventRecord(t0, s));
  }
  int enqueued = 0, batch = opts && opts->check_every > 0 ? opts->check_every : 4;
  g->stats.first_fp64 = 0;
  g->stats.fp64_anchors = 0;
  // mixed Jacobi solves: FP64 iterations (the first, then one each time the
  // residual has fallen by anchor_drop since the last), float32 increments between
  const bool fp64_its = sizeof(T) == 4 && g->fp64_first && g->first64 && incremental && !gs && !g->lte;
  double anchor_ref = -1.0;
  bool anchor_next = false;
  if constexpr (sizeof(T) == 4) {
    if (fp64_its && max_iter > 0) {
      rt_status r = fp64_iteration(g, L, 0, true, s);
      if (r != RT_OK) return r;
      enqueued = 1;
      g->stats.first_fp64 = 1;
    }
  }
  rtk::SolveState hs{};
  // the launches of m iterations (every later kernel of a batch does nothing
  // once the solve has converged)
  auto enqueue_batch = [&](int m) -> rt_status {
    for (int i = 0; i < m; ++i) {
      rt_status r = enqueue_sweep<T>(g, A, false, s, g->timing ? &ev : nullptr);
      if (r != RT_OK) return r;
      if (gs) {   // reverse phase (updates S), then the sweep copies of the new S (or dS)
        CU(rtk::launch_gs_reverse<T>(GA, s));
        CU(rtk::launch_permute<T>(g->d, incremental ? GA.dS : g->S, L.SP[0], L.SP[1], L.SP[2], s));
        g->launches += 2;
      } else {
        CU(rtk::launch_ali<T>(L, s));
        g->launches++;
      }
      CU(rtk::launch_finish(g->st, s));
      g->launches++;
    }
    return RT_OK;
  };
  // after the first batch (which also performs every kernel's one-time set-up),
  // batches are captured once as CUDA graphs and replayed: one launch per batch
  auto graph_for = [&](int m) -> const rt_grid_s::Graph * {
    for (auto it = g->graphs.begin(); it != g->graphs.end();) {
      if (it->gen != g->gen) {   // arguments of another plan or buffer set
        cudaGraphExecDestroy(it->exec);
        it = g->graphs.erase(it);
        continue;
      }
      if (it->m == m && it->gs == (gs ? 1 : 0) && it->inc == incremental) return &*it;
      ++it;
    }
    const long long l0 = g->launches;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g->graphs_ok = false;
      return nullptr;
    }
    const rt_status r = enqueue_batch(m);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    const long long n = g->launches - l0;
    g->launches = l0;
    cudaGraphExec_t exec = nullptr;
    if (r != RT_OK || e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();   // not capturable here: launch directly from now on
      if (graph) cudaGraphDestroy(graph);
      g->graphs_ok = false;
      return nullptr;
    }
    cudaGraphDestroy(graph);
    g->graphs.push_back(rt_grid_s::Graph{g->gen, m, gs ? 1 : 0, incremental, n, exec});
    return &g->graphs.back();
  };
  while (true) {
    int m = std::min(batch, max_iter - enqueued);
    if constexpr (sizeof(T) == 4) {
      if (anchor_next && m > 0) {   // this batch begins with an FP64 iteration
        rt_status r = fp64_iteration(g, L, (hs.fs_count + A.parity_offset) & 1, false, s);
        if (r != RT_OK) return r;
        ++enqueued;
        --m;
        g->stats.fp64_anchors++;
        anchor_next = false;
      }
    }
    const rt_grid_s::Graph *gr = (m > 0 && enqueued > 0 && !g->timing && g->graphs_ok) ? graph_for(m) : nullptr;
    if (gr) {
      CU(cudaGraphLaunch(gr->exec, s));
      g->launches += gr->nlaunch;
      g->graph_launches++;
    } else if (m > 0) {
      rt_status r = enqueue_batch(m);
      if (r != RT_OK) return r;
    }
    enqueued += m;
    CU(cudaMemcpyAsync(&hs, g->st, sizeof hs, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hs.err) return fail(RT_ERR_CUDA, "device check failed (code %d, index %d)", hs.err, hs.err_info);
    if (hs.done || enqueued >= max_iter) break;
    if (fp64_its && g->anchor_drop > 0.0) {
      if (anchor_ref < 0.0) {
        anchor_ref = hs.last_resid;
      } else if (hs.last_resid <= anchor_ref * g->anchor_drop) {
        anchor_next = true;
        anchor_ref = hs.last_resid;
      }
    }
    if (!(opts && opts->check_every > 0)) batch = std::min(batch * 2, 64);
  }
  if (g->timing) {
    CU(cudaEventRecord(t1, s));
    CU(cudaEventSynchronize(t1));
    float tt = 0.0f;
    CU(cudaEventElapsedTime(&tt, t0, t1));
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    g->stats.total_ms = tt;
    rt_status r = collect_events(ev, &g->stats.sweep_ms, &g->stats.sweep_launches,
                                 (size_t)std::max(0, hs.iter - g->stats.first_fp64 - g->stats.fp64_anchors));
    if (r != RT_OK) return r;
  }
  *iters = hs.iter;
  *resid = hs.last_resid;
  *converged = hs.converged != 0;
  g->fs_total = hs.fs_count;
  g->last_fs_from_Sfs = !g->lte;
  // (Gauss-Seidel: the J returned is that of a formal solution of Sfs)
  g->last_incremental = incremental != 0 && !gs;
  g->sp_is_delta = incremental != 0;
  return RT_OK;
}

// n Jacobi iterations continuing the solve begun by rt_ali_begin: the sweep
// (incremental on mixed grids after the first), the update, the decision kernel
// (whose stopping rule rt_ali_begin disabled); then the solve state is read.
template <typename T>
rt_status ali_iterate(rt_grid g, int n, cudaStream_t s, int *iters, double *resid) {
  const int incremental = (g->desc.prec == RT_PREC_MIXED && g->interp == RT_INTERP_LINEAR) ? 1 : 0;
  rt_status r = ensure_seg_table<T>(g, s);
  if (r != RT_OK) return r;
  rtk::SweepArgs<T> A = sweep_args<T>(g);
  A.incremental = incremental;
  rtk::AliArgs<T> L{};
  L.d = g->d;
  L.ngroups_per_f = (int)g->groups.size();
  L.Jpart = (const T *)g->Jpart;
  L.eps = g->eps;
  L.B = g->B;
  L.iden = g->iden;
  L.Opart = g->interp == RT_INTERP_QUADRATIC ? (const T *)g->Opart : nullptr;
  L.S64 = g->S;
  L.Sfs = g->Sfs;
  L.J64 = g->J;
  L.Jprev = g->Jprev;
  for (int a = 0; a < 3; ++a) L.SP[a] = g->used_axis[a] ? (T *)g->SP[a] : nullptr;
  L.st = g->st;
  L.lte = g->lte ? 1 : 0;
  L.incremental = incremental;
  for (int i = 0; i < n; ++i) {
    if ((r = enqueue_sweep<T>(g, A, false, s, nullptr)) != RT_OK) return r;
    CU(rtk::launch_ali<T>(L, s));
    CU(rtk::launch_finish(g->st, s));
    g->launches += 2;
  }
  rtk::SolveState hs{};
  CU(cudaMemcpyAsync(&hs, g->st, sizeof hs, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (hs.err) return fail(RT_ERR_CUDA, "device check failed (code %d, index %d)", hs.err, hs.err_info);
  if (iters) *iters = hs.iter;
  if (resid) *resid = hs.last_resid;
  g->fs_total = hs.fs_count;
  g->last_fs_from_Sfs = !g->lte;
  g->last_incremental = incremental != 0;
  g->sp_is_delta = incremental != 0;
  return RT_OK;
}

template <typename T>
rt_status formal_once(rt_grid g, cudaStream_t s) {
  rt_status r0 = ensure_seg_table<T>(g, s);
  if (r0 != RT_OK) return r0;
  rtk::SweepArgs<T> A = sweep_args<T>(g);
  A.skip_if_done = 0;
  std::vector<EventPair> ev;
  rt_status r = enqueue_sweep<T>(g, A, false, s, g->timing ? &ev : nullptr);
  if (r != RT_OK) return r;
  CU(rtk::launch_reduce_J<T>(g->d, (int)g->groups.size(), (const T *)g->Jpart, g->J, s));
  if (g->interp == RT_INTERP_QUADRATIC) {   // this solution's Lambda*
    CU(rtk::launch_quad_lstar<T>(g->d, (int)g->groups.size(), (const T *)g->Opart, g->lstar, s));
    g->launches++;
  }
  CU(rtk::launch_state_op(g->st, 1, 0, 0.0, 0, s));
  g->launches += 2;
  if (g->timing) {
    CU(cudaStreamSynchronize(s));
    r = collect_events(ev, &g->stats.sweep_ms, &g->stats.sweep_launches, ev.size());
    if (r != RT_OK) return r;
    g->stats.total_ms = g->stats.sweep_ms;
  }
  g->fs_total += 1;
  g->last_fs_from_Sfs = false;
  g->last_incremental = false;
  g->sp_is_delta = false;
  return RT_OK;
}

template <typename T>
rt_status moments_sweep(rt_grid g, cudaStream_t s) {
  const size_t need = g->groups.size();
  if (need > g->mpart_groups) {
    if (g->Mpart) cudaFree(g->Mpart);
    g->Mpart = nullptr;
    CU(cudaMalloc(&g->Mpart, need * 9 * (size_t)N_of(g) * sizeof(T)));
    g->mpart_groups = need;
  }
  rt_status r0 = ensure_seg_table<T>(g, s);
  if (r0 != RT_OK) return r0;
  rtk::SweepArgs<T> A = sweep_args<T>(g);
  A.parity_offset = -1;
  A.write_ghosts = 0;
  A.skip_if_done = 0;
  return enqueue_sweep<T>(g, A, true, s, nullptr);
}

rt_status ensure_tmp2(rt_grid g, size_t n) {
  if (n <= g->tmp2_n) return RT_OK;
  if (g->tmp2) cudaFree(g->tmp2);
  g->tmp2 = nullptr;
  g->tmp2_n = 0;
  CU(cudaMalloc((void **)&g->tmp2, n * sizeof(double)));
  g->tmp2_n = n;
  return RT_OK;
}

// copy frequency bins `bins` of a [nf][block] array into a packed [bins][block] array
// (gather) or back (scatter)
rt_status move_bins(const std::vector<int> &bins, double *packed, double *full, size_t block, bool gather,
                    cudaMemcpyKind kind, cudaStream_t s) {
  for (size_t k = 0; k < bins.size(); ++k) {
    double *a = packed + k * block, *b = full + (size_t)bins[k] * block;
    CU(cudaMemcpyAsync(gather ? a : b, gather ? b : a, block * sizeof(double), kind, s));
  }
  return RT_OK;
}

// Inflow intensities of fixed faces, restricted to the FP64 bins.
rt_status sync_sub_bc(rt_grid g, int face) {
  rt_grid h = g->sub64;
  if (!h || !g->user_bc[face]) return RT_OK;
  const size_t block = (size_t)g->na * g->d.face[face / 2];
  if (!h->user_bc[face]) CU(cudaMalloc((void **)&h->user_bc[face], g->bins64.size() * block * 8));
  rt_status r = move_bins(g->bins64, h->user_bc[face], g->user_bc[face], block, true, cudaMemcpyDeviceToDevice, g->own);
  if (r != RT_OK) return r;
  CU(cudaStreamSynchronize(g->own));
  return fill_bc_any(h, face, h->own);
}

// Decide which bins of a mixed grid need FP64 sweeps and (re)build the FP64 grid.
rt_status plan_bins(rt_grid g) {
  const int nf = g->d.nf;
  cudaStream_t s = g->own;
  if (!g->epsmin) CU(cudaMalloc((void **)&g->epsmin, nf * sizeof(unsigned long long)));
  std::vector<unsigned long long> init(nf, (unsigned long long)0x3FF0000000000000ULL);   // 1.0
  CU(cudaMemcpyAsync(g->epsmin, init.data(), nf * 8, cudaMemcpyHostToDevice, s));
  CU(rtk::launch_eps_thick_min(g->d, g->eps, g->oml, g->epsmin, s));
  g->launches++;
  std::vector<unsigned long long> bits(nf);
  CU(cudaMemcpyAsync(bits.data(), g->epsmin, nf * 8, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  std::vector<int> ill;
  const double u32 = 5.96e-8;   // float32 unit roundoff
  for (int f = 0; f < nf; ++f) {
    double e;
    std::memcpy(&e, &bits[f], 8);
    if (u32 / e > g->bin_limit) ill.push_back(f);
  }
  if (ill.empty()) {
    if (g->sub64) rt_destroy_grid(g->sub64);
    g->sub64 = nullptr;
    g->bins64.clear();
    if (g->fmask) cudaFree(g->fmask);
    g->fmask = nullptr;
    return RT_OK;
  }
  if (!g->sub64 || g->bins64 != ill) {
    if (g->sub64) rt_destroy_grid(g->sub64);
    g->sub64 = nullptr;
    rt_grid_desc d = g->desc;
    d.prec = RT_PREC_FP64;
    d.nfreq = (int)ill.size();
    rt_status r = rt_create_grid(&d, &g->sub64);
    if (r != RT_OK) return r;
    if ((r = rt_set_interpolation(g->sub64, g->interp)) != RT_OK) return r;
    if ((r = rt_set_iteration(g->sub64, g->iteration)) != RT_OK) return r;
    g->bins64 = ill;
  }
  const size_t C = (size_t)g->d.cells, m = ill.size();
  rt_status r = ensure_tmp(g, 3 * m * C + m);
  if (r != RT_OK) return r;
  double *tc = g->tmp, *te = tc + m * C, *tb = te + m * C, *tw = tb + m * C;
  if ((r = move_bins(ill, tc, g->chi, C, true, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  if ((r = move_bins(ill, te, g->eps, C, true, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  if ((r = move_bins(ill, tb, g->B, C, true, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  if ((r = move_bins(ill, tw, g->fw, 1, true, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  CU(cudaStreamSynchronize(s));
  if ((r = rt_set_opacity_source(g->sub64, tc, te, tb, tw, 1)) != RT_OK) return r;
  for (int face = 0; face < 6; ++face)
    if ((r = sync_sub_bc(g, face)) != RT_OK) return r;
  std::vector<unsigned char> mask(nf, 0);
  for (int f : ill) mask[f] = 1;
  if (!g->fmask) CU(cudaMalloc((void **)&g->fmask, nf));
  CU(cudaMemcpy(g->fmask, mask.data(), nf, cudaMemcpyHostToDevice));
  return RT_OK;
}

// Mixed grids: the internal FP64 grid that does the first formal solution of
// each Jacobi ALI solve with linear interpolation (not needed when every eps = 1,
// whose solves only iterate the boundary ghosts).
// Largest segment-weight table of a mixed grid's FP64-iteration grid.
constexpr double kShadowTableMax = 16.0 * (1 << 30);

rt_status plan_first64(rt_grid g) {
  g->fp64_first = !g->lte;
  if (!g->fp64_first) {
    if (g->first64) rt_destroy_grid(g->first64);
    g->first64 = nullptr;
    return RT_OK;
  }
  if (!g->first64) {
    rt_grid_desc d = g->desc;
    d.prec = RT_PREC_FP64;
    rt_status r = rt_create_grid(&d, &g->first64);
    if (r != RT_OK) return r;
    g->first64->shadow = true;
    // a few FP64 iterations per solve: their segment weights are tabulated per
    // medium when the table is modest (it holds E and Psi0 of every ray and cell)
    g->first64->wt_off = 2.0 * g->na * (double)N_of(g) * 8.0 > kShadowTableMax;
  }
  rt_status r = rt_set_opacity_source(g->first64, g->chi, g->eps, g->B, g->fw, 1);
  if (r != RT_OK) return r;
  for (int face = 0; face < 6; ++face) {
    if (!g->user_bc[face]) continue;
    rt_grid h = g->first64;
    const size_t n = (size_t)g->d.nf * g->na * g->d.face[face / 2];
    if (!h->user_bc[face]) CU(cudaMalloc((void **)&h->user_bc[face], n * 8));
    CU(cudaMemcpy(h->user_bc[face], g->user_bc[face], n * 8, cudaMemcpyDeviceToDevice));
    if ((r = fill_bc_any(h, face, h->own)) != RT_OK) return r;
  }
  CU(cudaStreamSynchronize(g->first64->own));
  return RT_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *rt_last_error(void) { return g_err.c_str(); }

rt_status rt_create_grid(const rt_grid_desc *desc, rt_grid *out) {
  if (!desc || !out) return fail(RT_ERR_ARG, "rt_create_grid: NULL argument");
  *out = nullptr;
  const rt_grid_desc &D = *desc;
  if (D.nx < 1 || D.ny < 1 || D.nz < 1 || D.nfreq < 1)
    return fail(RT_ERR_ARG, "grid sizes and nfreq must be >= 1");
  if (!(D.dx > 0) || !(D.dy > 0) || (D.nz > 1 && !(D.dz > 0)))
    return fail(RT_ERR_ARG, "cell spacings must be > 0");
  if (D.prec != RT_PREC_FP64 && D.prec != RT_PREC_MIXED) return fail(RT_ERR_ARG, "bad precision");
  for (int a = 0; a < 3; ++a) {
    const int lim = a == 2 ? RT_BC_EXTERNAL : RT_BC_FIXED;
    if (D.bc_lo[a] < 0 || D.bc_lo[a] > lim || D.bc_hi[a] < 0 || D.bc_hi[a] > lim)
      return fail(RT_ERR_ARG, "bad boundary type on axis %d", a);
    if (a < 2 || D.nz > 1)
      if ((D.bc_lo[a] == RT_BC_PERIODIC) != (D.bc_hi[a] == RT_BC_PERIODIC))
        return fail(RT_ERR_ARG, "axis %d: a periodic axis must be periodic on both faces", a);
  }
  const bool ext = D.bc_lo[2] == RT_BC_EXTERNAL || D.bc_hi[2] == RT_BC_EXTERNAL;
  if (ext) {
    if (D.nz < 2 || D.prec != RT_PREC_FP64)
      return fail(RT_ERR_ARG, "subdomain (external) z faces need an FP64 3D grid of >= 2 planes");
    for (int a = 0; a < 2; ++a)
      if (D.bc_lo[a] == RT_BC_FIXED || D.bc_hi[a] == RT_BC_FIXED)
        return fail(RT_ERR_ARG, "subdomain z faces do not combine with fixed x or y faces");
  }
  rt_grid g = new rt_grid_s();
  g->desc = D;
  g->two_d = D.nz == 1;
  if (g->two_d) {   // z-invariant: the z faces are never crossed; treat z as periodic
    g->desc.bc_lo[2] = g->desc.bc_hi[2] = RT_BC_PERIODIC;
    g->desc.dz = 1.0;
  }
  if (!level_symmetric(D.n_mu, g->two_d, g->mu, g->wq)) {
    delete g;
    return fail(RT_ERR_ARG, "n_mu must be 2, 4, 6, 8, 10 or 12 (got %d)", D.n_mu);
  }
  g->na = (int)g->wq.size();
  g->tsize = D.prec == RT_PREC_FP64 ? 8 : 4;
  rtk::Dims &d = g->d;
  d.n[0] = D.nx;
  d.n[1] = D.ny;
  d.n[2] = D.nz;
  d.nf = D.nfreq;
  d.cells = (long long)D.nx * D.ny * D.nz;
  for (int a = 0; a < 3; ++a) {
    d.bc_lo[a] = g->desc.bc_lo[a];
    d.bc_hi[a] = g->desc.bc_hi[a];
    d.periodic[a] = g->desc.bc_lo[a] == RT_BC_PERIODIC;
  }
  d.face[0] = (long long)D.nz * D.ny;
  d.face[1] = (long long)D.nz * D.nx;
  d.face[2] = (long long)D.ny * D.nx;
  d.gsize = d.face[0] + d.face[1] + d.face[2];
  build_rays(g);
  plan_groups(g);

  auto cleanup = [&](rt_status st) {
    rt_destroy_grid(g);
    return st;
  };
  cudaGetDevice(&g->device);
  const size_t N = (size_t)d.cells * d.nf;
  const size_t ts = g->tsize;
#define ALLOC(ptr, bytes)                                                               \
  do {                                                                                  \
    cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                              \
    if (e_ != cudaSuccess)                                                              \
      return cleanup(fail(RT_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", (size_t)(bytes), \
                          cudaGetErrorString(e_)));                                     \
  } while (0)
  ALLOC(g->chi, N * 8);
  ALLOC(g->eps, N * 8);
  ALLOC(g->B, N * 8);
  ALLOC(g->fw, (size_t)d.nf * 8);
  ALLOC(g->S, N * 8);
  ALLOC(g->Sfs, N * 8);
  ALLOC(g->J, N * 8);
  ALLOC(g->Jprev, N * 8);
  ALLOC(g->lstar, N * 8);
  ALLOC(g->oml, N * 8);
  ALLOC(g->iden, N * 8);
  if (D.prec == RT_PREC_MIXED) {
    ALLOC(g->ia, N * 8);
    ALLOC(g->ib, N * 8);
  }
  for (int a = 0; a < 3; ++a) {
    if (!g->used_axis[a]) continue;
    ALLOC(g->chiP[a], N * ts);
    ALLOC(g->SP[a], N * ts);
  }
  const size_t gbytes = (size_t)d.nf * g->na * d.gsize * ts;
  ALLOC(g->G[0], gbytes);
  ALLOC(g->G[1], gbytes);
  if (D.prec == RT_PREC_MIXED) {
    ALLOC(g->Gd[0], gbytes);
    ALLOC(g->Gd[1], gbytes);
  }
  for (int f = 0; f < 6; ++f) {
    if (d.periodic[f / 2] || (f % 2 ? D.bc_hi[f / 2] : D.bc_lo[f / 2]) == RT_BC_EXTERNAL) continue;
    ALLOC(g->Ibc[f], (size_t)d.nf * g->na * d.face[f / 2] * ts);
  }
  for (int side = 0; side < 2; ++side) {
    if ((side ? D.bc_hi[2] : D.bc_lo[2]) != RT_BC_EXTERNAL) continue;
    const size_t lay = (size_t)d.nf * d.face[2] * 8, ray = lay * g->na;
    ALLOC(g->xchi[side], lay);
    ALLOC(g->xS[side], lay);
    ALLOC(g->xB[side], lay);
    ALLOC(g->xI[side], ray);
    ALLOC(g->xout[side], ray);
    if (cudaMemset(g->xchi[side], 0, lay) != cudaSuccess || cudaMemset(g->xS[side], 0, lay) != cudaSuccess ||
        cudaMemset(g->xB[side], 0, lay) != cudaSuccess || cudaMemset(g->xI[side], 0, ray) != cudaSuccess ||
        cudaMemset(g->xout[side], 0, ray) != cudaSuccess)
      return cleanup(fail(RT_ERR_CUDA, "initialisation of the subdomain face buffers failed"));
    g->wt_off = true;   // the segment-weight table does not see the ghost layer's chi
  }
  ALLOC(g->rays_d, (size_t)g->na * sizeof(RayGeom));
  ALLOC(g->st, sizeof(rtk::SolveState));
  ALLOC(g->counts, 2 * sizeof(int));
#undef ALLOC
  if (cudaMemset(g->st, 0, sizeof(rtk::SolveState)) != cudaSuccess ||
      cudaMemset(g->G[0], 0, gbytes) != cudaSuccess || cudaMemset(g->G[1], 0, gbytes) != cudaSuccess ||
      (g->Gd[0] && cudaMemset(g->Gd[0], 0, gbytes) != cudaSuccess) ||
      (g->Gd[1] && cudaMemset(g->Gd[1], 0, gbytes) != cudaSuccess) ||
      cudaMemcpy(g->rays_d, g->rays.data(), g->na * sizeof(RayGeom), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(fail(RT_ERR_CUDA, "initialisation copy failed"));
  rt_status r = upload_plan_any(g);
  if (r != RT_OK) return cleanup(r);
  if (cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(RT_ERR_CUDA, "stream creation failed"));
  *out = g;
  return RT_OK;
}

rt_status rt_destroy_grid(rt_grid g) {
  if (!g) return RT_OK;
  if (g->own) cudaStreamSynchronize(g->own);
  if (g->first64) rt_destroy_grid(g->first64);
  if (g->sub64) rt_destroy_grid(g->sub64);
  for (void *p : {(void *)g->fmask, (void *)g->epsmin, (void *)g->tmp2})
    if (p) cudaFree(p);
  void *ptrs[] = {g->chi, g->eps, g->B, g->fw, g->S, g->Sfs, g->J, g->Jprev, g->lstar, g->oml, g->iden, g->ia, g->ib,
                  g->chiP[0], g->chiP[1], g->chiP[2], g->SP[0], g->SP[1], g->SP[2], g->G[0], g->G[1],
                  g->Gd[0], g->Gd[1],
                  g->Ibc[0], g->Ibc[1], g->Ibc[2], g->Ibc[3], g->Ibc[4], g->Ibc[5],
                  g->user_bc[0], g->user_bc[1], g->user_bc[2], g->user_bc[3], g->user_bc[4], g->user_bc[5],
                  g->Jpart, g->Opart, g->Mpart, g->angp, g->grp, g->rays_d, g->st, g->counts, g->tmp,
                  g->gsw, g->gsIr, g->gs_bar, g->gs_list, g->gs_acc, g->wt};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int side = 0; side < 2; ++side)
    for (double *p : {g->xchi[side], g->xS[side], g->xB[side], g->xI[side], g->xout[side]})
      if (p) cudaFree(p);
  for (auto &e : g->graphs) cudaGraphExecDestroy(e.exec);
  if (g->own) cudaStreamDestroy(g->own);
  delete g;
  return RT_OK;
}

int rt_num_angles(rt_grid g) { return g ? g->na : 0; }

rt_status rt_grid_footprint(const rt_grid_desc *desc, long long *bytes) {
  if (!desc || !bytes) return fail(RT_ERR_ARG, "rt_grid_footprint: NULL argument");
  const rt_grid_desc &D = *desc;
  if (D.nx < 1 || D.ny < 1 || D.nz < 1 || D.nfreq < 1) return fail(RT_ERR_ARG, "grid sizes and nfreq must be >= 1");
  std::vector<double> m, q;
  if (!level_symmetric(D.n_mu, D.nz == 1, m, q)) return fail(RT_ERR_ARG, "bad n_mu %d", D.n_mu);
  const long long na = (long long)q.size();
  const long long cells = (long long)D.nx * D.ny * D.nz;
  const long long gsize = (long long)D.nx * D.ny + (long long)D.ny * D.nz + (long long)D.nx * D.nz;
  const long long groups = (na + 1) / 2 + 6;   // the planner groups at least two rays where it can
  const long long N = cells * D.nfreq;
  const long long ts = D.prec == RT_PREC_FP64 ? 8 : 4;
  long long b = 8 * N * (D.prec == RT_PREC_MIXED ? 13 : 11)   // FP64 fields and state
              + ts * N * 6                     // permuted chi, S copies
              + 6 * D.nfreq * na * gsize * ts  // ghosts (two parities, increments) and inflow faces
              + groups * N * ts * 11           // J, Lambda* and moment partials
              + 8 * (16 * N + cells);          // moments outputs
  if (D.prec == RT_PREC_FP64) b += 2 * na * N * 8;   // tabulated segment weights (one-cell sweep)
  // a mixed grid's internal FP64 grid for its FP64 iterations: fields, FP64
  // copies, ghosts, J partials (no moments pass, no table)
  if (D.prec == RT_PREC_MIXED) {
    b += 8 * N * 11 + 8 * N * 6 + 6 * D.nfreq * na * gsize * 8 + groups * N * 8;
    if (2.0 * na * (double)N * 8.0 <= kShadowTableMax) b += 2 * na * N * 8;   // its segment-weight table
  }
  *bytes = b;
  return RT_OK;
}

int rt_angle_table(int n_mu, int two_d, double *mu, double *w) {
  std::vector<double> m, q;
  if (!level_symmetric(n_mu, two_d != 0, m, q)) {
    fail(RT_ERR_ARG, "n_mu must be 2, 4, 6, 8, 10 or 12 (got %d)", n_mu);
    return RT_ERR_ARG;
  }
  if (mu) std::memcpy(mu, m.data(), m.size() * sizeof(double));
  if (w) std::memcpy(w, q.data(), q.size() * sizeof(double));
  return (int)q.size();
}

rt_status rt_get_angles(rt_grid g, double *mu, double *w) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (mu) std::memcpy(mu, g->mu.data(), g->mu.size() * sizeof(double));
  if (w) std::memcpy(w, g->wq.data(), g->wq.size() * sizeof(double));
  return RT_OK;
}

rt_status rt_set_sweep_config(rt_grid g, int angles_per_group, int cluster_ctas, int threads, int variant) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (angles_per_group < 0 || angles_per_group > 8 || cluster_ctas < 0 || cluster_ctas > 16 ||
      threads < 0 || threads > 512 || (threads % 32) || variant < 0 || variant > 3)
    return fail(RT_ERR_ARG, "bad sweep configuration");
  if ((g->xI[0] || g->xI[1]) && variant > 1)
    return fail(RT_ERR_ARG, "a grid with subdomain z faces sweeps one cell per thread (variant 1)");
  cudaStreamSynchronize(g->own);
  g->req_apg = angles_per_group;
  g->req_cluster = cluster_ctas;
  g->req_threads = threads;
  g->req_variant = variant;
  plan_groups(g);
  if (g->groups.empty()) return fail(RT_ERR_ARG, "no feasible sweep configuration");
  if (g->smem > 227 * 1024) return fail(RT_ERR_ARG, "sweep configuration needs %zu bytes of shared memory", g->smem);
  return upload_plan_any(g);
}

rt_status rt_set_opacity_source(rt_grid g, const double *chi_tot, const double *eps, const double *B,
                                const double *freq_w, int on_device) {
  if (!g || !chi_tot || !eps || !B) return fail(RT_ERR_ARG, "rt_set_opacity_source: NULL argument");
  cudaStream_t s = g->own;
  const size_t N = (size_t)N_of(g);
  rt_status r;
  if ((r = copy_in(g, g->chi, chi_tot, N, on_device, s)) != RT_OK) return r;
  if ((r = copy_in(g, g->eps, eps, N, on_device, s)) != RT_OK) return r;
  if ((r = copy_in(g, g->B, B, N, on_device, s)) != RT_OK) return r;
  if (freq_w) {
    if ((r = copy_in(g, g->fw, freq_w, g->d.nf, on_device, s)) != RT_OK) return r;
  } else {
    std::vector<double> ones(g->d.nf, 1.0);
    CU(cudaMemcpyAsync(g->fw, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
  }
  if (g->shadow) {
    // another grid's FP64 first-solution shadow: that grid validated the medium
    // and owns Lambda*; only the formal solution's inputs are needed here
    g->lte = false;
  } else {
    CU(cudaMemsetAsync(g->counts, 0, 2 * sizeof(int), s));
    CU(rtk::launch_validate((long long)N, g->chi, g->eps, g->B, g->counts, s));
    int counts[2] = {0, 0};
    CU(cudaMemcpyAsync(counts, g->counts, sizeof counts, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    g->launches++;
    if (counts[0]) {
      g->have_medium = false;
      return fail(RT_ERR_ARG, "%d input values violate chi >= 0, 0 < eps <= 1, B >= 0 or are not finite",
                  counts[0]);
    }
    g->lte = counts[1] == 0;
  }
  if ((r = permute_any(g, g->chi, g->chiP, s)) != RT_OK) return r;
  if (!g->shadow) {
    if (g->desc.prec == RT_PREC_FP64) {
      CU(rtk::launch_lstar<double>(g->d, g->chi, g->rays_d, g->na, g->lstar, g->oml, g->xchi, s));
    } else {
      CU(rtk::launch_lstar<float>(g->d, g->chi, g->rays_d, g->na, g->lstar, g->oml, g->xchi, s));
    }
    CU(rtk::launch_inv_denominator((long long)N, g->eps, g->oml, g->iden, g->B, g->ia, g->ib, s));
    g->launches += 2;
  }
  CU(cudaMemcpyAsync(g->S, g->B, N * 8, cudaMemcpyDeviceToDevice, s));
  if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  if ((r = init_ghosts_any(g, g->S, s)) != RT_OK) return r;
  for (int f = 0; f < 6; ++f)
    if ((r = fill_bc_any(g, f, s)) != RT_OK) return r;
  if (g->desc.prec == RT_PREC_MIXED && ((r = plan_first64(g)) != RT_OK || (r = plan_bins(g)) != RT_OK)) return r;
  g->gs_ready = false;
  g->gen++;
  g->have_medium = true;
  g->stepped = false;
  return RT_OK;
}

rt_status rt_set_boundary_intensity(rt_grid g, int face, const double *I) {
  if (!g || !I) return fail(RT_ERR_ARG, "rt_set_boundary_intensity: NULL argument");
  if (face < 0 || face > 5) return fail(RT_ERR_ARG, "face must be 0..5");
  const int ax = face / 2, side = face % 2;
  const int bc = side ? g->desc.bc_hi[ax] : g->desc.bc_lo[ax];
  if (bc != RT_BC_FIXED) return fail(RT_ERR_STATE, "face %d is not RT_BC_FIXED", face);
  const size_t n = (size_t)g->d.nf * g->na * g->d.face[ax];
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(I[i]) || I[i] < 0.0) return fail(RT_ERR_ARG, "boundary intensity must be finite and >= 0");
  if (!g->user_bc[face]) CU(cudaMalloc((void **)&g->user_bc[face], n * 8));
  CU(cudaMemcpyAsync(g->user_bc[face], I, n * 8, cudaMemcpyHostToDevice, g->own));
  rt_status r = fill_bc_any(g, face, g->own);
  if (r != RT_OK) return r;
  CU(cudaStreamSynchronize(g->own));
  if (g->first64 && (r = rt_set_boundary_intensity(g->first64, face, I)) != RT_OK) return r;
  return sync_sub_bc(g, face);
}

rt_status rt_formal_solve(rt_grid g, const double *S, double *J_out, double *lstar_out, int on_device,
                          const rt_solve_opts *opts) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  g->stepped = false;
  if (!g->have_medium) return fail(RT_ERR_STATE, "rt_set_opacity_source has not succeeded");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) {   // order after the grid's own stream (set-up work)
    CU(cudaStreamSynchronize(g->own));
  }
  const size_t N = (size_t)N_of(g);
  rt_status r;
  if (S) {
    if ((r = copy_in(g, g->S, S, N, on_device, s)) != RT_OK) return r;
    if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
    if ((r = init_ghosts_any(g, g->S, s)) != RT_OK) return r;
  } else if (g->sp_is_delta) {
    // the sweep copies hold the last increment: restore the full S
    if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  }
  r = g->desc.prec == RT_PREC_FP64 ? formal_once<double>(g, s) : formal_once<float>(g, s);
  if (r != RT_OK) return r;
  if (g->sub64) {   // FP64 bins: their formal solution replaces the float32 one
    const size_t C = (size_t)g->d.cells, m = g->bins64.size();
    if ((r = ensure_tmp2(g, 2 * m * C)) != RT_OK) return r;
    double *tj = g->tmp2, *tl = tj + m * C;
    const double *Ssub = nullptr;
    if (S) {
      if ((r = move_bins(g->bins64, tj, g->S, C, true, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
      Ssub = tj;
    }
    CU(cudaStreamSynchronize(s));
    rt_solve_opts o2{};
    o2.stream = (void *)s;
    if ((r = rt_formal_solve(g->sub64, Ssub, tj, tl, 1, &o2)) != RT_OK) return r;
    CU(cudaStreamSynchronize(s));
    if ((r = move_bins(g->bins64, tj, g->J, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, tl, g->lstar, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  }
  if (J_out && (r = copy_out(J_out, g->J, N, on_device, s)) != RT_OK) return r;
  if (lstar_out && (r = copy_out(lstar_out, g->lstar, N, on_device, s)) != RT_OK) return r;
  if (!on_device || !opts || !opts->stream) {
    CU(cudaStreamSynchronize(s));
    if ((r = check_device_error(g)) != RT_OK) return r;
  }
  g->stats.iters = 1;
  g->stats.updates = (long long)g->d.cells * g->na * g->d.nf;
  g->stats.kernel_launches = g->launches;
  return RT_OK;
}

// An ALI solve's start: S = S_init (or B), its sweep copies and the first ghosts.
static rt_status solve_prologue(rt_grid g, const double *S_init, int on_device, cudaStream_t s) {
  const size_t N = (size_t)N_of(g);
  rt_status r;
  if (S_init) {
    if ((r = copy_in(g, g->S, S_init, N, on_device, s)) != RT_OK) return r;
  } else {
    CU(cudaMemcpyAsync(g->S, g->B, N * 8, cudaMemcpyDeviceToDevice, s));
  }
  if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  return init_ghosts_any(g, g->S, s);
}

// An ALI solve's end: the FP64 bins of a mixed grid solved by their FP64 grid and
// their S, J and last-formal-solution S merged back; the statistics.
static rt_status solve_epilogue(rt_grid g, const double *S_init, int on_device, const rt_solve_opts *opts,
                         cudaStream_t s, int *iters, double *resid, bool *conv) {
  rt_status r;
  if (g->sub64) {
    const size_t C = (size_t)g->d.cells, m = g->bins64.size();
    if ((r = ensure_tmp2(g, m * C)) != RT_OK) return r;
    const double *Ssub = nullptr;
    if (S_init) {
      if ((r = move_bins(g->bins64, g->tmp2, const_cast<double *>(S_init), C, true,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s)) != RT_OK)
        return r;
      Ssub = g->tmp2;
    }
    CU(cudaStreamSynchronize(s));
    rt_solve_opts o2 = opts ? *opts : rt_solve_opts{1e-6, 1000, 0, nullptr};
    o2.stream = (void *)s;
    int it2 = 0;
    double res2 = 0.0;
    r = rt_ali_solve(g->sub64, Ssub, 1, &o2, &it2, &res2);
    if (r != RT_OK && r != RT_ERR_NOT_CONVERGED) return r;
    if (r == RT_ERR_NOT_CONVERGED) *conv = false;
    *iters = std::max(*iters, it2);
    *resid = std::max(*resid, res2);
    if ((r = move_bins(g->bins64, g->sub64->S, g->S, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, g->sub64->J, g->J, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, g->sub64->Sfs, g->Sfs, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    CU(cudaStreamSynchronize(s));
    g->stats.sweep_ms += g->sub64->stats.sweep_ms;
  }
  g->stats.iters = *iters;
  g->stats.resid = *resid;
  g->stats.updates = (long long)g->d.cells * g->na * g->d.nf * *iters;
  g->stats.kernel_launches = g->launches;
  if (!*conv) return fail(RT_ERR_NOT_CONVERGED, "not converged after %d formal solutions (residual %g)", *iters, *resid);
  return RT_OK;
}

rt_status rt_ali_solve(rt_grid g, const double *S_init, int on_device, const rt_solve_opts *opts,
                       int *iters_out, double *resid_out) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  g->stepped = false;
  if (!g->have_medium) return fail(RT_ERR_STATE, "rt_set_opacity_source has not succeeded");
  if (opts && !(opts->tol >= 0.0)) return fail(RT_ERR_ARG, "tol must be >= 0");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  rt_status r = solve_prologue(g, S_init, on_device, s);
  if (r != RT_OK) return r;
  int iters = 0;
  double resid = 0.0;
  bool conv = false;
  r = g->desc.prec == RT_PREC_FP64 ? ali_loop<double>(g, opts, s, &iters, &resid, &conv)
                                   : ali_loop<float>(g, opts, s, &iters, &resid, &conv);
  if (r != RT_OK) return r;
  r = solve_epilogue(g, S_init, on_device, opts, s, &iters, &resid, &conv);
  if (iters_out) *iters_out = iters;
  if (resid_out) *resid_out = resid;
  return r;
}

rt_status rt_moments(rt_grid g, double *J, double *H, double *K, double *f, double *Q, int on_device,
                     const rt_solve_opts *opts) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!g->have_medium || g->fs_total < 1) return fail(RT_ERR_STATE, "no formal solution to take moments of");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  const size_t N = (size_t)N_of(g);
  rt_status r;
  // device outputs: J(N) H(3N) K(6N) F(6N) Q(cells)
  if ((r = ensure_tmp(g, 16 * N + (size_t)g->d.cells)) != RT_OK) return r;
  double *dJ = g->tmp, *dH = dJ + N, *dK = dH + 3 * N, *dF = dK + 6 * N, *dQ = dF + 6 * N;
  const double *Ssrc = g->last_fs_from_Sfs ? g->Sfs : g->S;
  if ((r = permute_any(g, Ssrc, g->SP, s)) != RT_OK) return r;
  if (g->desc.prec == RT_PREC_FP64) {
    if ((r = moments_sweep<double>(g, s)) != RT_OK) return r;
    CU(rtk::launch_reduce_moments<double>(g->d, (int)g->groups.size(), (const double *)g->Jpart,
                                          (const double *)g->Mpart, dJ, dH, dK, dF, g->two_d, s));
  } else {
    if ((r = moments_sweep<float>(g, s)) != RT_OK) return r;
    CU(rtk::launch_reduce_moments<float>(g->d, (int)g->groups.size(), (const float *)g->Jpart,
                                         (const float *)g->Mpart, dJ, dH, dK, dF, g->two_d, s));
  }
  if (g->last_incremental) {
    // J of the last formal solution as the solve accumulated it in FP64
    CU(cudaMemcpyAsync(dJ, g->J, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (g->sub64) {   // the FP64 bins' moments replace the float32 ones
    const size_t C = (size_t)g->d.cells, m = g->bins64.size();
    if ((r = ensure_tmp2(g, 16 * m * C + C)) != RT_OK) return r;
    double *sJ = g->tmp2, *sH = sJ + m * C, *sK = sH + 3 * m * C, *sF = sK + 6 * m * C, *sQ = sF + 6 * m * C;
    CU(cudaStreamSynchronize(s));
    rt_solve_opts o2{};
    o2.stream = (void *)s;
    if ((r = rt_moments(g->sub64, sJ, sH, sK, sF, sQ, 1, &o2)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, sJ, dJ, C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, sH, dH, 3 * C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, sK, dK, 6 * C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
    if ((r = move_bins(g->bins64, sF, dF, 6 * C, false, cudaMemcpyDeviceToDevice, s)) != RT_OK) return r;
  }
  const double h[3] = {g->desc.dx, g->desc.dy, g->desc.dz};
  CU(rtk::launch_heating(g->d, g->fw, g->chi, g->eps, dJ, g->B, dH, h, g->heat_form, dQ, s));
  g->launches += 2;   // moment reduction + heating rate
  if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  g->sp_is_delta = false;   // the sweep copies hold the full S again
  if (J && (r = copy_out(J, dJ, N, on_device, s)) != RT_OK) return r;
  if (H && (r = copy_out(H, dH, 3 * N, on_device, s)) != RT_OK) return r;
  if (K && (r = copy_out(K, dK, 6 * N, on_device, s)) != RT_OK) return r;
  if (f && (r = copy_out(f, dF, 6 * N, on_device, s)) != RT_OK) return r;
  if (Q && (r = copy_out(Q, dQ, (size_t)g->d.cells, on_device, s)) != RT_OK) return r;
  CU(cudaStreamSynchronize(s));
  return check_device_error(g);
}

rt_status rt_set_external_face(rt_grid g, int side, const double *chi, const double *S, const double *B,
                               const double *I, int on_device, const rt_solve_opts *opts) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (side < 0 || side > 1 || !g->xI[side]) return fail(RT_ERR_STATE, "z face %d is not a subdomain face", side);
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  const size_t lay = (size_t)g->d.nf * g->d.face[2];
  rt_status r;
  if (chi && (r = copy_in(g, g->xchi[side], chi, lay, on_device, s)) != RT_OK) return r;
  if (S && (r = copy_in(g, g->xS[side], S, lay, on_device, s)) != RT_OK) return r;
  if (B && (r = copy_in(g, g->xB[side], B, lay, on_device, s)) != RT_OK) return r;
  if (I && (r = copy_in(g, g->xI[side], I, lay * g->na, on_device, s)) != RT_OK) return r;
  if (chi && g->have_medium) {   // Lambda* sees the ghost layer's chi
    CU(rtk::launch_lstar<double>(g->d, g->chi, g->rays_d, g->na, g->lstar, g->oml, g->xchi, s));
    CU(rtk::launch_inv_denominator((long long)N_of(g), g->eps, g->oml, g->iden, g->B, g->ia, g->ib, s));
    g->launches += 2;
  }
  if (!on_device || !opts || !opts->stream) CU(cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_get_face_intensity(rt_grid g, int side, double *I, int on_device, const rt_solve_opts *opts) {
  if (!g || !I) return fail(RT_ERR_ARG, "NULL argument");
  if (side < 0 || side > 1 || !g->xout[side]) return fail(RT_ERR_STATE, "z face %d is not a subdomain face", side);
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  rt_status r = copy_out(I, g->xout[side], (size_t)g->d.nf * g->na * g->d.face[2], on_device, s);
  if (r != RT_OK) return r;
  CU(cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_ali_begin(rt_grid g, const double *S_init, int on_device, const rt_solve_opts *opts) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!g->have_medium) return fail(RT_ERR_STATE, "rt_set_opacity_source has not succeeded");
  if (g->iteration != RT_ITER_JACOBI) return fail(RT_ERR_STATE, "stepped ALI solves take the Jacobi iteration");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  const size_t N = (size_t)N_of(g);
  rt_status r;
  if (S_init) {
    if ((r = copy_in(g, g->S, S_init, N, on_device, s)) != RT_OK) return r;
  } else {
    CU(cudaMemcpyAsync(g->S, g->B, N * 8, cudaMemcpyDeviceToDevice, s));
  }
  if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  if ((r = init_ghosts_any(g, g->S, s)) != RT_OK) return r;
  // no stopping rule of its own: the caller decides after each rt_ali_iterate
  CU(rtk::launch_state_op(g->st, 0, std::numeric_limits<int>::max(), -1.0, g->lte ? 1 : 0, s));
  g->launches++;
  g->stepped = true;
  CU(cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_ali_iterate(rt_grid g, int n, const rt_solve_opts *opts, int *iters_out, double *resid_out) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!g->stepped) return fail(RT_ERR_STATE, "rt_ali_begin has not been called since the medium was set");
  if (n < 1) return fail(RT_ERR_ARG, "n must be >= 1");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  rt_status r = g->desc.prec == RT_PREC_FP64 ? ali_iterate<double>(g, n, s, iters_out, resid_out)
                                             : ali_iterate<float>(g, n, s, iters_out, resid_out);
  if (r != RT_OK) return r;
  g->stats.iters = iters_out ? *iters_out : 0;
  g->stats.resid = resid_out ? *resid_out : 0.0;
  g->stats.updates = (long long)g->d.cells * g->na * g->d.nf * n;
  g->stats.kernel_launches = g->launches;
  return RT_OK;
}

rt_status rt_get_S(rt_grid g, double *S, int on_device, const rt_solve_opts *opts) {
  if (!g || !S) return fail(RT_ERR_ARG, "NULL argument");
  cudaStream_t s = pick_stream(g, opts);
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  rt_status r = copy_out(S, g->S, (size_t)N_of(g), on_device, s);
  if (r != RT_OK) return r;
  CU(cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_set_interpolation(rt_grid g, int order) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (order != RT_INTERP_LINEAR && order != RT_INTERP_QUADRATIC)
    return fail(RT_ERR_ARG, "interpolation order must be 1 (linear) or 2 (quadratic), not %d", order);
  if (order == g->interp) return RT_OK;
  if (order == RT_INTERP_QUADRATIC && g->iteration == RT_ITER_GAUSS_SEIDEL)
    return fail(RT_ERR_STATE, "the Gauss-Seidel iteration takes linear interpolation");
  g->interp = order;
  plan_groups(g);
  rt_status r = upload_plan_any(g);
  if (r != RT_OK) return r;
  if (g->sub64) return rt_set_interpolation(g->sub64, order);
  return RT_OK;
}

rt_status rt_set_iteration(rt_grid g, int scheme) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (scheme != RT_ITER_JACOBI && scheme != RT_ITER_GAUSS_SEIDEL)
    return fail(RT_ERR_ARG, "iteration scheme must be 0 (Jacobi) or 1 (Gauss-Seidel), not %d", scheme);
  if (scheme == RT_ITER_GAUSS_SEIDEL && g->interp != RT_INTERP_LINEAR)
    return fail(RT_ERR_STATE, "the Gauss-Seidel iteration takes linear interpolation");
  if (scheme == g->iteration) return RT_OK;
  g->iteration = scheme;
  // tied rays change sweep groups: rays, their axes' buffers, plan, Lambda*
  // (same values, other summation order) and the ghosts (laid out per group axis)
  build_rays(g);
  cudaStream_t s = g->own;
  const size_t N = (size_t)N_of(g);
  for (int a = 0; a < 3; ++a) {
    if (!g->used_axis[a] || g->SP[a]) continue;
    CU(cudaMalloc(&g->chiP[a], N * g->tsize));
    CU(cudaMalloc(&g->SP[a], N * g->tsize));
  }
  CU(cudaMemcpyAsync(g->rays_d, g->rays.data(), g->na * sizeof(RayGeom), cudaMemcpyHostToDevice, s));
  plan_groups(g);
  rt_status r = upload_plan_any(g);
  if (r != RT_OK) return r;
  g->gs_ready = false;
  if (g->have_medium) {
    if ((r = permute_any(g, g->chi, g->chiP, s)) != RT_OK) return r;
    if (g->desc.prec == RT_PREC_FP64) {
      CU(rtk::launch_lstar<double>(g->d, g->chi, g->rays_d, g->na, g->lstar, g->oml, g->xchi, s));
    } else {
      CU(rtk::launch_lstar<float>(g->d, g->chi, g->rays_d, g->na, g->lstar, g->oml, g->xchi, s));
    }
    CU(rtk::launch_inv_denominator((long long)N, g->eps, g->oml, g->iden, g->B, g->ia, g->ib, s));
    g->launches += 2;
    if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
    g->sp_is_delta = false;
    if ((r = init_ghosts_any(g, g->S, s)) != RT_OK) return r;
    g->fs_total = 0;
  }
  CU(cudaStreamSynchronize(s));
  if (g->sub64) return rt_set_iteration(g->sub64, scheme);
  return RT_OK;
}

rt_status rt_set_wait_limit(rt_grid g, long long polls) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (polls < 0) return fail(RT_ERR_ARG, "the poll limit must be >= 0");
  g->gs_polls = polls;
  g->gen++;   // captured batches hold the old limit
  return RT_OK;
}

rt_status rt_set_fp64_anchors(rt_grid g, double drop) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!(drop >= 0.0 && drop < 1.0)) return fail(RT_ERR_ARG, "drop must be in [0, 1)");
  g->anchor_drop = drop;
  return RT_OK;
}

rt_status rt_set_fp64_bin_limit(rt_grid g, double limit) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!(limit >= 0.0)) return fail(RT_ERR_ARG, "the limit must be >= 0");
  g->bin_limit = limit;
  return RT_OK;
}

rt_status rt_set_heating_form(rt_grid g, int form) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (form != RT_HEAT_INTEGRAL && form != RT_HEAT_DIFFERENTIAL && form != RT_HEAT_SWITCH)
    return fail(RT_ERR_ARG, "unknown heating form %d", form);
  g->heat_form = form;
  return RT_OK;
}

rt_status rt_enable_timing(rt_grid g, int enable) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  g->timing = enable != 0;
  return RT_OK;
}

// Plans chosen by rt_autotune, keyed by problem shape (process-wide cache).
struct TuneKey {
  int n[3], nf, n_mu, prec, bc[6], interp, iteration;
  bool operator==(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) == 0; }
};
struct TuneVal {
  int variant, apg, cluster, threads;
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

TuneKey tune_key(rt_grid g) {
  TuneKey k;
  std::memset(&k, 0, sizeof k);
  for (int a = 0; a < 3; ++a) {
    k.n[a] = g->d.n[a];
    k.bc[a] = g->desc.bc_lo[a];
    k.bc[3 + a] = g->desc.bc_hi[a];
  }
  k.nf = g->d.nf;
  k.n_mu = g->desc.n_mu;
  k.prec = g->desc.prec;
  k.interp = g->interp;
  k.iteration = g->iteration;
  return k;
}

rt_status rt_autotune(rt_grid g, int *plan_out) {
  if (!g) return fail(RT_ERR_ARG, "NULL grid");
  if (!g->have_medium) return fail(RT_ERR_STATE, "rt_set_opacity_source has not succeeded");
  const TuneKey key = tune_key(g);
  TuneVal best{0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : g_tune_cache)
      if (kv.first == key) best = kv.second;
  }
  cudaStream_t s = g->own;
  const int saved[4] = {g->req_apg, g->req_cluster, g->req_threads, g->req_variant};
  rt_status r;
  if (best.variant == 0) {
    int minNv = 1 << 30;
    for (int a = 0; a < 3; ++a) {
      if (!g->used_axis[a]) continue;
      int cax[3];
      rtk::plane_axes(a, cax);
      minNv = std::min(minNv, g->d.n[cax[1]]);
    }
    const bool ext = g->xI[0] || g->xI[1];
    const int variants[3] = {3, 2, 1};
    const int apgs[7] = {2, 3, 4, 5, 6, 7, 8};
    const int clusters[9] = {1, 2, 4, 6, 8, 9, 10, 12, 16};
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    double best_ms = 1e300;
    // second order: pipelined only; subdomain faces: one cell per thread only
    const int nvar = g->interp == RT_INTERP_QUADRATIC ? 1 : 3;
    for (int vi = ext ? 2 : 0; vi < nvar; ++vi) {
      for (int ai = 0; ai < 7; ++ai) {
        for (int ci = 0; ci < 9; ++ci) {
          if (clusters[ci] > minNv) continue;
          // the evenly spread CTA (planner default) and, if different, the largest
          int balanced = 0;
          for (int ti = 0; ti < 2; ++ti) {
            g->req_variant = variants[vi];
            g->req_apg = apgs[ai];
            g->req_cluster = clusters[ci];
            g->req_threads = ti == 0 ? 0 : sweep_thread_cap(g, variants[vi]);
            plan_groups(g);
            if (g->groups.empty() || g->smem > kSweepSmemBudget || g->apg != apgs[ai] || g->cluster != clusters[ci])
              break;
            if (ti == 0) balanced = g->threads;
            else if (g->threads == balanced) break;
            if ((r = upload_plan_any(g)) != RT_OK) return r;
            float ms = 1e30f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {   // one warm-up, the best of three
              CU(cudaEventRecord(e0, s));
              r = g->desc.prec == RT_PREC_FP64 ? formal_once<double>(g, s) : formal_once<float>(g, s);
              if (r != RT_OK) { ok = false; cudaGetLastError(); break; }
              CU(cudaEventRecord(e1, s));
              CU(cudaEventSynchronize(e1));
              float t = 0.0f;
              CU(cudaEventElapsedTime(&t, e0, e1));
              if (rep > 0) ms = std::min(ms, t);
            }
            if (ok && ms < best_ms) {
              best_ms = ms;
              best = TuneVal{variants[vi], apgs[ai], clusters[ci], g->req_threads};
            }
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best.variant == 0) {
      g->req_apg = saved[0]; g->req_cluster = saved[1]; g->req_threads = saved[2]; g->req_variant = saved[3];
      plan_groups(g);
      upload_plan_any(g);
      return fail(RT_ERR_CUDA, "autotune found no runnable sweep configuration");
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.push_back({key, best});
  }
  g->req_variant = best.variant;
  g->req_apg = best.apg;
  g->req_cluster = best.cluster;
  g->req_threads = best.threads;
  plan_groups(g);
  if ((r = upload_plan_any(g)) != RT_OK) return r;
  // leave the solver state as rt_set_opacity_source does: S = B, fresh ghosts
  CU(cudaMemcpyAsync(g->S, g->B, (size_t)N_of(g) * 8, cudaMemcpyDeviceToDevice, s));
  if ((r = permute_any(g, g->S, g->SP, s)) != RT_OK) return r;
  if ((r = init_ghosts_any(g, g->S, s)) != RT_OK) return r;
  g->last_incremental = false;
  g->sp_is_delta = false;
  CU(cudaStreamSynchronize(s));
  if (plan_out) return rt_get_sweep_plan(g, plan_out);
  return RT_OK;
}

rt_status rt_get_sweep_plan(rt_grid g, int *plan) {
  if (!g || !plan) return fail(RT_ERR_ARG, "NULL argument");
  plan[0] = g->variant;
  plan[1] = (int)g->groups.size();
  plan[2] = g->slots;
  plan[3] = g->cluster;
  plan[4] = g->threads;
  plan[5] = (int)g->smem;
  plan[6] = (int)g->bins64.size();
  return RT_OK;
}

rt_status rt_get_stats(rt_grid g, rt_stats *out) {
  if (!g || !out) return fail(RT_ERR_ARG, "NULL argument");
  *out = g->stats;
  out->kernel_launches = g->launches;
  out->graph_launches = g->graph_launches;
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------- lock-step solves
// Jacobi ALI solves of several grids advanced together on one stream.  Every
// iteration: one shared sweep launch per set of grids whose pipelined sweeps can
// share a launch (same precision, cluster size and row vectorisation; up to
// kMultiMax grids each), a launch of its own for any other grid's sweep, then
// each grid's Jacobi update and decision.  Each grid goes through the same
// iterations as rt_ali_solve: the same kernels on the same data (a cell's
// arithmetic does not depend on the CTA size or on the other grids of the
// launch), its host checks after the same iterations (batches of 4, doubling to
// 64, or check_every) and so its FP64 iterations on the same iterations -- the
// results are the same bit for bit.  The step runs up to the nearest check of
// any member, so members that began at different times are checked on their
// own schedules.
struct LsMember {
  rt_grid g = nullptr;
  void *tag = nullptr;
  rt_solve_opts opts{};
  int max_iter = 1000;
  bool f32 = false;
  int incremental = 0;
  rtk::SweepArgs<float> Af{};
  rtk::AliArgs<float> Lf{};
  rtk::SweepArgs<double> Ad{};
  rtk::AliArgs<double> Ld{};
  int enqueued = 0, batch = 4, next_check = 0;
  bool fp64_its = false, anchor_next = false;
  double anchor_ref = -1.0;
  rtk::SolveState hs{};
};

struct rt_lockstep_s {
  cudaStream_t s = nullptr;
  std::vector<LsMember *> m;
  rtk::SolveState *hs = nullptr;   // pinned, one per member
  size_t hs_cap = 0;
  long long shared = 0;
};

rt_status ls_create(cudaStream_t s, rt_lockstep *out) {
  if (!out) return fail(RT_ERR_ARG, "NULL out");
  rt_lockstep L = new rt_lockstep_s();
  L->s = s;
  *out = L;
  return RT_OK;
}

void ls_destroy(rt_lockstep L) {
  if (!L) return;
  for (LsMember *x : L->m) delete x;
  if (L->hs) cudaFreeHost(L->hs);
  delete L;
}

size_t ls_size(rt_lockstep L) { return L ? L->m.size() : 0; }
long long ls_shared_launches(rt_lockstep L) { return L ? L->shared : 0; }
void ls_reset_shared(rt_lockstep L) {
  if (L) L->shared = 0;
}

rt_status ls_add(rt_lockstep L, rt_grid g, const rt_solve_opts *opts, void *tag) {
  if (!L || !g) return fail(RT_ERR_ARG, "NULL argument");
  if (!g->have_medium) return fail(RT_ERR_STATE, "rt_set_opacity_source has not succeeded");
  if (g->iteration == RT_ITER_GAUSS_SEIDEL || g->interp != RT_INTERP_LINEAR)
    return fail(RT_ERR_STATE, "lock-step solves take the Jacobi iteration with linear interpolation");
  if (opts && !(opts->tol >= 0.0)) return fail(RT_ERR_ARG, "tol must be >= 0");
  g->stepped = false;
  cudaStream_t s = L->s;
  if (s != g->own) CU(cudaStreamSynchronize(g->own));
  rt_status r = solve_prologue(g, nullptr, 0, s);
  if (r != RT_OK) return r;
  LsMember *x = new LsMember();
  x->g = g;
  x->tag = tag;
  x->opts = opts ? *opts : rt_solve_opts{1e-6, 1000, 0, nullptr};
  x->opts.stream = (void *)s;
  x->max_iter = x->opts.max_iter > 0 ? x->opts.max_iter : 1000;
  x->f32 = g->desc.prec == RT_PREC_MIXED;
  x->incremental = x->f32 ? 1 : 0;
  x->batch = x->opts.check_every > 0 ? x->opts.check_every : 4;
  auto bail = [&](rt_status e) { delete x; return e; };
  if (cudaSuccess != rtk::launch_state_op(g->st, 0, x->max_iter, x->opts.tol, g->lte ? 1 : 0, s))
    return bail(fail(RT_ERR_CUDA, "state reset launch failed"));
  g->launches++;
  g->stats.first_fp64 = 0;
  g->stats.fp64_anchors = 0;
  if (x->f32) {
    if ((r = ensure_seg_table<float>(g, s)) != RT_OK) return bail(r);
    solve_args<float>(g, x->incremental, false, x->Af, x->Lf);
    x->fp64_its = g->fp64_first && g->first64 && !g->lte;
    if (x->fp64_its) {
      if ((r = fp64_iteration(g, x->Lf, 0, true, s)) != RT_OK) return bail(r);
      x->enqueued = 1;
      g->stats.first_fp64 = 1;
    }
  } else {
    if ((r = ensure_seg_table<double>(g, s)) != RT_OK) return bail(r);
    solve_args<double>(g, 0, false, x->Ad, x->Ld);
  }
  x->next_check = x->enqueued + std::min(x->batch, x->max_iter - x->enqueued);
  L->m.push_back(x);
  return RT_OK;
}

namespace {

bool ls_mergeable(const LsMember *x) { return x->g->variant == 3; }

// shared launches of the pipelined sweeps of members `idx` (one precision)
template <typename T>
rt_status ls_sweep_shared(rt_lockstep L, const std::vector<LsMember *> &idx) {
  // sets of the same cluster size and vectorisation
  std::vector<bool> used(idx.size(), false);
  for (size_t i = 0; i < idx.size(); ++i) {
    if (used[i]) continue;
    const rt_grid g0 = idx[i]->g;
    // (rows of every sweep axis a multiple of 4 cells: the float32 kernel's 128-bit rows)
    const bool v0 = sizeof(T) == 4 && g0->d.n[0] % 4 == 0 && g0->d.n[1] % 4 == 0;
    std::vector<LsMember *> set;
    for (size_t j = i; j < idx.size(); ++j) {
      const rt_grid gj = idx[j]->g;
      const bool vj = sizeof(T) == 4 && gj->d.n[0] % 4 == 0 && gj->d.n[1] % 4 == 0;
      if (!used[j] && gj->cluster == g0->cluster && vj == v0) {
        used[j] = true;
        set.push_back(idx[j]);
      }
    }
    for (size_t k0 = 0; k0 < set.size(); k0 += rtk::kMultiMax) {
      const size_t k1 = std::min(set.size(), k0 + rtk::kMultiMax);
      rtk::MultiSweep<T> M{};
      M.n = (int)(k1 - k0);
      M.base[0] = 0;
      int amax = 1, threads = 32;
      size_t smem = 0;
      for (size_t k = k0; k < k1; ++k) {
        LsMember *x = set[k];
        const int q = (int)(k - k0);
        if constexpr (sizeof(T) == 4) M.a[q] = x->Af;
        else M.a[q] = x->Ad;
        M.base[q + 1] = M.base[q] + (int)x->g->groups.size() * x->g->d.nf;
        amax = std::max(amax, x->g->amax);
        threads = std::max(threads, x->g->threads);
        smem = std::max(smem, x->g->smem);
        x->g->launches++;
        if (M.n > 1) x->g->stats.shared_launches++;
      }
      CU(rtk::launch_sweep_multi<T>(M, amax, threads, smem, L->s));
      L->shared++;
    }
  }
  return RT_OK;
}

template <typename T>
rt_status ls_update(LsMember *x, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) CU(rtk::launch_ali<float>(x->Lf, s));
  else CU(rtk::launch_ali<double>(x->Ld, s));
  CU(rtk::launch_finish(x->g->st, s));
  x->g->launches += 2;
  return RT_OK;
}

}  // namespace

rt_status ls_step(rt_lockstep L, std::vector<LsResult> *done) {
  if (!L) return fail(RT_ERR_ARG, "NULL lock-step set");
  cudaStream_t s = L->s;
  int m = INT_MAX;
  for (LsMember *x : L->m) m = std::min(m, x->next_check - x->enqueued);
  if (L->m.empty()) m = 0;
  for (int it = 0; it < m; ++it) {
    std::vector<LsMember *> sh32, sh64, own;
    for (LsMember *x : L->m) {
      if (it == 0 && x->anchor_next) {   // this batch of x begins with an FP64 iteration
        rt_status r = fp64_iteration(x->g, x->Lf, (x->hs.fs_count + x->Af.parity_offset) & 1, false, s);
        if (r != RT_OK) return r;
        x->g->stats.fp64_anchors++;
        x->anchor_next = false;
        x->enqueued++;
        continue;
      }
      (ls_mergeable(x) ? (x->f32 ? sh32 : sh64) : own).push_back(x);
    }
    rt_status r;
    if (!sh32.empty() && (r = ls_sweep_shared<float>(L, sh32)) != RT_OK) return r;
    if (!sh64.empty() && (r = ls_sweep_shared<double>(L, sh64)) != RT_OK) return r;
    for (LsMember *x : own) {
      r = x->f32 ? enqueue_sweep<float>(x->g, x->Af, false, s, nullptr)
                 : enqueue_sweep<double>(x->g, x->Ad, false, s, nullptr);
      if (r != RT_OK) return r;
    }
    for (auto *v : {&sh32, &sh64, &own})
      for (LsMember *x : *v) {
        r = x->f32 ? ls_update<float>(x, s) : ls_update<double>(x, s);
        if (r != RT_OK) return r;
        x->enqueued++;
      }
  }
  // every member's state, then the members at their checks
  if (L->m.size() > L->hs_cap) {
    if (L->hs) cudaFreeHost(L->hs);
    L->hs = nullptr;
    L->hs_cap = 0;
    CU(cudaMallocHost((void **)&L->hs, L->m.size() * sizeof(rtk::SolveState)));
    L->hs_cap = L->m.size();
  }
  for (size_t i = 0; i < L->m.size(); ++i)
    CU(cudaMemcpyAsync(&L->hs[i], L->m[i]->g->st, sizeof(rtk::SolveState), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  std::vector<LsMember *> keep;
  for (size_t i = 0; i < L->m.size(); ++i) {
    LsMember *x = L->m[i];
    x->hs = L->hs[i];
    if (x->enqueued < x->next_check) {
      keep.push_back(x);
      continue;
    }
    rt_grid g = x->g;
    const rtk::SolveState &hs = x->hs;
    bool finished = true;
    rt_status st = RT_OK;
    if (hs.err) {
      st = fail(RT_ERR_CUDA, "device check failed (code %d, index %d)", hs.err, hs.err_info);
    } else if (!(hs.done || x->enqueued >= x->max_iter)) {
      finished = false;
      if (x->fp64_its && g->anchor_drop > 0.0) {
        if (x->anchor_ref < 0.0) {
          x->anchor_ref = hs.last_resid;
        } else if (hs.last_resid <= x->anchor_ref * g->anchor_drop) {
          x->anchor_next = true;
          x->anchor_ref = hs.last_resid;
        }
      }
      if (!(x->opts.check_every > 0)) x->batch = std::min(x->batch * 2, 64);
      x->next_check = x->enqueued + std::min(x->batch, x->max_iter - x->enqueued);
    }
    if (!finished) {
      keep.push_back(x);
      continue;
    }
    int iters = hs.iter;
    double resid = hs.last_resid;
    bool conv = hs.converged != 0;
    if (st == RT_OK) {
      g->fs_total = hs.fs_count;
      g->last_fs_from_Sfs = !g->lte;
      g->last_incremental = x->incremental != 0;
      g->sp_is_delta = x->incremental != 0;
      st = solve_epilogue(g, nullptr, 0, &x->opts, s, &iters, &resid, &conv);
    }
    done->push_back(LsResult{g, x->tag, st, iters, resid, st == RT_OK ? std::string() : g_err});
    delete x;
  }
  L->m.swap(keep);
  return RT_OK;
}

extern "C" rt_status rt_ali_solve_many(rt_grid *grids, int n, const rt_solve_opts *opts, int *iters,
                                       double *resid, int *status) {
  if (n < 0 || (n > 0 && !grids)) return fail(RT_ERR_ARG, "NULL grids or n < 0");
  for (int i = 0; i < n; ++i) {
    if (!grids[i]) return fail(RT_ERR_ARG, "grid %d is NULL", i);
    if (!grids[i]->have_medium) return fail(RT_ERR_STATE, "grid %d: rt_set_opacity_source has not succeeded", i);
    if (grids[i]->iteration == RT_ITER_GAUSS_SEIDEL || grids[i]->interp != RT_INTERP_LINEAR)
      return fail(RT_ERR_STATE, "grid %d: lock-step solves take the Jacobi iteration with linear interpolation", i);
  }
  if (opts && !(opts->tol >= 0.0)) return fail(RT_ERR_ARG, "tol must be >= 0");
  cudaStream_t s = opts && opts->stream ? (cudaStream_t)opts->stream : (n > 0 ? grids[0]->own : nullptr);
  rt_lockstep L = nullptr;
  rt_status r = ls_create(s, &L);
  if (r != RT_OK) return r;
  std::vector<int> idx(n);
  rt_status first = RT_OK;
  std::string first_msg;
  for (int i = 0; i < n; ++i) {
    idx[i] = i;
    if ((r = ls_add(L, grids[i], opts, &idx[i])) != RT_OK) {
      ls_destroy(L);
      return r;
    }
  }
  std::vector<LsResult> done;
  while (ls_size(L) > 0) {
    if ((r = ls_step(L, &done)) != RT_OK) {
      ls_destroy(L);
      return r;
    }
  }
  ls_destroy(L);
  for (const LsResult &d : done) {
    const int i = *(const int *)d.tag;
    if (iters) iters[i] = d.iters;
    if (resid) resid[i] = d.resid;
    if (status) status[i] = d.status;
    if (d.status != RT_OK && first == RT_OK) {
      first = d.status;
      first_msg = d.message;
    }
  }
  return first == RT_OK ? RT_OK : fail(first, "%s", first_msg.c_str());
}

// ----------------------------------------------------- allocation-free formal solution
// Working memory for rt_formal_solve_noalloc: one array in this library's device
// image.  Every GPU that loads the library holds it until the process exits;
// every call uses it, so calls that overlap on the GPU race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};   // device address of g_noalloc_scratch per device ordinal

// Looked up once per device, with that device current (host code cannot use the
// array's name as a device address).
rt_status noalloc_base(char **out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(RT_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(RT_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = (char *)g_noalloc_addr[dev];
  return RT_OK;
}

// Carves 256-byte aligned pieces off the scratch array (or measures, with base NULL).
struct ScratchCarver {
  char *base;
  size_t off = 0;
  void *take(size_t bytes) {
    const size_t a = (off + 255) & ~(size_t)255;
    off = a + bytes;
    return base ? base + a : nullptr;
  }
};

template <typename T>
rt_status noalloc_run(rt_grid_s &g, const double *chi, const double *S, const double *B, double *J,
                      cudaStream_t s) {
  // the same per-ray constants as a grid's sweep plan
  std::vector<AngleParam<T>> ap(g.group_angles.size());
  for (size_t gi = 0; gi < g.groups.size(); ++gi) {
    const GroupParam &gp = g.groups[gi];
    int cax[3];
    rtk::plane_axes(gp.axis, cax);
    for (int q = 0; q < gp.na; ++q) {
      const int k = g.group_angles[gp.a0 + q];
      const RayGeom &r = g.rays[k];
      const double fu = r.frac[cax[0]], fv = r.frac[cax[1]];
      AngleParam<T> p{};
      p.wq = (T)r.w;
      p.hs = (T)(0.5 * r.s);
      p.wa = (T)((1.0 - fu) * (1.0 - fv));
      p.wb = (T)(fu * (1.0 - fv));
      p.wc = (T)((1.0 - fu) * fv);
      p.wd = (T)(fu * fv);
      for (int a = 0; a < 3; ++a) p.mu[a] = (T)g.mu[3 * k + a];
      p.su = r.sgn[cax[0]];
      p.sv = r.sgn[cax[1]];
      p.angle = k;
      ap[gp.a0 + q] = p;
    }
  }
  const size_t N = (size_t)g.d.cells * g.d.nf;
  const size_t gbytes = (size_t)g.d.nf * g.na * g.d.gsize * sizeof(T);
  auto layout = [&](ScratchCarver &c) {
    g.st = (rtk::SolveState *)c.take(sizeof(rtk::SolveState));
    g.angp = c.take(std::max<size_t>(1, ap.size()) * sizeof(AngleParam<T>));
    g.grp = (GroupParam *)c.take(std::max<size_t>(1, g.groups.size()) * sizeof(GroupParam));
    g.rays_d = (RayGeom *)c.take((size_t)g.na * sizeof(RayGeom));
    for (int a = 0; a < 3; ++a) {
      g.chiP[a] = g.used_axis[a] ? c.take(N * sizeof(T)) : nullptr;
      g.SP[a] = g.used_axis[a] ? c.take(N * sizeof(T)) : nullptr;
    }
    g.G[0] = c.take(gbytes);
    g.G[1] = c.take(gbytes);
    for (int f = 0; f < 6; ++f)
      g.Ibc[f] = g.d.periodic[f / 2] ? nullptr : c.take((size_t)g.d.nf * g.na * g.d.face[f / 2] * sizeof(T));
    g.Jpart = c.take(g.groups.size() * N * sizeof(T));
  };
  ScratchCarver measure{nullptr};
  layout(measure);
  if (measure.off > RT_NOALLOC_SCRATCH_BYTES)
    return fail(RT_ERR_ARG, "rt_formal_solve_noalloc: this problem needs %zu bytes of scratch, more than the %llu available",
                measure.off, (unsigned long long)RT_NOALLOC_SCRATCH_BYTES);
  if (!chi || !S || !B || !J) return fail(RT_ERR_ARG, "rt_formal_solve_noalloc: NULL array");
  char *base = nullptr;
  rt_status r = noalloc_base(&base);
  if (r != RT_OK) return r;
  ScratchCarver carve{base};
  layout(carve);
  g.jpart_groups = g.groups.size();
  g.chi = const_cast<double *>(chi);
  g.B = const_cast<double *>(B);
  g.J = J;
  // the array keeps the previous call's contents: only the control block must start at zero
  CU(cudaMemsetAsync(g.st, 0, sizeof(rtk::SolveState), s));
  CU(cudaMemcpyAsync(g.angp, ap.data(), ap.size() * sizeof(AngleParam<T>), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(g.grp, g.groups.data(), g.groups.size() * sizeof(GroupParam), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(g.rays_d, g.rays.data(), g.na * sizeof(RayGeom), cudaMemcpyHostToDevice, s));
  if ((r = permute_into<T>(&g, chi, g.chiP, s)) != RT_OK) return r;
  if ((r = permute_into<T>(&g, S, g.SP, s)) != RT_OK) return r;
  if ((r = init_ghosts<T>(&g, S, s)) != RT_OK) return r;
  for (int f = 0; f < 6; ++f)
    if ((r = fill_bc<T>(&g, f, s)) != RT_OK) return r;
  if ((r = formal_once<T>(&g, s)) != RT_OK) return r;
  CU(cudaStreamSynchronize(s));   // also keeps the host tables alive until copied
  return check_device_error(&g);
}

}  // namespace

extern "C" rt_status rt_formal_solve_noalloc(const rt_grid_desc *desc, const double *chi, const double *S,
                                             const double *B, double *J_out, void *stream) {
  if (!desc) return fail(RT_ERR_ARG, "rt_formal_solve_noalloc: NULL descriptor");
  const rt_grid_desc &D = *desc;
  if (D.nx < 1 || D.ny < 1 || D.nz < 1 || D.nfreq < 1) return fail(RT_ERR_ARG, "grid sizes and nfreq must be >= 1");
  if (!(D.dx > 0) || !(D.dy > 0) || (D.nz > 1 && !(D.dz > 0))) return fail(RT_ERR_ARG, "cell spacings must be > 0");
  if (D.prec != RT_PREC_FP64 && D.prec != RT_PREC_MIXED) return fail(RT_ERR_ARG, "bad precision");
  for (int a = 0; a < 3; ++a) {
    if (D.bc_lo[a] < 0 || D.bc_lo[a] > 2 || D.bc_hi[a] < 0 || D.bc_hi[a] > 2)
      return fail(RT_ERR_ARG, "rt_formal_solve_noalloc supports periodic, vacuum and thermal faces only");
    if ((a < 2 || D.nz > 1) && (D.bc_lo[a] == RT_BC_PERIODIC) != (D.bc_hi[a] == RT_BC_PERIODIC))
      return fail(RT_ERR_ARG, "axis %d: a periodic axis must be periodic on both faces", a);
  }
  // the size limit is checked before any pointer is touched
  rt_grid_s g;
  g.wt_off = true;   // no segment-weight table: this entry point allocates nothing
  g.desc = D;
  g.two_d = D.nz == 1;
  if (g.two_d) {
    g.desc.bc_lo[2] = g.desc.bc_hi[2] = RT_BC_PERIODIC;
    g.desc.dz = 1.0;
  }
  if (!level_symmetric(D.n_mu, g.two_d, g.mu, g.wq))
    return fail(RT_ERR_ARG, "n_mu must be 2, 4, 6, 8, 10 or 12 (got %d)", D.n_mu);
  g.na = (int)g.wq.size();
  g.tsize = D.prec == RT_PREC_FP64 ? 8 : 4;
  g.d.n[0] = D.nx;
  g.d.n[1] = D.ny;
  g.d.n[2] = D.nz;
  g.d.nf = D.nfreq;
  g.d.cells = (long long)D.nx * D.ny * D.nz;
  for (int a = 0; a < 3; ++a) {
    g.d.bc_lo[a] = g.desc.bc_lo[a];
    g.d.bc_hi[a] = g.desc.bc_hi[a];
    g.d.periodic[a] = g.desc.bc_lo[a] == RT_BC_PERIODIC;
  }
  g.d.face[0] = (long long)D.nz * D.ny;
  g.d.face[1] = (long long)D.nz * D.nx;
  g.d.face[2] = (long long)D.ny * D.nx;
  g.d.gsize = g.d.face[0] + g.d.face[1] + g.d.face[2];
  build_rays(&g);
  plan_groups(&g);
  cudaStream_t s = (cudaStream_t)stream;
  return D.prec == RT_PREC_FP64 ? noalloc_run<double>(g, chi, S, B, J_out, s)
                                : noalloc_run<float>(g, chi, S, B, J_out, s);
}

