"""FP64 CPU oracle: formal solution, Jacobi ALI and outputs (test infrastructure only).

Follows Davis, Stone & Jiang (2012):
  * ``formal_solution``  - one short-characteristics formal solution J = Lambda[S]
    (Sec. 3.3, Eq. 20 with linear interpolation, or with monotonic quadratic
    face interpolation and second-order Bezier-controlled segment integration),
    also returning the diagonal Lambda* (Sec. 3.4, Olson & Kunasz 1987) and, on
    request, H and K (Eqs. 18-19).  The sweeps are the C functions in
    ``sc_oracle.c``.
  * ``init_ghosts``      - first-iteration periodic ghost intensities: I = S of the
    periodic image cell (the paper lags incoming periodic/subdomain intensities
    by one iteration, Sec. 3; with no previous iteration the image S is used).
  * ``ali_solve``        - Jacobi ALI (Eq. 24; with the second-order scheme Lambda*
    is taken from each formal solution):
        dS = [(1 - eps) J + eps B - S] / [1 - (1 - eps) Lambda*],  S <- S + dS,
    stopped when max |dS|/S <= delta_c (Eq. 25); when every eps = 1 the test uses
    the change of J between consecutive formal solutions (Sec. 3.4).  The
    iteration count is the number of formal solutions performed.
  * ``ali_solve(method="gauss_seidel")`` - the Gauss-Seidel ALI of Sec. 3.4 in
    its plane-wavefront form (``gs_reverse_rays``, ``gs_reverse`` and
    ``orc_gs_reverse`` in sc_oracle.c): forward rays from the old S, then the
    reverse sweep updating S plane by plane with the freshest J.
  * ``slab_ali_solve``   - the same Jacobi ALI on z slabs (the paper's domain
    decomposition, Sec. 3.5): each slab sweeps alone with a one-cell ghost layer
    on its subdomain faces holding the neighbour's chi and S and, lagged by one
    iteration, its intensities (``formal_solution(..., ext=...)``).
  * ``heating_rate``     - Q = 4 pi sum_nu w_nu chi_abs,nu (J_nu - B_nu) (Sec. 4, Q^int).
  * ``heating_rate_dif`` - Q^dif = -4 pi sum_nu w_nu div H_nu (Sec. 4), div H by
    centred differences of the cell-centred H (one-sided at non-periodic faces).
  * ``heating_rate_switch`` - per cell and frequency Q^int where chi dx <= 1,
    else Q^dif (the switch of Sec. 4).

Parity: pinned by tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build
from .quadrature import level_symmetric

PERIODIC, VACUUM, THERMAL, FIXED, EXTERNAL = 0, 1, 2, 3, 4

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_oracle()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        for fn in (lib.orc_formal_solution, lib.orc_formal_solution_quad):
            fn.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ip, ip, ctypes.c_int, d, d, d, d, d, d, d, d, d, d, d, d,
                ctypes.c_int]
            fn.restype = ctypes.c_int
        lib.orc_gs_reverse.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ip, ip, ctypes.c_int, d, d, ip, d, d, d, d, d, d, d, d, d, d, d, d]
        lib.orc_gs_reverse.restype = ctypes.c_int
        lib.orc_gs_is_reverse.argtypes = [ctypes.c_int, d, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double]
        lib.orc_gs_is_reverse.restype = ctypes.c_int
        geo = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
               ctypes.c_double, ip, ip]
        lib.orc_gs_cell_is_reverse.argtypes = lib.orc_gs_is_reverse.argtypes
        lib.orc_gs_cell_is_reverse.restype = ctypes.c_int
        lib.orc_gs_cell_weights.argtypes = geo + [ctypes.c_int, d, d, ip, d, d]
        lib.orc_gs_cell_weights.restype = ctypes.c_int
        lib.orc_gs_cell_reverse.argtypes = geo + [ctypes.c_int, d, d, ip, d, d, d, d, d, d, d, d,
                                                  d, d, ctypes.c_int, d, d, d, d]
        lib.orc_gs_cell_reverse.restype = ctypes.c_int
        lib.orc_formal_solution_ext.argtypes = lib.orc_formal_solution.argtypes + [d] * 11
        lib.orc_formal_solution_ext.restype = ctypes.c_int
        lib.orc_bezier_weights.argtypes = [ctypes.c_double, d]
        lib.orc_bezier_weights.restype = None
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Grid:
    """Uniform Cartesian grid with per-face boundary types and its angle set."""

    def __init__(self, nx, ny, nz, n_mu, bc_lo=(PERIODIC, PERIODIC, THERMAL),
                 bc_hi=(PERIODIC, PERIODIC, VACUUM), dx=1.0, dy=1.0, dz=1.0):
        self.n = (int(nx), int(ny), int(nz))
        self.d = (float(dx), float(dy), float(dz))
        self.bc_lo = tuple(int(b) for b in bc_lo)
        self.bc_hi = tuple(int(b) for b in bc_hi)
        for a in range(3):
            if (self.bc_lo[a] == PERIODIC) != (self.bc_hi[a] == PERIODIC):
                raise ValueError("a periodic axis must be periodic on both faces")
        self.two_d = self.n[2] == 1
        self.mu, self.w = level_symmetric(n_mu, two_d=self.two_d)
        self.na = len(self.w)
        nx, ny, nz = self.n
        self.face = (nz * ny, nz * nx, ny * nx)
        self.goff = (0, self.face[0], self.face[0] + self.face[1])
        self.gsize = sum(self.face)

    @classmethod
    def from_problem(cls, p):
        return cls(p.nx, p.ny, p.nz, p.n_mu, p.bc_lo, p.bc_hi, p.dx, p.dy, p.dz)

    @property
    def cells(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


def init_ghosts(grid: Grid, S: np.ndarray) -> np.ndarray:
    """Ghost block [na][gsize] holding S of the periodic image of each ghost vertex.

    The image of the upwind ghost along axis a is the outflow cell of that axis
    (index n_a - 1 for mu_a > 0, 0 for mu_a < 0)."""
    S = np.asarray(S, dtype=np.float64).reshape(grid.shape)
    G = np.zeros((grid.na, grid.gsize))
    for k in range(grid.na):
        for a in range(3):
            if grid.bc_lo[a] != PERIODIC:
                continue
            out = grid.n[a] - 1 if grid.mu[k, a] >= 0 else 0
            if a == 0:
                face = S[:, :, out]          # [nz][ny]
            elif a == 1:
                face = S[:, out, :]          # [nz][nx]
            else:
                face = S[out, :, :]          # [ny][nx]
            G[k, grid.goff[a]:grid.goff[a] + grid.face[a]] = face.ravel()
    return G


def bezier_weights(dtau):
    """(a, b, c) of the second-order segment integration (see sc_oracle.c)."""
    out = np.empty(3)
    _load().orc_bezier_weights(float(dtau), _ptr(out))
    return out


def _ray_subset_fixed(grid: Grid, I_fixed, rays):
    """Rows of the rays ``rays`` of a [6][na][face] boundary array."""
    out = []
    off = 0
    for f in range(6):
        n = grid.face[f // 2]
        block = I_fixed[off:off + grid.na * n].reshape(grid.na, n)
        out.append(block[rays].ravel())
        off += grid.na * n
    return np.concatenate(out)


def formal_solution(grid: Grid, chi, S, B, G_prev=None, I_fixed=None, moments=False,
                    nthreads=1, interp="linear", rays=None, ext=None, S_ghost=None):
    """One formal solution for one frequency.

    ``interp``: "linear" (bilinear face interpolation, linear S along the segment)
    or "quadratic" (monotonic quadratic face interpolation and second-order
    Bezier-controlled integration of S, Sec. 3.3).

    ``G_prev`` defaults to ``init_ghosts(grid, S)``; ``I_fixed`` is the user
    incident-intensity array for RT_BC_FIXED faces
    ([6][na][face cells], faces x-lo, x-hi, y-lo, y-hi, z-lo, z-hi).
    ``rays``: indices of the rays to solve (default all); J, lstar, H, K then
    sum over those rays only and G_next holds their rows only.
    ``ext`` (linear only): the ghost layers of EXTERNAL z faces, a dict with
    "lo" and/or "hi" entries (chi [ny][nx], S [ny][nx], I [na][ny][nx],
    B [ny][nx]); past such a face an out-of-range non-periodic x or y face
    decides the ghost intensity (thermal: the ghost layer's B), as in the
    undecomposed domain, and otherwise the layer's I applies; the
    result then also holds I_zlo and I_zhi, every ray's intensity on the first
    and last z plane [na][ny][nx].
    ``S_ghost`` (linear only): S at ghost vertices is read from this array
    (the cell it copies or images) instead of from S.
    Returns a dict with J, lstar, G_next (and H [3], K [6] when ``moments``)."""
    lib = _load()
    C = grid.cells
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(-1)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(-1)
    B = np.ascontiguousarray(B, dtype=np.float64).reshape(-1)
    if G_prev is None:
        G_prev = init_ghosts(grid, S)
    G_prev = np.ascontiguousarray(G_prev, dtype=np.float64)
    G_next = G_prev.copy()
    if I_fixed is not None:
        I_fixed = np.ascontiguousarray(I_fixed, dtype=np.float64).reshape(-1)
        need = 2 * grid.na * sum(grid.face)
        if I_fixed.size != need:
            raise ValueError(f"I_fixed must hold {need} values")
    mu, wq, na = grid.mu, grid.w, grid.na
    if rays is not None:
        rays = np.asarray(rays, dtype=np.int64)
        mu, wq, na = grid.mu[rays], grid.w[rays], len(rays)
        G_prev = np.ascontiguousarray(G_prev[rays])
        G_next = G_prev.copy()
        if I_fixed is not None:
            I_fixed = _ray_subset_fixed(grid, I_fixed, rays)
    J = np.empty(C)
    L = np.empty(C)
    H = np.empty(3 * C) if moments else None
    K = np.empty(6 * C) if moments else None
    bl = (ctypes.c_int * 3)(*grid.bc_lo)
    bh = (ctypes.c_int * 3)(*grid.bc_hi)
    mu = np.ascontiguousarray(mu).reshape(-1)
    wq = np.ascontiguousarray(wq)
    fn = {"linear": lib.orc_formal_solution, "quadratic": lib.orc_formal_solution_quad}[interp]
    args = (grid.n[0], grid.n[1], grid.n[2], grid.d[0], grid.d[1],
            grid.d[2], bl, bh, na, _ptr(mu), _ptr(wq),
            _ptr(chi), _ptr(S), _ptr(B), _ptr(I_fixed), _ptr(G_prev),
            _ptr(G_next), _ptr(J), _ptr(L), _ptr(H), _ptr(K),
            int(nthreads))
    Izlo = Izhi = None
    faces_out = ext is not None
    if S_ghost is not None and ext is None:
        ext = {}
    if ext is not None:
        if interp != "linear":
            raise ValueError("external faces are supported with linear interpolation")
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        side = {}
        for key in ("lo", "hi"):
            side[key] = tuple(f64(a) for a in ext[key]) if key in ext else (None, None, None, None)
        nface = grid.n[0] * grid.n[1]
        Izlo = np.empty(na * nface)
        Izhi = np.empty(na * nface)
        Sg = None if S_ghost is None else np.ascontiguousarray(S_ghost, dtype=np.float64).reshape(-1)
        rc = lib.orc_formal_solution_ext(*args, *[_ptr(a) for a in side["lo"]],
                                         *[_ptr(a) for a in side["hi"]], _ptr(Izlo), _ptr(Izhi),
                                         _ptr(Sg))
    else:
        rc = fn(*args)
    if rc != 0:
        raise RuntimeError(f"oracle formal solution failed ({rc})")
    out = dict(J=J.reshape(grid.shape), lstar=L.reshape(grid.shape), G_next=G_next)
    if faces_out:
        out["I_zlo"] = Izlo.reshape(na, grid.n[1], grid.n[0])
        out["I_zhi"] = Izhi.reshape(na, grid.n[1], grid.n[0])
    if moments:
        H = H.reshape((3,) + grid.shape)
        K = K.reshape((6,) + grid.shape)
        if grid.two_d:
            # 2D keeps only mu_z > 0; the mirrored rays (mu_z -> -mu_z) carry the
            # same intensity (Sec. 3.2), so moments odd in mu_z vanish.
            H[2] = 0.0
            K[4] = 0.0
            K[5] = 0.0
        out["H"] = H
        out["K"] = K
    return out


def gs_reverse_rays(grid: Grid) -> np.ndarray:
    """Mask of the reverse rays of the Gauss-Seidel iteration: crossed face
    normal to z (y in 2D), ties with that axis included, and mu along it < 0."""
    lib = _load()
    mu = np.ascontiguousarray(grid.mu).reshape(-1)
    return np.array([bool(lib.orc_gs_is_reverse(grid.n[2], _ptr(mu), k, *grid.d))
                     for k in range(grid.na)])


def gs_reverse(grid: Grid, chi, eps, B, lstar, J_F, S, G_prev, G_next, I_fixed=None):
    """The reverse phase of one Gauss-Seidel iteration for one frequency (see
    orc_gs_reverse).  S is updated in place; G_next receives the reverse rays'
    outflow ghosts.  Returns dict(J, dS, C): the J each cell was updated with,
    the change of S and the first-order correction of the forward rays."""
    lib = _load()
    C = grid.cells
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    chi, eps, B, lstar, J_F = f64(chi), f64(eps), f64(B), f64(lstar), f64(J_F)
    assert S.dtype == np.float64 and S.flags.c_contiguous and S.size == C
    assert G_next.dtype == np.float64 and G_next.flags.c_contiguous
    G_prev = np.ascontiguousarray(G_prev, dtype=np.float64)
    if I_fixed is not None:
        I_fixed = f64(I_fixed)
    rev = np.ascontiguousarray(gs_reverse_rays(grid), dtype=np.int32)
    J = np.empty(C)
    dS = np.empty(C)
    corr = np.empty(C)
    bl = (ctypes.c_int * 3)(*grid.bc_lo)
    bh = (ctypes.c_int * 3)(*grid.bc_hi)
    mu = np.ascontiguousarray(grid.mu).reshape(-1)
    rc = lib.orc_gs_reverse(grid.n[0], grid.n[1], grid.n[2], grid.d[0], grid.d[1], grid.d[2],
                            bl, bh, grid.na, _ptr(mu), _ptr(grid.w),
                            rev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _ptr(chi), _ptr(B), _ptr(eps), _ptr(lstar), _ptr(J_F), _ptr(S),
                            _ptr(I_fixed), _ptr(G_prev), _ptr(G_next), _ptr(J), _ptr(dS),
                            _ptr(corr))
    if rc != 0:
        raise RuntimeError(f"oracle Gauss-Seidel sweep failed ({rc})")
    return dict(J=J.reshape(grid.shape), dS=dS.reshape(grid.shape), C=corr.reshape(grid.shape))


def gs_cell_reverse_rays(grid: Grid) -> np.ndarray:
    """Mask of the reverse rays of the cell-order Gauss-Seidel sweep: mu_V < 0
    and every upwind vertex visited before the cell in decreasing cell index."""
    lib = _load()
    mu = np.ascontiguousarray(grid.mu).reshape(-1)
    return np.array([bool(lib.orc_gs_cell_is_reverse(grid.n[2], _ptr(mu), k, *grid.d))
                     for k in range(grid.na)])


def gs_cell_weights(grid: Grid, chi) -> np.ndarray:
    """The forward rays' correction weights [27][nz][ny][nx] (orc_gs_cell_weights)."""
    lib = _load()
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(-1)
    fwd = np.ascontiguousarray(~gs_cell_reverse_rays(grid), dtype=np.int32)
    Wc = np.empty(27 * grid.cells)
    mu = np.ascontiguousarray(grid.mu).reshape(-1)
    rc = lib.orc_gs_cell_weights(grid.n[0], grid.n[1], grid.n[2], grid.d[0], grid.d[1], grid.d[2],
                                 (ctypes.c_int * 3)(*grid.bc_lo), (ctypes.c_int * 3)(*grid.bc_hi),
                                 grid.na, _ptr(mu), _ptr(grid.w),
                                 fwd.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(chi), _ptr(Wc))
    if rc != 0:
        raise RuntimeError(f"oracle Gauss-Seidel weights failed ({rc})")
    return Wc.reshape((27,) + grid.shape)


def gs_cell_reverse(grid: Grid, chi, eps, B, lstar, J_F, Wc, S, G_prev, G_next, I_fixed=None,
                    update=True):
    """The cell-order reverse sweep of one Gauss-Seidel iteration for one
    frequency (orc_gs_cell_reverse).  S is updated in place (unless
    ``update`` is False); G_next holds the forward rays' outflow of the old S
    and receives the reverse rays' rows.  Returns dict(J, dS, JR, C)."""
    lib = _load()
    C = grid.cells
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    chi, eps, B, lstar, J_F, Wc = f64(chi), f64(eps), f64(B), f64(lstar), f64(J_F), f64(Wc)
    assert S.dtype == np.float64 and S.flags.c_contiguous and S.size == C
    assert G_next.dtype == np.float64 and G_next.flags.c_contiguous
    G_prev = np.ascontiguousarray(G_prev, dtype=np.float64)
    if I_fixed is not None:
        I_fixed = f64(I_fixed)
    rev = np.ascontiguousarray(gs_cell_reverse_rays(grid), dtype=np.int32)
    J, dS, JR, corr = (np.empty(C) for _ in range(4))
    mu = np.ascontiguousarray(grid.mu).reshape(-1)
    rc = lib.orc_gs_cell_reverse(grid.n[0], grid.n[1], grid.n[2], grid.d[0], grid.d[1], grid.d[2],
                                 (ctypes.c_int * 3)(*grid.bc_lo), (ctypes.c_int * 3)(*grid.bc_hi),
                                 grid.na, _ptr(mu), _ptr(grid.w),
                                 rev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _ptr(chi), _ptr(B), _ptr(eps), _ptr(lstar), _ptr(J_F), _ptr(Wc),
                                 _ptr(S), _ptr(I_fixed), _ptr(G_prev), _ptr(G_next), int(bool(update)),
                                 _ptr(J), _ptr(dS), _ptr(JR), _ptr(corr))
    if rc != 0:
        raise RuntimeError(f"oracle Gauss-Seidel sweep failed ({rc})")
    sh = grid.shape
    return dict(J=J.reshape(sh), dS=dS.reshape(sh), JR=JR.reshape(sh), C=corr.reshape(sh))


def max_relative_change(dS: np.ndarray, S: np.ndarray) -> float:
    """max_i |dS_i|/|S_i| (Eq. 25); a cell with S_i = 0 counts 0 if dS_i = 0, else inf."""
    a = np.abs(dS)
    s = np.abs(S)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(s > 0, a / np.where(s > 0, s, 1.0), np.where(a > 0, np.inf, 0.0))
    return float(r.max()) if r.size else 0.0


def heating_rate(chi, eps, J, B, freq_w):
    """Q = 4 pi sum_nu w_nu eps_nu chi_nu (J_nu - B_nu)  (integral form, Sec. 4)."""
    fw = np.asarray(freq_w, dtype=np.float64).reshape((-1,) + (1,) * (np.ndim(J) - 1))
    return 4.0 * math.pi * np.sum(fw * eps * chi * (J - B), axis=0)


def _derivative(F, axis, h, periodic):
    """dF/dx along one array axis of cell-centred values: centred differences
    (F[i+1] - F[i-1]) / 2h, wrapped on a periodic axis; at the first and last
    cell of a non-periodic axis the one-sided difference; zero on an axis of one
    cell."""
    n = F.shape[axis]
    if n == 1:
        return np.zeros_like(F)
    if periodic:
        return (np.roll(F, -1, axis=axis) - np.roll(F, 1, axis=axis)) / (2.0 * h)
    F = np.moveaxis(F, axis, 0)
    out = np.empty_like(F)
    out[1:-1] = (F[2:] - F[:-2]) / (2.0 * h)
    out[0] = (F[1] - F[0]) / h
    out[-1] = (F[-1] - F[-2]) / h
    return np.moveaxis(out, 0, axis)


def divergence(grid: Grid, H):
    """div H per cell for H [..., 3, nz, ny, nx] (components x, y, z)."""
    H = np.asarray(H, dtype=np.float64)
    hx, hy, hz = grid.d
    per = [grid.bc_lo[a] == PERIODIC for a in range(3)]
    return (_derivative(H[..., 0, :, :, :], -1, hx, per[0])
            + _derivative(H[..., 1, :, :, :], -2, hy, per[1])
            + _derivative(H[..., 2, :, :, :], -3, hz, per[2]))


def heating_rate_dif(grid: Grid, H, freq_w):
    """Q^dif = -4 pi sum_nu w_nu div H_nu (differential form, Sec. 4)."""
    divH = divergence(grid, np.asarray(H, dtype=np.float64).reshape((-1, 3) + grid.shape))
    fw = np.asarray(freq_w, dtype=np.float64).reshape((-1, 1, 1, 1))
    return -4.0 * math.pi * np.sum(fw * divH, axis=0)


def cell_width(grid: Grid):
    """Width of a cell in the heating-rate switch: the largest spacing along the
    axes that have more than one cell."""
    return max(grid.d[a] for a in range(3) if grid.n[a] > 1) if max(grid.n) > 1 else grid.d[0]


def heating_rate_switch(grid: Grid, chi, eps, J, B, H, freq_w):
    """Q per cell and frequency: the integral form where chi_nu dx <= 1, else the
    differential form (Sec. 4), summed over frequency with the weights w_nu."""
    chi = np.asarray(chi, dtype=np.float64).reshape((-1,) + grid.shape)
    eps = np.asarray(eps, dtype=np.float64).reshape(chi.shape)
    J = np.asarray(J, dtype=np.float64).reshape(chi.shape)
    B = np.asarray(B, dtype=np.float64).reshape(chi.shape)
    divH = divergence(grid, np.asarray(H, dtype=np.float64).reshape((-1, 3) + grid.shape))
    q_int = eps * chi * (J - B)
    q_dif = -divH
    q = np.where(chi * cell_width(grid) <= 1.0, q_int, q_dif)
    fw = np.asarray(freq_w, dtype=np.float64).reshape((-1, 1, 1, 1))
    return 4.0 * math.pi * np.sum(fw * q, axis=0)


def ali_solve(grid: Grid, chi, eps, B, freq_w=None, tol=1e-6, max_iter=1000, S_init=None,
              I_fixed=None, nthreads=1, moments=True, interp="linear", method="jacobi"):
    """Jacobi (or Gauss-Seidel) ALI to max|dS|/S <= tol (Eqs. 24-25), all
    frequencies per iteration.

    chi, eps, B: [nf][nz][ny][nx].  I_fixed: None or a list (per frequency) of
    user boundary arrays.  Returns dict(S, J, lstar, H, K, f, Q, iters, resid,
    converged, history); J, H, K are those of the last formal solution, S is the
    source function after the last update.

    method="gauss_seidel" (linear interpolation, eps < 1 somewhere): each
    iteration solves the forward rays with the old S, then ``gs_reverse``
    updates S plane by plane; the J, H, K returned are those of a formal
    solution of the S (and ghosts) that the last iteration started from, and
    ``J_gs`` holds the J each cell was last updated with.

    method="gauss_seidel_cell": the paper's cell order (Sec. 3.4): the forward
    rays of ``gs_cell_reverse_rays`` are solved with the old S, then
    ``gs_cell_reverse`` visits the cells by decreasing index, updating each
    cell's S with the reverse rays' J of the current S plus the forward rays'
    J corrected to first order with the weights of ``gs_cell_weights``;
    outputs as for "gauss_seidel"."""
    if method not in ("jacobi", "gauss_seidel", "gauss_seidel_cell"):
        raise ValueError(f"unknown ALI method {method!r}")
    chi = np.asarray(chi, dtype=np.float64).reshape((-1,) + grid.shape)
    eps = np.asarray(eps, dtype=np.float64).reshape(chi.shape)
    B = np.asarray(B, dtype=np.float64).reshape(chi.shape)
    nf = chi.shape[0]
    fw = np.ones(nf) if freq_w is None else np.asarray(freq_w, dtype=np.float64)
    S = B.copy() if S_init is None else np.asarray(S_init, dtype=np.float64).reshape(chi.shape).copy()
    G = [init_ghosts(grid, S[f]) for f in range(nf)]
    lte = bool(np.all(eps == 1.0))
    fixed = (lambda f: None) if I_fixed is None else (lambda f: I_fixed[f])
    lstar = np.empty_like(chi)
    J = np.empty_like(chi)
    J_prev = None
    history = []
    r = math.inf
    it = 0
    S_fs, G_fs = S, G
    gs = method in ("gauss_seidel", "gauss_seidel_cell") and not lte
    cell = method == "gauss_seidel_cell"
    if gs and interp != "linear":
        raise ValueError("the Gauss-Seidel iteration takes linear interpolation")
    if gs:
        fwd = np.flatnonzero(~(gs_cell_reverse_rays(grid) if cell else gs_reverse_rays(grid)))
    else:
        fwd = None
    J_gs = np.empty_like(chi) if gs else None
    Wc = [gs_cell_weights(grid, chi[f]) for f in range(nf)] if (gs and cell) else None
    for it in range(1, max_iter + 1):
        if gs:
            S_new = S.copy()
            dS = np.empty_like(S)
            G_new = []
            for f in range(nf):
                if it == 1:
                    lstar[f] = formal_solution(grid, chi[f], S[f], B[f], G[f], fixed(f),
                                               nthreads=nthreads)["lstar"]
                res = formal_solution(grid, chi[f], S[f], B[f], G[f], fixed(f),
                                      nthreads=nthreads, rays=fwd)
                Gn = G[f].copy()
                Gn[fwd] = res["G_next"]
                Sf = np.ascontiguousarray(S_new[f]).reshape(-1)
                if cell:
                    out = gs_cell_reverse(grid, chi[f], eps[f], B[f], lstar[f], res["J"], Wc[f], Sf,
                                          G[f], Gn, fixed(f))
                else:
                    out = gs_reverse(grid, chi[f], eps[f], B[f], lstar[f], res["J"], Sf, G[f], Gn,
                                     fixed(f))
                S_new[f] = Sf.reshape(grid.shape)
                dS[f] = out["dS"]
                J_gs[f] = out["J"]
                J[f] = out["J"]
                G_new.append(Gn)
            S_fs, G_fs = S, G
            G = G_new
            S = S_new
            r = max_relative_change(dS, S)
            history.append(r)
            if r <= tol:
                break
            continue
        G_new = []
        for f in range(nf):
            res = formal_solution(grid, chi[f], S[f], B[f], G[f], fixed(f), nthreads=nthreads,
                                  interp=interp)
            J[f] = res["J"]
            # the linear scheme's Lambda* depends on chi alone; the second-order
            # scheme's on S too (through its clamps): take it from every solution
            if it == 1 or interp == "quadratic":
                lstar[f] = res["lstar"]
            G_new.append(res["G_next"])
        S_fs, G_fs = S, G
        G = G_new
        if lte:
            r = math.inf if J_prev is None else max_relative_change(J - J_prev, J)
        else:
            dS = ((1.0 - eps) * J + eps * B - S) / (1.0 - (1.0 - eps) * lstar)
            S = S + dS
            r = max_relative_change(dS, S)
        J_prev = J.copy()
        history.append(r)
        if r <= tol:
            break
    if gs:
        # outputs of the formal solution the last iteration started from
        for f in range(nf):
            J[f] = formal_solution(grid, chi[f], S_fs[f], B[f], G_fs[f], fixed(f),
                                   nthreads=nthreads)["J"]
    out = dict(S=S, J=J.copy(), lstar=lstar, iters=it, resid=r, converged=r <= tol,
               history=history, Q=heating_rate(chi, eps, J, B, fw))
    if gs:
        out["J_gs"] = J_gs
    if moments:
        H = np.empty((nf, 3) + grid.shape)
        K = np.empty((nf, 6) + grid.shape)
        for f in range(nf):
            res = formal_solution(grid, chi[f], S_fs[f], B[f], G_fs[f], fixed(f), moments=True,
                                  nthreads=nthreads, interp=interp)
            H[f] = res["H"]
            K[f] = res["K"]
        out["H"] = H
        out["K"] = K
        with np.errstate(divide="ignore", invalid="ignore"):
            out["f"] = K / J[:, None]
    return out


def slab_ali_solve(grid: Grid, chi, eps, B, nslab, freq_w=None, tol=1e-6, max_iter=1000, nthreads=1):
    """Jacobi ALI (Eqs. 24-25) with the z axis split into ``nslab`` slabs (the
    paper's domain decomposition, Sec. 3.5).

    Every slab is solved as a grid of its own.  A face between two slabs (and,
    on a periodic z axis, the wrap) is an EXTERNAL face: its one-cell ghost
    layer holds the neighbour's chi and current S on the adjacent plane and,
    for the rays entering through it, the neighbour's intensities there from
    the previous iteration (before the first, its S, as for periodic ghosts);
    the other faces keep the grid's boundaries.  Lambda* comes from each slab's
    first formal solution, the stopping rule is the global max |dS|/S.
    Returns dict(S, J, iters, resid, converged, history) with J that of the
    last formal solution.  3D grids (nz >= nslab)."""
    chi = np.asarray(chi, dtype=np.float64).reshape((-1,) + grid.shape)
    eps = np.asarray(eps, dtype=np.float64).reshape(chi.shape)
    B = np.asarray(B, dtype=np.float64).reshape(chi.shape)
    nf = chi.shape[0]
    nx, ny, nz = grid.n
    if grid.two_d or not (1 <= nslab <= nz):
        raise ValueError("slabs split the z axis of a 3D grid into 1..nz parts")
    if nslab > 1 and FIXED in tuple(grid.bc_lo[:2]) + tuple(grid.bc_hi[:2]):
        raise ValueError("slabs need x and y faces without fixed incident intensities")
    per_z = grid.bc_lo[2] == PERIODIC
    z0 = [(d * nz) // nslab for d in range(nslab + 1)]
    n_mu = {8: 2, 24: 4, 48: 6, 80: 8, 120: 10, 168: 12}[grid.na]
    slabs = []
    for d in range(nslab):
        lo = EXTERNAL if (d > 0 or per_z) else grid.bc_lo[2]
        hi = EXTERNAL if (d < nslab - 1 or per_z) else grid.bc_hi[2]
        slabs.append(Grid(nx, ny, z0[d + 1] - z0[d], n_mu, bc_lo=(grid.bc_lo[0], grid.bc_lo[1], lo),
                          bc_hi=(grid.bc_hi[0], grid.bc_hi[1], hi), dx=grid.d[0], dy=grid.d[1], dz=grid.d[2]))
    S = B.copy()
    lte = bool(np.all(eps == 1.0))
    # incoming intensities of each slab's z faces: [f][d] -> [na][ny][nx]
    below = lambda d: (z0[d] - 1) % nz      # global plane under slab d
    above = lambda d: z0[d + 1] % nz        # global plane over slab d
    I_lo = [[np.repeat(S[f, below(d)][None], grid.na, axis=0) for d in range(nslab)] for f in range(nf)]
    I_hi = [[np.repeat(S[f, above(d)][None], grid.na, axis=0) for d in range(nslab)] for f in range(nf)]
    G = [[init_ghosts(slabs[d], S[f, z0[d]:z0[d + 1]]) for d in range(nslab)] for f in range(nf)]
    lstar = np.empty_like(chi)
    J = np.empty_like(chi)
    J_prev = None
    history = []
    r = math.inf
    it = 0
    for it in range(1, max_iter + 1):
        out_lo, out_hi = [[None] * nslab for _ in range(nf)], [[None] * nslab for _ in range(nf)]
        for f in range(nf):
            for d in range(nslab):
                g = slabs[d]
                sl = slice(z0[d], z0[d + 1])
                ext = {}
                if g.bc_lo[2] == EXTERNAL:
                    ext["lo"] = (chi[f, below(d)], S[f, below(d)], I_lo[f][d], B[f, below(d)])
                if g.bc_hi[2] == EXTERNAL:
                    ext["hi"] = (chi[f, above(d)], S[f, above(d)], I_hi[f][d], B[f, above(d)])
                res = formal_solution(g, chi[f, sl], S[f, sl], B[f, sl], G[f][d], nthreads=nthreads, ext=ext)
                J[f, sl] = res["J"]
                if it == 1:
                    lstar[f, sl] = res["lstar"]
                G[f][d] = res["G_next"]
                out_lo[f][d], out_hi[f][d] = res["I_zlo"], res["I_zhi"]
        # the neighbours' intensities for the next iteration: slab d's top plane
        # feeds the slab above's lower ghost layer, its bottom plane the slab below's
        for f in range(nf):
            for d in range(nslab):
                I_lo[f][d] = out_hi[f][(d - 1) % nslab]
                I_hi[f][d] = out_lo[f][(d + 1) % nslab]
        if lte:
            r = math.inf if J_prev is None else max_relative_change(J - J_prev, J)
        else:
            dS = ((1.0 - eps) * J + eps * B - S) / (1.0 - (1.0 - eps) * lstar)
            S = S + dS
            r = max_relative_change(dS, S)
        J_prev = J.copy()
        history.append(r)
        if r <= tol:
            break
    return dict(S=S, J=J.copy(), iters=it, resid=r, converged=r <= tol, history=history)


def solve_problem(p, **kw):
    """ALI solve of a ``workloads.Problem``."""
    g = Grid.from_problem(p)
    kw.setdefault("tol", p.tol)
    return g, ali_solve(g, p.chi, p.eps, p.B, p.freq_w, **kw)
