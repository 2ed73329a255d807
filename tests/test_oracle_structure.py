"""Further pins of the oracle's formal solution (Sec. 3.3): one ray at a time.

A single ray's intensity is read out by giving that ray weight 1 and every other
ray weight 0 (J = sum_k w_k I_k).

* 1D structure: a z-stratified medium with periodic x, y keeps every column
  identical for every ray, and a ray that crosses the z face (its upwind point
  lies on the plane below, where the medium is uniform) follows exactly the 1D
  short-characteristics recurrence along z with path length dz/|mu_z|, written
  out here with its own exponential weights.
* Long characteristics: on small grids, the SC intensity of a ray approaches
  the formal solution integrated along the whole ray through the trilinear chi
  and S fields (the same extended domain and boundary: vacuum at the ghost
  layer, chi and S held at the boundary layer's values beyond it); the mean gap
  shrinks as the grid is refined (a consistency check of the discretisation).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

P, V, T = O.PERIODIC, O.VACUUM, O.THERMAL


def _one_ray(g, k):
    g1 = O.Grid(*g.n, n_mu=_nmu(g), bc_lo=g.bc_lo, bc_hi=g.bc_hi, dx=g.d[0], dy=g.d[1], dz=g.d[2])
    w = np.zeros(g1.na)
    w[k] = 1.0
    g1.w = w
    return g1


def _nmu(g):
    return {8: 2, 24: 4, 48: 6, 80: 8}[g.na] if not g.two_d else {4: 2, 12: 4, 24: 6, 40: 8}[g.na]


def _settled(g, chi, S, B, n=200, tol=1e-15):
    """Formal solutions with fixed S until the lagged periodic ghosts settle."""
    G = O.init_ghosts(g, S)
    J = None
    for _ in range(n):
        r = O.formal_solution(g, chi, S, B, G_prev=G)
        if J is not None and np.max(np.abs(r["J"] - J)) <= tol * np.max(np.abs(r["J"])):
            return r["J"]
        J, G = r["J"], r["G_next"]
    raise AssertionError("periodic ghosts did not settle")


def _sc_1d_upward(chi_z, S_z, I_bottom, s):
    """1D SC along z for an upward ray: dtau = (chi_{k-1} + chi_k) s / 2, the
    ghost layer below holding the bottom layer's chi and S and I = I_bottom."""
    I = np.empty_like(S_z)
    Im, Sm, cm = I_bottom, S_z[0], chi_z[0]
    for k in range(len(S_z)):
        dt = 0.5 * (cm + chi_z[k]) * s
        e0 = -math.expm1(-dt)
        psi0 = (dt - e0) / dt
        I[k] = Im * (1.0 - e0) + (e0 - psi0) * Sm + psi0 * S_z[k]
        Im, Sm, cm = I[k], S_z[k], chi_z[k]
    return I


def _sc_1d_downward(chi_z, S_z, s):
    return _sc_1d_upward(chi_z[::-1], S_z[::-1], 0.0, s)[::-1]


@pytest.mark.parametrize("n_mu", [4, 6, 8])
def test_stratified_medium_follows_the_1d_recurrence(n_mu):
    nx, ny, nz = 6, 5, 16
    rng = np.random.default_rng(21)
    chi_z = np.exp(rng.uniform(math.log(0.5), math.log(5.0), nz))
    S_z = rng.uniform(0.5, 2.0, nz)
    g = O.Grid(nx, ny, nz, n_mu, (P, P, T), (P, P, V))
    chi = np.broadcast_to(chi_z[:, None, None], g.shape).copy()
    S = np.broadcast_to(S_z[:, None, None], g.shape).copy()
    B = S.copy()
    n_z_rays = 0
    for k in range(g.na):
        mu = g.mu[k]
        I3 = _settled(_one_ray(g, k), chi, S, B)
        # every column identical
        np.testing.assert_allclose(I3, np.broadcast_to(I3[:, :1, :1], g.shape), rtol=1e-12, atol=0)
        # rays crossing the z face (ties go to z): the 1D recurrence exactly
        if abs(mu[2]) >= max(abs(mu[0]), abs(mu[1])) - 1e-12:
            n_z_rays += 1
            s = 1.0 / abs(mu[2])
            I1 = _sc_1d_upward(chi_z, S_z, S_z[0], s) if mu[2] > 0 else _sc_1d_downward(chi_z, S_z, s)
            np.testing.assert_allclose(I3[:, 0, 0], I1, rtol=1e-12)
    assert n_z_rays >= 8


def _trilinear(F, x, y, z):
    """F [nz][ny][nx] at fractional cell-centre indices, held constant beyond the
    outermost cell centres."""
    nz, ny, nx = F.shape
    x = np.clip(x, 0, nx - 1)
    y = np.clip(y, 0, ny - 1)
    z = np.clip(z, 0, nz - 1)
    i0 = np.minimum(np.floor(x).astype(int), nx - 2)
    j0 = np.minimum(np.floor(y).astype(int), ny - 2)
    k0 = np.minimum(np.floor(z).astype(int), nz - 2)
    fx, fy, fz = x - i0, y - j0, z - k0
    out = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                w = (fx if di else 1 - fx) * (fy if dj else 1 - fy) * (fz if dk else 1 - fz)
                out = out + w * F[k0 + dk, j0 + dj, i0 + di]
    return out


def _long_characteristic(chi, S, n, h, steps_per_cell=24):
    """I at every cell centre along direction n (vacuum at the ghost layer, one cell
    outside the outermost centres), integrating dI/dl = chi (S - I) from the
    ghost layer to the cell with the midpoint rule on a fine grid."""
    nz, ny, nx = chi.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = [x.astype(float), y.astype(float), z.astype(float)]
    # path length (physical) back to the ghost layer, along -n
    lmax = np.full(x.shape, np.inf)
    for a, m in enumerate((nx, ny, nz)):
        if n[a] > 0:
            lmax = np.minimum(lmax, (p[a] + 1.0) * h / n[a])
        elif n[a] < 0:
            lmax = np.minimum(lmax, (m - p[a]) * h / -n[a])
    nst = int(math.ceil(lmax.max() / h * steps_per_cell))
    I = np.zeros(x.shape)
    # march from the ghost layer towards the cell: l counts down from lmax to 0
    for q in range(nst):
        l_hi = lmax * (1.0 - q / nst)
        l_lo = lmax * (1.0 - (q + 1) / nst)
        lm = 0.5 * (l_hi + l_lo)
        pts = [p[a] - n[a] * lm / h for a in range(3)]
        c = _trilinear(chi, *pts)
        s = _trilinear(S, *pts)
        dt = c * (l_hi - l_lo)
        I = I * np.exp(-dt) + s * (-np.expm1(-dt))
    return I


def _sc_vs_lc(N, k):
    h = 1.0 / N
    g = O.Grid(N, N, N, 4, (V, V, V), (V, V, V), dx=h, dy=h, dz=h)
    z, y, x = np.meshgrid(*(np.arange(N) * h,) * 3, indexing="ij")
    chi = 3.0 + 1.5 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y) + z
    S = 1.0 + 0.5 * np.cos(2 * math.pi * (x + 0.5 * y)) + 0.3 * z
    I_sc = O.formal_solution(_one_ray(g, k), chi, S, np.zeros_like(S))["J"]
    I_lc = _long_characteristic(chi, S, g.mu[k], h)
    return np.mean(np.abs(I_sc - I_lc)) / np.mean(np.abs(I_lc))


@pytest.mark.parametrize("k", [0, 7, 17])
def test_short_characteristics_approach_long_characteristics(k):
    # mean relative gap: the continuum intensity has a kink along the characteristic
    # from each domain edge, which both schemes smear over a cell, so the largest
    # gap stays O(1) at those cells while the mean falls with the cell size
    e = [_sc_vs_lc(N, k) for N in (6, 12, 24)]   # about 0.06, 0.045, 0.027
    assert e[1] < 0.85 * e[0] and e[2] < 0.75 * e[1], e
    assert e[2] < 0.035, e
