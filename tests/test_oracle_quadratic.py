"""Pins of the oracle's second-order formal solution (Sec. 3.3): monotonic
quadratic interpolation on the crossed face and Bezier-controlled parabolic
integration of S along the segment.

* The segment weights against direct numerical quadrature of the Bernstein
  polynomials times exp(-(dtau - t)), on both sides of the series threshold.
* Constant S is preserved exactly (the weights sum to 1 - exp(-dtau); the
  interpolants of constants are constants).
* A quadratic S in a uniform medium, monotone along every ray and face axis (so
  neither clamp acts),
  is transported exactly: along each ray I = S - S'/chi + S''/chi^2 (primes: d/ds
  along the ray), so J = S + lap(S) / (3 chi^2) -- on cells far enough from the
  inflow faces for the boundary copies to have decayed.  The linear scheme is
  not exact for the same field (the test separates the two).
* No new extrema: a step in S keeps every intensity inside [min S, max S].
* A searchlight beam crossing the grid at a slant through vacuum spreads much
  less than with linear interpolation (the paper's reason for the option) and
  stays on the geometric ray to within a cell or so.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O

P, V, T, F = O.PERIODIC, O.VACUUM, O.THERMAL, O.FIXED


@pytest.mark.parametrize("t", [1e-6, 1e-3, 0.05, 0.0999, 0.1001, 0.7, 3.0, 40.0])
def test_bezier_weights_match_quadrature(t):
    w = O.bezier_weights(t)
    ref = [quad(f, 0, t, epsabs=0, epsrel=1e-13, limit=200)[0] for f in (
        lambda x: (x / t) ** 2 * math.exp(-x),
        lambda x: (1 - x / t) ** 2 * math.exp(-x),
        lambda x: 2 * (x / t) * (1 - x / t) * math.exp(-x))]
    np.testing.assert_allclose(w, ref, rtol=1e-12)
    assert abs(w.sum() + math.expm1(-t)) <= 1e-15 * max(1.0, t)


@pytest.mark.parametrize("n_mu", [4, 8])
@pytest.mark.parametrize("per", [True, False])
def test_constant_source_preserved(n_mu, per):
    bc = (P, P, P) if per else (T, T, T)
    g = O.Grid(6, 5, 7, n_mu, bc, bc, dx=1.0, dy=1.3, dz=0.8)
    rng = np.random.default_rng(3)
    chi = np.exp(rng.uniform(-4, 2, g.shape))
    S = np.full(g.shape, 1.7)
    r = O.formal_solution(g, chi, S, S.copy(), interp="quadratic")
    np.testing.assert_allclose(r["J"], 1.7, rtol=1e-13)


def _quadratic_field(g):
    nx, ny, nz = g.n
    z, y, x = np.meshgrid(np.arange(nz) * g.d[2], np.arange(ny) * g.d[1], np.arange(nx) * g.d[0],
                          indexing="ij")
    # the y slope dominates (every ray of these sets has |mu_y| >= 0.2), so S is
    # monotone along every ray and along every face axis in the tested cells
    c = 1e-3
    S = 5.0 + y + c * (x * x + z * z + x * y + y * z)
    grad = (c * (2 * x + y), 1.0 + c * (x + z), c * (2 * z + y))
    hess = c * np.array([[2.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 2.0]])
    return S, grad, hess


def _one_ray(g, k):
    g1 = O.Grid(*g.n, n_mu={24: 4, 48: 6, 80: 8}[g.na], bc_lo=g.bc_lo, bc_hi=g.bc_hi,
                dx=g.d[0], dy=g.d[1], dz=g.d[2])
    g1.w = np.eye(g1.na)[k]
    return g1


@pytest.mark.parametrize("n_mu", [4, 6, 8])
def test_quadratic_source_transported_exactly(n_mu):
    chi0, n, band = 5.0, 20, 7
    g = O.Grid(n, n, n, n_mu, (T, T, T), (T, T, T))
    S, grad, hess = _quadratic_field(g)
    chi = np.full(g.shape, chi0)
    core = (slice(band, n - band),) * 3
    worst_lin = 0.0
    for k in range(0, g.na, 3):
        m = g.mu[k]
        d1 = m[0] * grad[0] + m[1] * grad[1] + m[2] * grad[2]
        d2 = m @ hess @ m
        want = S - d1 / chi0 + d2 / chi0 ** 2
        g1 = _one_ray(g, k)
        I = O.formal_solution(g1, chi, S, S.copy(), interp="quadratic")["J"]
        np.testing.assert_allclose(I[core], want[core], rtol=1e-11)
        I_lin = O.formal_solution(g1, chi, S, S.copy())["J"]
        worst_lin = max(worst_lin, np.max(np.abs(I_lin[core] / want[core] - 1)))
    assert worst_lin > 1e-6
    # and the angle sum: J = S + lap S / (3 chi^2)
    J = O.formal_solution(g, chi, S, S.copy(), interp="quadratic")["J"]
    np.testing.assert_allclose(J[core], (S + np.trace(hess) / (3 * chi0 ** 2))[core], rtol=1e-11)


def test_no_new_extrema_at_a_step():
    g = O.Grid(12, 10, 14, 8, (P, P, P), (P, P, P))
    rng = np.random.default_rng(5)
    chi = np.exp(rng.uniform(-3, 2, g.shape))
    S = np.where(np.arange(12)[None, None, :] < 6, 0.2, 3.0) * np.ones(g.shape)
    G = O.init_ghosts(g, S)
    for _ in range(6):   # let the lagged periodic ghosts settle a little
        r = O.formal_solution(g, chi, S, S, G_prev=G, interp="quadratic")
        G = r["G_next"]
    assert r["J"].min() >= 0.2 - 1e-12 and r["J"].max() <= 3.0 + 1e-12
    for k in range(0, g.na, 4):
        I = O.formal_solution(_one_ray(g, k), chi, S, S, G_prev=G, interp="quadratic")["J"]
        assert I.min() >= 0.2 - 1e-12 and I.max() <= 3.0 + 1e-12, (k, I.min(), I.max())


def _beam(interp, nplanes=24):
    n = 40
    g = O.Grid(n, n, nplanes, 4, (V, V, F), (V, V, V))
    k = next(i for i in range(g.na) if np.all(g.mu[i] > 0))   # mu = (0.35, 0.35, 0.87)
    m = g.mu[k]
    x0 = y0 = 8
    def fill(a, side, ang, i, j, kk):
        return 1.0 if (a == 2 and side == 0 and ang == k and i == x0 and j == y0) else 0.0
    I_fixed = _fixed_faces(g, fill)
    g1 = _one_ray(g, k)
    I = O.formal_solution(g1, np.zeros(g.shape), np.zeros(g.shape), np.zeros(g.shape),
                          I_fixed=I_fixed, interp=interp)["J"]
    top = I[-1]
    tot = top.sum()
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cx, cy = (top * xx).sum() / tot, (top * yy).sum() / tot
    var = ((top * (xx - cx) ** 2).sum() + (top * (yy - cy) ** 2).sum()) / tot
    # geometric ray: from the ghost vertex below (x0, y0) up nplanes planes
    gx = x0 + nplanes * m[0] / m[2]
    return tot, cx, cy, var, gx, top.max()


def _fixed_faces(grid, fill):
    nx, ny, nz = grid.n
    out = []
    for a in range(3):
        for side in range(2):
            blk = np.zeros((grid.na, grid.face[a]))
            for k in range(grid.na):
                if a == 0:
                    i = -1 if side == 0 else nx
                    vals = [fill(a, side, k, i, jj, kk) for kk in range(nz) for jj in range(ny)]
                elif a == 1:
                    j = -1 if side == 0 else ny
                    vals = [fill(a, side, k, ii, j, kk) for kk in range(nz) for ii in range(nx)]
                else:
                    kz = -1 if side == 0 else nz
                    vals = [fill(a, side, k, ii, jj, kz) for jj in range(ny) for ii in range(nx)]
                blk[k] = vals
            out.append(blk.ravel())
    return np.concatenate(out)


def test_searchlight_spreads_less_than_linear():
    tot_l, cx_l, cy_l, var_l, gx, pk_l = _beam("linear")
    tot_q, cx_q, cy_q, var_q, _, pk_q = _beam("quadratic")
    # linear interpolation conserves the beam and its centroid exactly (a random walk)
    assert abs(tot_l - 1.0) < 1e-12 and abs(cx_l - gx) < 1e-9 and abs(cy_l - gx) < 1e-9
    # the clamped quadratic keeps the beam about half as wide and several times
    # brighter; clamping its undershoots is not conservative (the beam's sum grows,
    # about 2.4x after 24 planes, and its centroid trails the ray by about a cell)
    assert var_q < 0.6 * var_l, (var_q, var_l)
    assert pk_q > 3 * pk_l, (pk_q, pk_l)
    assert abs(cx_q - gx) < 1.5 and abs(cy_q - gx) < 1.5, (cx_q, gx)


@pytest.mark.parametrize("n_mu", [4, 8])
def test_lambda_star_of_uniform_medium(n_mu):
    """Uniform chi and S: every ray has dtau- = dtau+ = chi s and an unclamped
    control point with dSc/dS0 = 1, so Lambda* = sum_k w_k (b + c)
    = sum_k w_k (1 - e^-t - a), a from direct quadrature."""
    chi0 = 0.7
    g = O.Grid(5, 4, 6, n_mu, (P, P, P), (P, P, P), dx=1.0, dy=1.2, dz=0.9)
    r = O.formal_solution(g, np.full(g.shape, chi0), np.ones(g.shape), np.ones(g.shape),
                          interp="quadratic")
    want = 0.0
    for k in range(g.na):
        m = g.mu[k]
        s = min(g.d[a] / abs(m[a]) for a in range(3))
        t = chi0 * s
        a = quad(lambda x: (x / t) ** 2 * math.exp(-x), 0, t, epsabs=0, epsrel=1e-13)[0]
        want += g.w[k] * (-math.expm1(-t) - a)
    np.testing.assert_allclose(r["lstar"], want, rtol=1e-12)


def test_lambda_star_is_the_limited_local_derivative():
    """Lambda*_ii = b + c dSc/dS0 with dSc/dS0 limited to [0, 1].  In a thick
    z-stratified medium (chi s >= 30 per segment) S_i reaches I_i through other
    cells only via exp(-dtau-) ~ 1e-13, so a finite difference of a z-crossing
    ray's I_i in S_i is the unlimited local derivative b + c dSc/dS0; with b, c
    from the segment's dtau- = (chi_{z-1} + chi_z) s / 2 that gives dSc/dS0, and
    Lambda* must be b + c min(1, max(0, dSc/dS0))."""
    nz = 8
    g = O.Grid(5, 5, nz, 6, (P, P, P), (P, P, P))
    rng = np.random.default_rng(8)
    chi_z = rng.uniform(30.0, 60.0, nz)
    chi = np.broadcast_to(chi_z[:, None, None], g.shape).copy()
    S = 1.0 + 0.1 * rng.uniform(size=g.shape)
    h = 1e-7
    checked = 0
    for k in range(g.na):
        m = g.mu[k]
        if abs(m[2]) < max(abs(m[0]), abs(m[1])):
            continue
        g1 = _one_ray(g, k)
        base = O.formal_solution(g1, chi, S, S, interp="quadratic")
        s = 1.0 / abs(m[2])
        for c in ((2, 3, 1), (4, 1, 4), (5, 2, 2)):
            zu = (c[0] - (1 if m[2] > 0 else -1)) % nz
            hm = 0.5 * (chi_z[zu] + chi_z[c[0]]) * s
            _, b, cc = O.bezier_weights(hm)
            S2 = S.copy()
            S2[c] += h
            J2 = O.formal_solution(g1, chi, S2, S, G_prev=O.init_ghosts(g1, S), interp="quadratic")["J"]
            d = (J2[c] - base["J"][c]) / h
            dsc = (d - b) / cc
            np.testing.assert_allclose(base["lstar"][c], b + cc * min(1.0, max(0.0, dsc)), rtol=2e-6)
            checked += 1
    assert checked >= 12


def test_quadratic_ali_reaches_a_stationary_fixed_point():
    from paper_1201_2222_gb300.workloads import stratified_atmosphere
    p = stratified_atmosphere(12, nxy=6)
    g = O.Grid.from_problem(p)
    res = O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=1e-10, max_iter=5000,
                      interp="quadratic", moments=False)
    assert res["converged"] and res["iters"] > 20
    lin = O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=1e-10, max_iter=5000, moments=False)
    # the two schemes solve different discrete problems: close, not equal
    d = np.max(np.abs(res["S"] / lin["S"] - 1))
    assert 1e-6 < d < 0.2, d
