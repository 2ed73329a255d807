"""Pins of the oracle's Gauss-Seidel ALI (Sec. 3.4, plane-wavefront form).

* Fixed point: Gauss-Seidel and Jacobi solve the same discretised problem, so
  they stop at the same S (within the stopping tolerance), and Gauss-Seidel
  needs fewer iterations on a scattering atmosphere (the paper's comparison of
  the two schemes; the ratio approaches 2 when every downward ray is swept in
  reverse, n_mu = 2).
* First plane: the top plane is updated before any S has changed, so its new S
  is the Jacobi update of a formal solution of the old S.
* Reverse rays: the J the reverse rays contribute at plane k is that of a formal
  solution of the reverse rays alone through an S holding the new values above
  plane k and the old ones elsewhere (brute force: one formal solution per
  plane).
* Correction: in a uniform medium on one periodic column (every upwind vertex
  on the plane above is that plane's one cell), the first-order correction at
  plane k is dS(k+1) times the closed form
  sum over downward forward rays of w Psi-(chi s) (s |mu_z| / dz), the share of
  the upwind point's interpolation weight on the plane above.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1201_2222_gb300 import workloads as W

P, V, T = O.PERIODIC, O.VACUUM, O.THERMAL


def _solve(p, method, tol=1e-6, **kw):
    g = O.Grid.from_problem(p)
    return g, O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=tol, max_iter=5000,
                          moments=False, method=method, **kw)


@pytest.mark.parametrize("n_mu,min_ratio", [(2, 1.5), (4, 1.2), (8, 1.2)])
def test_same_fixed_point_in_fewer_iterations(n_mu, min_ratio):
    p = W.stratified_atmosphere(16, n_mu=n_mu)
    _, rj = _solve(p, "jacobi")
    _, rg = _solve(p, "gauss_seidel")
    assert rj["converged"] and rg["converged"]
    assert rj["iters"] >= min_ratio * rg["iters"], (rj["iters"], rg["iters"])
    # both stop within tol of the fixed point; the distance to it is bounded by
    # tol over the iteration's convergence factor
    np.testing.assert_allclose(rg["S"], rj["S"], rtol=2e-5)


def test_fixed_point_matches_a_tight_jacobi_solve_on_a_random_periodic_box():
    p = W.random_box(8, 8, 8, seed=4, n_mu=6, bc_lo=(P, P, P), bc_hi=(P, P, P))
    _, rj = _solve(p, "jacobi", tol=1e-12)
    _, rg = _solve(p, "gauss_seidel", tol=1e-12)
    np.testing.assert_allclose(rg["S"], rj["S"], rtol=1e-10)
    assert rg["iters"] < rj["iters"]


def test_two_d_fixed_point():
    p = W.random_box(12, 10, 1, seed=5, n_mu=4, bc_lo=(P, T, P), bc_hi=(P, V, P))
    _, rj = _solve(p, "jacobi", tol=1e-12)
    _, rg = _solve(p, "gauss_seidel", tol=1e-12)
    np.testing.assert_allclose(rg["S"], rj["S"], rtol=1e-10)


def test_reverse_rays():
    g = O.Grid(4, 4, 4, n_mu=8)
    rev = O.gs_reverse_rays(g)
    # downward rays whose largest direction cosine is mu_z (ties included):
    # (1,1,4), (1,2,3), (2,1,3), (2,2,2) per octant of the LQ8 set
    dom = np.abs(g.mu[:, 2]) >= np.abs(g.mu[:, :2]).max(axis=1) - 1e-12
    np.testing.assert_array_equal(rev, dom & (g.mu[:, 2] < 0))
    assert rev.sum() == 16
    g2 = O.Grid(4, 4, 1, n_mu=4)
    rev2 = O.gs_reverse_rays(g2)
    dom2 = np.abs(g2.mu[:, 1]) >= np.abs(g2.mu[:, 0]) - 1e-12
    np.testing.assert_array_equal(rev2, dom2 & (g2.mu[:, 1] < 0))


def _one_iteration(g, chi, eps, B, S, G=None):
    """One Gauss-Seidel iteration from S (ghosts G, default the first-iteration
    ones); returns the pieces: forward J, reverse-phase outputs, new S, Lambda*,
    ghosts."""
    if G is None:
        G = O.init_ghosts(g, S)
    lstar = O.formal_solution(g, chi, S, B, G)["lstar"]
    fwd = np.flatnonzero(~O.gs_reverse_rays(g))
    rf = O.formal_solution(g, chi, S, B, G, rays=fwd)
    Sn = np.ascontiguousarray(S, dtype=np.float64).reshape(-1).copy()
    Gn = G.copy()
    out = O.gs_reverse(g, chi, eps, B, lstar, rf["J"], Sn, G, Gn)
    return rf["J"], out, Sn.reshape(g.shape), lstar, G


@pytest.mark.parametrize("bc", ["atmosphere", "periodic"])
def test_first_plane_is_the_jacobi_update(bc):
    p = (W.stratified_atmosphere(8, n_mu=6) if bc == "atmosphere"
         else W.random_box(6, 7, 8, seed=2, n_mu=6, bc_lo=(P, P, P), bc_hi=(P, P, P)))
    g = O.Grid.from_problem(p)
    chi, eps, B = p.chi[0], p.eps[0], p.B[0]
    S = B * (1.0 + 0.3 * np.sin(np.arange(B.size).reshape(B.shape)))   # not a fixed point
    _, out, Sn, lstar, G = _one_iteration(g, chi, eps, B, S)
    full = O.formal_solution(g, chi, S, B, G)
    dS_jac = ((1 - eps) * full["J"] + eps * B - S) / (1 - (1 - eps) * lstar)
    top = g.n[2] - 1
    np.testing.assert_allclose(Sn[top], (S + dS_jac)[top], rtol=1e-13, atol=0)
    # below the top the freshest J differs from the Jacobi one
    assert np.max(np.abs(Sn[:top] - (S + dS_jac)[:top])) > 1e-6 * np.max(np.abs(S))


@pytest.mark.parametrize("case", ["atmosphere", "periodic", "two_d"])
def test_reverse_rays_see_the_new_s_above(case):
    if case == "atmosphere":
        p = W.stratified_atmosphere(6, n_mu=8, nxy=5)
    elif case == "periodic":
        p = W.random_box(5, 6, 7, seed=8, n_mu=6, bc_lo=(P, P, P), bc_hi=(P, P, P))
    else:
        p = W.random_box(9, 7, 1, seed=9, n_mu=6, bc_lo=(P, T, P), bc_hi=(P, V, P))
    g = O.Grid.from_problem(p)
    chi, eps, B = p.chi[0], p.eps[0], p.B[0]
    rng = np.random.default_rng(3)
    S = B * (0.5 + rng.random(B.shape))
    JF, out, Sn, _, G = _one_iteration(g, chi, eps, B, S)
    rev = np.flatnonzero(O.gs_reverse_rays(g))
    JR_seen = out["J"] - JF - out["C"]
    vax = 1 if g.two_d else 0          # array axis of the reverse axis ([nz][ny][nx])
    nV = g.shape[vax]
    for k in range(nV):
        above = np.zeros(g.shape, dtype=bool)
        sl = [slice(None)] * 3
        sl[vax] = slice(k + 1, None)
        above[tuple(sl)] = True
        S_mix = np.where(above, Sn, S)
        JR = O.formal_solution(g, chi, S_mix, B, G, rays=rev)["J"]
        sl[vax] = k
        np.testing.assert_allclose(JR_seen[tuple(sl)], JR[tuple(sl)], rtol=1e-12,
                                   atol=1e-13 * np.max(np.abs(JR)))


@pytest.mark.parametrize("n_mu", [4, 8])
def test_first_order_correction_closed_form(n_mu):
    # one periodic column: every upwind vertex on the plane above is its one cell
    n, chi0 = 6, 0.7
    g = O.Grid(1, 1, n, n_mu=n_mu, bc_lo=(P, P, T), bc_hi=(P, P, V))
    chi = np.full(g.shape, chi0)
    eps = np.full(g.shape, 0.05)
    B = np.ones(g.shape)
    z = np.arange(n)[:, None, None]
    S = np.broadcast_to(0.2 + 0.1 * z + 0.02 * z ** 2, g.shape).copy()
    _, out, Sn, _, _ = _one_iteration(g, chi, eps, B, S)
    dS = out["dS"]
    assert np.all(np.abs(dS) > 1e-3)
    rev = O.gs_reverse_rays(g)
    coef = 0.0
    for k in range(g.na):
        m = g.mu[k]
        if rev[k] or m[2] >= 0:
            continue
        s = min(g.d[a] / abs(m[a]) for a in range(3))
        tau = chi0 * s
        e0 = 1.0 - math.exp(-tau)
        psi_minus = e0 - (tau - e0) / tau
        coef += g.w[k] * psi_minus * (s * abs(m[2]) / g.d[2])
    assert coef > 0
    C = out["C"]
    np.testing.assert_array_equal(C[n - 1], 0.0)            # first plane: nothing updated yet
    for k in range(n - 1):
        np.testing.assert_allclose(C[k], coef * dS[k + 1, 0, 0], rtol=1e-12)


def test_lte_falls_back_to_the_jacobi_test():
    p = W.uniform_box(6, chi=1.0, eps=1.0, B=2.0, n_mu=4)
    _, rj = _solve(p, "jacobi")
    _, rg = _solve(p, "gauss_seidel")
    assert rg["iters"] == rj["iters"]
    np.testing.assert_array_equal(rg["J"], rj["J"])


def test_rejects_second_order_and_unknown_methods():
    p = W.stratified_atmosphere(4)
    g = O.Grid.from_problem(p)
    with pytest.raises(ValueError):
        O.ali_solve(g, p.chi, p.eps, p.B, method="gauss_seidel", interp="quadratic")
    with pytest.raises(ValueError):
        O.ali_solve(g, p.chi, p.eps, p.B, method="sor")


def test_paper_comparison_setting():
    # the paper's comparison of the two schemes (Sec. 5.1): a scattering
    # atmosphere with eps = 1e-6, nine zones per decade of optical depth, started
    # from LTE; with two-stream rays (every downward ray swept in reverse) the
    # Gauss-Seidel scheme needs close to half the iterations
    p = W.stratified_atmosphere(63, eps=1e-6, n_mu=2, nxy=2)
    g = O.Grid.from_problem(p)
    rj = O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=1e-6, max_iter=20000, moments=False)
    rg = O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=1e-6, max_iter=20000, moments=False,
                     method="gauss_seidel")
    assert rj["converged"] and rg["converged"]
    assert 1.6 <= rj["iters"] / rg["iters"] <= 2.2, (rj["iters"], rg["iters"])
