"""Pins of the oracle's slab decomposition (the paper's domain decomposition,
Sec. 3.5): z slabs solved alone, each with a one-cell ghost layer on its
subdomain faces (the neighbour's chi, S and, lagged one iteration, intensities).

* One slab is the single domain: bit for bit on a bounded z axis (no subdomain
  face), and on a periodic z axis too, where the wrap becomes a subdomain face
  whose lagged intensities are exactly the periodic lagged ghosts.
* Several slabs converge to the single domain's solution within about the
  stopping tolerance (the paper reports converged J within ~delta_c J of the
  undecomposed domain), taking a few more iterations (the lag across slab
  faces).
* Constant chi and S stay exact across the slab faces (I = S everywhere).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1201_2222_gb300 import workloads as W

P = O.PERIODIC


def _single(p, tol):
    g = O.Grid.from_problem(p)
    return g, O.ali_solve(g, p.chi, p.eps, p.B, p.freq_w, tol=tol, max_iter=5000, moments=False)


def test_one_slab_is_the_single_domain_bounded_z():
    p = W.stratified_atmosphere(10, nxy=5)
    g, ref = _single(p, 1e-8)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, 1, tol=1e-8, max_iter=5000)
    assert rs["iters"] == ref["iters"]
    np.testing.assert_array_equal(rs["S"], ref["S"])
    np.testing.assert_array_equal(rs["J"], ref["J"])


def test_one_slab_is_the_single_domain_periodic_z():
    p = W.random_box(6, 5, 7, seed=31, n_mu=6, bc_lo=(P, P, P), bc_hi=(P, P, P))
    g, ref = _single(p, 1e-9)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, 1, tol=1e-9, max_iter=5000)
    assert rs["iters"] == ref["iters"]
    np.testing.assert_array_equal(rs["S"], ref["S"])


@pytest.mark.parametrize("nslab", [2, 3, 4])
def test_slabs_converge_to_the_single_domain(nslab):
    tol = 1e-6
    p = W.stratified_atmosphere(12, nxy=6)
    g, ref = _single(p, tol)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, nslab, tol=tol, max_iter=5000)
    assert rs["converged"]
    assert rs["iters"] >= ref["iters"]
    np.testing.assert_allclose(rs["J"], ref["J"], rtol=5 * tol)
    np.testing.assert_allclose(rs["S"], ref["S"], rtol=5 * tol)


@pytest.mark.parametrize("nslab", [2, 3])
def test_periodic_slabs_converge_to_the_single_domain(nslab):
    tol = 1e-10
    p = W.random_box(6, 5, 9, seed=32, n_mu=4, nf=2, bc_lo=(P, P, P), bc_hi=(P, P, P))
    g, ref = _single(p, tol)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, nslab, tol=tol, max_iter=5000)
    assert rs["converged"]
    np.testing.assert_allclose(rs["S"], ref["S"], rtol=50 * tol)


@pytest.mark.parametrize("nslab", [2, 3])
def test_slabs_with_bounded_side_faces_converge_to_the_single_domain(nslab):
    # vacuum and thermal x and y faces: a ghost vertex past a slab face and past
    # one of them takes that face's rule, as in the undecomposed domain
    tol = 1e-9
    T, V = O.THERMAL, O.VACUUM
    p = W.random_box(5, 6, 9, seed=33, n_mu=4, bc_lo=(T, V, T), bc_hi=(V, T, V))
    g, ref = _single(p, tol)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, nslab, tol=tol, max_iter=5000)
    assert rs["converged"]
    np.testing.assert_allclose(rs["S"], ref["S"], rtol=50 * tol)
    np.testing.assert_allclose(rs["J"], ref["J"], rtol=50 * tol)


def test_slabs_reject_fixed_side_faces():
    p = W.random_box(4, 4, 6, seed=3, n_mu=4, bc_lo=(O.FIXED, P, O.THERMAL), bc_hi=(O.FIXED, P, O.VACUUM))
    g = O.Grid.from_problem(p)
    with pytest.raises(ValueError):
        O.slab_ali_solve(g, p.chi, p.eps, p.B, 2)


def test_constant_fields_stay_exact_across_slab_faces():
    p = W.uniform_box(6, chi=0.7, eps=0.3, B=2.0, n_mu=6)
    g = O.Grid.from_problem(p)
    rs = O.slab_ali_solve(g, p.chi, p.eps, p.B, 3, tol=0.0, max_iter=2)
    np.testing.assert_allclose(rs["J"], 2.0, rtol=1e-14)
    np.testing.assert_allclose(rs["S"], 2.0, rtol=1e-14)


def test_rejects_two_d_and_bad_counts():
    p = W.random_box(5, 4, 1, seed=3, n_mu=4)
    g = O.Grid.from_problem(p)
    with pytest.raises(ValueError):
        O.slab_ali_solve(g, p.chi, p.eps, p.B, 2)
    p3 = W.random_box(4, 4, 3, seed=3, n_mu=4)
    g3 = O.Grid.from_problem(p3)
    with pytest.raises(ValueError):
        O.slab_ali_solve(g3, p3.chi, p3.eps, p3.B, 4)
