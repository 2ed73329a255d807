"""GPU parity of the second-order formal solution (monotonic quadratic face
interpolation, Bezier-controlled segment integration; Sec. 3.3) against the
oracle, through the C ABI.

Gates: the FP64 path to 1e-10 relative (J, Lambda*); the float32 path to 1e-4
relative plus 1e-5 of the frequency bin's largest value (the clamps compare
float32 values, so a near-tie can switch a clamp that FP64 leaves alone).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1201_2222_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, V, T = 0, 1, 2


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2222_gb300 import build, rt as _rt
    build.build()
    return _rt


def _binwise_ok(x, ref, rtol, floor):
    binmax = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1).reshape((-1,) + (1,) * (ref.ndim - 1))
    return bool(np.all(np.abs(x - ref) <= rtol * np.abs(ref) + floor * binmax))


CASES = [
    lambda: W.random_box(9, 8, 7, seed=1, n_mu=4, nf=2, bc_lo=(T, P, V), bc_hi=(V, P, T)),
    lambda: dataclasses.replace(W.random_box(6, 10, 5, seed=2, n_mu=6, bc_lo=(P, V, T), bc_hi=(P, T, V)),
                                dx=0.7, dy=1.3, dz=1.0),
    lambda: W.random_box(12, 12, 12, seed=3, n_mu=8),
    lambda: W.stratified_atmosphere(12, nxy=8),
    lambda: W.random_box(7, 5, 1, seed=4, n_mu=4, bc_lo=(P, V, P), bc_hi=(P, T, P)),   # 2D
]


def _oracle_fs(p):
    og = O.Grid.from_problem(p)
    J = np.empty_like(p.chi)
    L = np.empty_like(p.chi)
    for f in range(p.nf):
        r = O.formal_solution(og, p.chi[f], p.B[f], p.B[f], interp="quadratic", nthreads=O.max_threads())
        J[f], L[f] = r["J"], r["lstar"]
    return J, L


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_quadratic_formal_solution(rt, prec, case):
    p = CASES[case]()
    J_ref, L_ref = _oracle_fs(p)
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_interpolation("quadratic")
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    J, L = g.formal_solve(p.B, want_lstar=True)
    if prec == "fp64":
        np.testing.assert_allclose(J, J_ref, rtol=1e-10)
        np.testing.assert_allclose(L, L_ref, rtol=1e-10, atol=1e-14)
    else:
        assert _binwise_ok(J, J_ref, 1e-4, 1e-5)
        assert np.max(np.abs(L - L_ref)) < 1e-4
    # and not the linear result
    J_lin = O.formal_solution(O.Grid.from_problem(p), p.chi[0], p.B[0], p.B[0])["J"]
    assert np.max(np.abs(J[0] - J_lin) / np.abs(J_lin)) > 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["random", "turbulent", "stratified"])
def test_quadratic_ali_solve(rt, prec, which):
    p = {"random": lambda: W.random_box(8, 7, 6, seed=3, n_mu=4, nf=2, bc_lo=(T, P, V), bc_hi=(V, P, T)),
         "turbulent": lambda: W.turbulent_box(12, n_mu=4),
         "stratified": lambda: W.stratified_atmosphere(12, nxy=6)}[which]()
    tol = 1e-8 if prec == "fp64" else 1e-4
    og, ref = O.solve_problem(p, tol=tol, max_iter=5000, interp="quadratic", nthreads=O.max_threads())
    assert ref["converged"]
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_interpolation(rt.INTERP_QUADRATIC)
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    iters, resid, st = g.ali_solve(tol=tol, max_iter=5000)
    assert st == rt.RT_OK and resid <= tol
    assert abs(iters - ref["iters"]) <= 1, (iters, ref["iters"])
    S = g.get_S()
    m = g.moments()
    if prec == "fp64":
        np.testing.assert_allclose(S, ref["S"], rtol=1e-7)
        np.testing.assert_allclose(m["J"], ref["J"], rtol=1e-7)
    else:
        # both stop within tol of the same fixed point
        assert _binwise_ok(S, ref["S"], 2e-3, 1e-5)
        assert _binwise_ok(m["J"], ref["J"], 2e-3, 1e-5)


def test_interpolation_switch_and_validation(rt):
    p = W.random_box(6, 5, 4, seed=9, n_mu=4)
    lin = rt.Grid.from_problem(p, prec="fp64")
    lin.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    J_lin = lin.formal_solve(p.B)
    g = rt.Grid.from_problem(p, prec="fp64")
    g.set_interpolation("quadratic")
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    J_q = g.formal_solve(p.B)
    g.set_interpolation("linear")
    np.testing.assert_array_equal(g.formal_solve(p.B), J_lin)
    assert np.max(np.abs(J_q - J_lin)) > 0
    with pytest.raises(rt.RTError):
        g.set_interpolation(3)
