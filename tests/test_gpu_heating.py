"""GPU parity of the heating-rate forms (Sec. 4) against the oracle.

Q^dif = -4 pi sum w div H differences neighbouring values of H, so its error
gate has an absolute part on the scale 4 pi sum_nu w_nu max|J_nu| sum_a 1/h_a
(|H| <= J) besides the relative one; the integral part keeps the gate of the
converged-solve tests (|dQ| <= rtol |Q| + atol 4 pi chi_abs B, with rtol = 1e-3
and atol = 1e-6 on the mixed path).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1201_2222_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, V, T = 0, 1, 2
GATE = {"fp64": (1e-8, 1e-10), "mixed": (1e-3, 1e-6)}


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2222_gb300 import build, rt as _rt
    build.build()
    return _rt


def _problem():
    # thin and thick cells (chi dx from 5e-3 to 15), non-cubic spacing, all boundary kinds
    p = W.random_box(9, 8, 7, seed=11, n_mu=4, nf=2, bc_lo=(T, P, V), bc_hi=(V, P, T),
                     chi_range=(1e-2, 10.0), eps_range=(3e-2, 1.0))
    return dataclasses.replace(p, dx=0.5, dy=1.5, dz=1.0)


@pytest.fixture(scope="module")
def reference():
    p = _problem()
    og, ref = O.solve_problem(p, tol=1e-10, max_iter=5000)
    return p, og, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("form", ["integral", "differential", "switch"])
def test_heating_form_matches_oracle(rt, reference, prec, form):
    p, og, ref = reference
    if form == "integral":
        q_ref = O.heating_rate(p.chi, p.eps, ref["J"], p.B, p.freq_w)
    elif form == "differential":
        q_ref = O.heating_rate_dif(og, ref["H"], p.freq_w)
    else:
        q_ref = O.heating_rate_switch(og, p.chi, p.eps, ref["J"], p.B, ref["H"], p.freq_w)
    thin = p.chi * O.cell_width(og) <= 1.0
    assert 0.2 < thin.mean() < 0.8   # both forms are exercised by the switch
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    iters, resid, st = g.ali_solve(tol=1e-10, max_iter=5000)
    assert st == rt.RT_OK
    g.set_heating_form(form)
    q = g.moments()["Q"]
    rtol, atol = GATE[prec]
    fw = p.freq_w[:, None, None, None]
    emission = 4 * math.pi * np.sum(fw * p.eps * p.chi * p.B, axis=0)
    inv_h = sum(1.0 / h for h, n in zip((p.dx, p.dy, p.dz), (p.nx, p.ny, p.nz)) if n > 1)
    dif_scale = 4 * math.pi * float(np.sum(p.freq_w * np.abs(ref["J"]).reshape(p.nf, -1).max(axis=1))) * inv_h
    bound = rtol * np.abs(q_ref) + atol * (emission + dif_scale)
    assert np.all(np.abs(q - q_ref) <= bound), float(np.max(np.abs(q - q_ref) / bound))


def test_heating_form_default_and_validation(rt):
    p = W.random_box(6, 5, 4, seed=2, n_mu=4)
    g = rt.Grid.from_problem(p, prec="fp64")
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    g.ali_solve(tol=1e-8, max_iter=2000)
    q0 = g.moments()["Q"]
    g.set_heating_form("integral")
    np.testing.assert_array_equal(g.moments()["Q"], q0)
    with pytest.raises(rt.RTError):
        g.set_heating_form(3)
