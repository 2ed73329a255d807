"""Grid life cycle on the mixed path: a medium set again on the same grid (LTE
media, which need no internal FP64 grid, between media that do) leaves the grid
solving as a fresh one, and destroying grids with internal FP64 grids (the one
of the FP64 iterations, the one of ill-conditioned bins) returns their device
memory."""
import numpy as np
import pytest

from paper_1201_2222_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = 0


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2222_gb300 import build, rt as _rt
    build.build()
    return _rt


def _solve(rt, g, p):
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    it, res, st = g.ali_solve(tol=1e-6, max_iter=5000)
    assert st == rt.RT_OK
    return it, g.get_S(), g.moments(want=("J",))["J"]


def test_media_set_again_solve_as_on_a_fresh_grid(rt):
    lte = W.random_box(8, 8, 8, seed=81, n_mu=4, eps_range=(1.0, 1.0), bc_lo=(P, P, P), bc_hi=(P, P, P))
    scat = W.random_box(8, 8, 8, seed=82, n_mu=4, eps_range=(1e-5, 1e-2), bc_lo=(P, P, P), bc_hi=(P, P, P))
    g = rt.Grid.from_problem(scat, prec="mixed")
    seq = [lte, lte, scat, lte, scat, scat]
    for p in seq:
        it, S, J = _solve(rt, g, p)
        f = rt.Grid.from_problem(p, prec="mixed")
        it1, S1, J1 = _solve(rt, f, p)
        f.close()
        assert it == it1
        np.testing.assert_array_equal(S, S1)
        np.testing.assert_array_equal(J, J1)
        if p is lte:
            np.testing.assert_array_equal(S, p.B)         # LTE: S = B
    g.close()


def test_destroy_returns_internal_grids_memory(rt):
    # 4 bins, eps down to 1e-6 in thick cells: FP64 bins and the FP64-iteration grid
    p = W.multifrequency_atmosphere(16, nf=4)
    g = rt.Grid.from_problem(p, prec="mixed")
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    assert g.sweep_plan()["fp64_bins"] > 0
    g.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        g = rt.Grid.from_problem(p, prec="mixed")
        g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
        g.ali_solve(tol=1e-6, max_iter=5000, raise_on_fail=False)
        g.close()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
