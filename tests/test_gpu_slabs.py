"""GPU slab decomposition (Sec. 3.5): z slabs as FP64 grids of the library with
subdomain z faces, driven by paper_1201_2222_gb300.slabs, against the oracle's
slab solve of the same decomposition (same ghost-layer rules and lag): the
same iteration count and the same S and J to FP64 round-off.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1201_2222_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, V, T, F = 0, 1, 2, 3


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2222_gb300 import build, rt as _rt
    build.build()
    return _rt


CASES = {
    "atmosphere_3": lambda: (W.stratified_atmosphere(12, nxy=6), 3),
    "periodic_2": lambda: (W.random_box(6, 5, 8, seed=61, n_mu=6, nf=2, bc_lo=(P, P, P), bc_hi=(P, P, P)), 2),
    "bounded_sides_4": lambda: (W.random_box(5, 6, 9, seed=62, n_mu=4, bc_lo=(T, V, T), bc_hi=(V, T, V)), 4),
    "one_slab_periodic": lambda: (W.random_box(5, 4, 6, seed=63, n_mu=4, bc_lo=(P, P, P), bc_hi=(P, P, P)), 1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_gpu_slabs_match_the_oracle_slab_solve(rt, case):
    from paper_1201_2222_gb300 import slabs as SL
    p, nslab = CASES[case]()
    tol = 1e-9
    got = SL.slab_ali_solve(p, nslab, tol=tol, max_iter=5000)
    ref = O.slab_ali_solve(O.Grid.from_problem(p), p.chi, p.eps, p.B, nslab, tol=tol, max_iter=5000,
                           nthreads=O.max_threads())
    assert got["converged"] and ref["converged"]
    assert got["iters"] == ref["iters"], (got["iters"], ref["iters"])
    np.testing.assert_allclose(got["S"], ref["S"], rtol=1e-10)
    np.testing.assert_allclose(got["J"], ref["J"], rtol=1e-10)


def test_slabs_converge_to_the_single_domain(rt):
    # the paper: decomposed and single-domain J agree to about delta_c J
    from paper_1201_2222_gb300 import slabs as SL
    p = W.stratified_atmosphere(16, nxy=8)
    tol = 1e-7
    got = SL.slab_ali_solve(p, 4, tol=tol, max_iter=5000)
    g = rt.Grid.from_problem(p, prec="fp64")
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    it1, _, _ = g.ali_solve(tol=tol, max_iter=5000)
    assert got["iters"] >= it1
    np.testing.assert_allclose(got["S"], g.get_S(), rtol=20 * tol)


def test_subdomain_face_validation(rt):
    p = W.random_box(4, 4, 6, seed=3, n_mu=4)
    with pytest.raises(rt.RTError):      # mixed precision
        rt.Grid(4, 4, 6, bc_lo=(P, P, rt.EXTERNAL), bc_hi=(P, P, V), prec="mixed")
    with pytest.raises(rt.RTError):      # with a fixed x face
        rt.Grid(4, 4, 6, bc_lo=(F, P, rt.EXTERNAL), bc_hi=(F, P, V), prec="fp64")
    with pytest.raises(rt.RTError):      # on an x face
        rt.Grid(4, 4, 6, bc_lo=(rt.EXTERNAL, P, T), bc_hi=(V, P, V), prec="fp64")
    g = rt.Grid(4, 4, 6, bc_lo=(P, P, T), bc_hi=(P, P, rt.EXTERNAL), prec="fp64")
    g.set_opacity_source(p.chi, p.eps, p.B)
    with pytest.raises(rt.RTError) as e:  # the low face is not a subdomain face
        g.set_external_face(0, S=np.ones((1, 4, 4)))
    assert e.value.status == rt.RT_ERR_STATE
    with pytest.raises(rt.RTError):
        g.set_sweep_config(variant=3)
    with pytest.raises(rt.RTError):      # stepping before rt_ali_begin
        g.ali_iterate(1)
