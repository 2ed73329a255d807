"""Lock-step solves (rt_ali_solve_many): several grids' Jacobi solves advanced
together, the sweeps of grids with the same precision and cluster size merged
into shared launches.  Each grid's iterates are the same as in its own
rt_ali_solve (same kernels on the same data, host checks after the same
iterations), so every result must be equal bit for bit, iteration counts
included, while grids of other plans (the one-cell-per-thread FP64 sweep) run
their own launches in the same steps."""
import numpy as np
import pytest

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


def _problems():
    return [
        (W.stratified_atmosphere(16, nxy=8), "mixed", (0, 2, 0, 3)),
        (W.turbulent_box(24, n_mu=8), "mixed", (0, 2, 0, 3)),
        (W.multifrequency_atmosphere(16, nf=4), "mixed", (0, 2, 0, 3)),
        (W.random_box(12, 8, 10, seed=71, n_mu=6, bc_lo=(T, P, V), bc_hi=(V, P, T)), "mixed", (0, 2, 0, 3)),
        (W.stratified_atmosphere(12, nxy=4, eps=1e-3), "mixed", (0, 2, 0, 3)),
        (W.random_box(8, 8, 8, seed=72, n_mu=4), "fp64", (0, 2, 0, 3)),      # FP64, pipelined: the two
        (W.random_box(8, 12, 6, seed=75, n_mu=6), "fp64", (0, 2, 0, 3)),     # share their own launches
        (W.random_box(9, 7, 6, seed=73, n_mu=4), "fp64", (0, 0, 0, 0)),      # one cell per thread: own launch
        (W.stratified_atmosphere(20, nxy=8), "mixed", (0, 4, 0, 3)),        # another cluster size: alone
    ]


def _grid(rt, p, prec, cfg):
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_sweep_config(*cfg)
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    return g


def test_many_equal_each_alone_bit_for_bit(rt):
    probs = _problems()
    alone = []
    for p, prec, cfg in probs:
        g = _grid(rt, p, prec, cfg)
        it, res, st = g.ali_solve(tol=p.tol, max_iter=5000)
        m = g.moments(want=("J", "Q"))
        alone.append((it, g.get_S(), m["J"], m["Q"], g.stats()["fp64_anchors"]))
        g.close()
    grids = [_grid(rt, p, prec, cfg) for p, prec, cfg in probs]
    out = rt.ali_solve_many(grids, tol=1e-6, max_iter=5000)
    for k, ((p, prec, cfg), g, (it, res, st), a) in enumerate(zip(probs, grids, out, alone)):
        assert st == rt.RT_OK and res <= p.tol, (k, st, res)
        assert it == a[0], (k, it, a[0])
        m = g.moments(want=("J", "Q"))
        np.testing.assert_array_equal(g.get_S(), a[1], err_msg=str(k))
        np.testing.assert_array_equal(m["J"], a[2], err_msg=str(k))
        np.testing.assert_array_equal(m["Q"], a[3], err_msg=str(k))
        stt = g.stats()
        assert stt["fp64_anchors"] == a[4]
        if cfg[3] == 3 and cfg[1] == 2:
            assert stt["shared_launches"] > 0, k        # swept together with other grids
        else:
            assert stt["shared_launches"] == 0, k       # no partner of its precision and plan
    for g in grids:
        g.close()


def test_out_of_iterations(rt):
    # every grid stops after max_iter formal solutions with RT_ERR_NOT_CONVERGED,
    # at the same S as its own rt_ali_solve
    probs = _problems()[:3]
    alone = []
    for p, prec, cfg in probs:
        g = _grid(rt, p, prec, cfg)
        it, res, st = g.ali_solve(tol=1e-6, max_iter=7, raise_on_fail=False)
        assert st == rt.RT_ERR_NOT_CONVERGED and it == 7
        alone.append(g.get_S())
        g.close()
    grids = [_grid(rt, p, prec, cfg) for p, prec, cfg in probs]
    out = rt.ali_solve_many(grids, tol=1e-6, max_iter=7, raise_on_fail=False)
    for g, (it, res, st), S in zip(grids, out, alone):
        assert st == rt.RT_ERR_NOT_CONVERGED and it == 7
        np.testing.assert_array_equal(g.get_S(), S)
        g.close()


def test_rejects_what_it_cannot_step(rt):
    p = W.random_box(8, 8, 8, seed=74, n_mu=4)
    a = _grid(rt, p, "mixed", (0, 2, 0, 3))
    b = _grid(rt, p, "mixed", (0, 0, 0, 0))
    b.set_iteration("gauss_seidel")
    with pytest.raises(rt.RTError) as e:
        rt.ali_solve_many([a, b])
    assert e.value.status == rt.RT_ERR_STATE
    c = rt.Grid.from_problem(p, prec="mixed")           # no medium
    with pytest.raises(rt.RTError) as e:
        rt.ali_solve_many([a, c])
    assert e.value.status == rt.RT_ERR_STATE
    assert rt.ali_solve_many([]) == []
    for g in (a, b, c):
        g.close()
