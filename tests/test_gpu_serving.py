"""The request server (rt_server_*): queued solves of mixed sizes, frequency counts
and angle sets on several worker streams at once give, each, the same result as
the same solve run alone; admission keeps the running footprint under the budget;
errors and waits are reported per request."""
import time

import numpy as np
import pytest

from paper_1201_2222_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2222_gb300 import build, rt as _rt
    build.build()
    return _rt


def _mix():
    base = W.serving_stream(10, seed=11, rate=1.0)
    reqs = []
    for i, d in enumerate(base):
        shape = (40, 40, 1) if (d["shape"][2] == 1 or i == 5) else ((12, 12, 12), (16, 16, 16), (20, 16, 12))[i % 3]
        d = dict(d, shape=shape, eps=max(d["eps"], 0.05))
        prec = "mixed" if i % 3 else "fp64"
        interp = "quadratic" if i % 4 == 3 else "linear"
        scheme = "gauss_seidel" if i % 4 == 2 else "jacobi"
        # the second-order mixed path sweeps S itself: float32 rounding limits tol
        tol = 1e-5 if interp == "quadratic" else 1e-6
        reqs.append((W.build_request(d, tol=tol), prec, interp, scheme))
    return reqs


def _alone(rt, p, prec, interp, scheme):
    g = rt.Grid.from_problem(p, prec=prec)
    g.set_interpolation(interp)
    g.set_iteration(scheme)
    g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
    iters, resid, st = g.ali_solve(tol=p.tol, max_iter=3000)
    m = g.moments()
    return iters, m["J"], g.get_S(), m["Q"]


def test_results_in_the_mix_equal_results_alone(rt):
    reqs = _mix()
    srv = rt.Server(workers=3)
    ids = [srv.submit(p, prec=prec, interp=interp, iteration=scheme, max_iter=3000)
           for p, prec, interp, scheme in reqs]
    seen_running = 0
    while True:
        infos = [srv.poll(i) for i in ids]
        seen_running = max(seen_running, sum(x["state"] == rt.REQ_RUNNING for x in infos))
        if all(x["state"] == rt.REQ_DONE for x in infos):
            break
        time.sleep(0.002)
    assert seen_running >= 2           # solves overlapped
    for rid, (p, prec, interp, scheme) in zip(ids, reqs):
        info = srv.wait(rid, timeout=60)
        assert info["status"] == rt.RT_OK and info["resid"] <= p.tol
        J, S, Q, st = srv.fetch(rid)
        iters, J1, S1, Q1 = _alone(rt, p, prec, interp, scheme)
        assert info["iters"] == iters
        np.testing.assert_array_equal(J, J1)
        np.testing.assert_array_equal(S, S1)
        np.testing.assert_array_equal(Q, Q1)
    srv.close()


def test_shared_launches_equal_results_alone(rt):
    # shared mode: the Jacobi requests run in lock-step on the scheduler, their
    # sweeps merged; each equals the same solve alone with the server's cluster
    # size (the Gauss-Seidel and second-order requests run on workers as before)
    reqs = _mix()
    srv = rt.Server(workers=3, shared_cluster=2)
    ids = [srv.submit(p, prec=prec, interp=interp, iteration=scheme, max_iter=3000)
           for p, prec, interp, scheme in reqs]
    for rid, (p, prec, interp, scheme) in zip(ids, reqs):
        info = srv.wait(rid, timeout=120)
        assert info["status"] == rt.RT_OK and info["resid"] <= p.tol
        J, S, Q, st = srv.fetch(rid)
        g = rt.Grid.from_problem(p, prec=prec)
        g.set_interpolation(interp)
        g.set_iteration(scheme)
        if interp == "linear" and scheme == "jacobi":
            try:
                g.set_sweep_config(0, 2, 0, 3)
            except rt.RTError:
                g.set_sweep_config(0, 0, 0, 0)
        g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
        iters, resid, st1 = g.ali_solve(tol=p.tol, max_iter=3000)
        m = g.moments()
        assert info["iters"] == iters
        np.testing.assert_array_equal(J, m["J"])
        np.testing.assert_array_equal(S, g.get_S())
        np.testing.assert_array_equal(Q, m["Q"])
        g.close()
    assert srv.shared_launches() > 0
    srv.close()


def test_admission_by_footprint(rt):
    reqs = _mix()[:5]
    fps = [rt.grid_footprint(p, prec) for p, prec, _, _ in reqs]
    assert all(f > 8 * 11 * p.chi.size for f, (p, _, _, _) in zip(fps, reqs))
    # a budget below every request: they run one at a time (each alone when nothing else runs)
    srv = rt.Server(workers=3, device_bytes=1)
    ids = [srv.submit(p, prec=prec, interp=interp, iteration=scheme, max_iter=3000)
           for p, prec, interp, scheme in reqs]
    while True:
        infos = [srv.poll(i) for i in ids]
        assert sum(x["state"] == rt.REQ_RUNNING for x in infos) <= 1
        if all(x["state"] == rt.REQ_DONE for x in infos):
            break
        time.sleep(0.001)
    assert all(srv.fetch(i)[3] == rt.RT_OK for i in ids)
    srv.close()


def test_errors_and_timeouts(rt):
    srv = rt.Server(workers=1)
    good = W.build_request(dict(shape=(24, 24, 24), nf=4, n_mu=8, eps=0.01, seed=5), tol=1e-9)
    bad = W.build_request(dict(shape=(8, 8, 8), nf=1, n_mu=4, eps=0.5, seed=6))
    bad.eps[0, 0, 0, 0] = 0.0       # eps must be > 0: rejected when the solve sets the medium
    r1 = srv.submit(good, prec="mixed", max_iter=5000)
    r2 = srv.submit(bad, prec="mixed")
    with pytest.raises(rt.RTError) as e:
        srv.wait(r2, timeout=1e-3)    # still queued behind r1 on the only worker
    assert e.value.status == rt.RT_ERR_TIMEOUT
    assert srv.wait(r2, timeout=120)["status"] == rt.RT_ERR_ARG
    with pytest.raises(rt.RTError):
        srv.fetch(r2)
    assert srv.wait(r1, timeout=120)["status"] == rt.RT_OK
    srv.fetch(r1)
    with pytest.raises(rt.RTError):
        srv.poll(r1)                  # forgotten after fetch
    srv.close()
