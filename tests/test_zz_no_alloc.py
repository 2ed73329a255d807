"""The allocation-free formal solution against the regular entry point (GPU).

rt_formal_solve_noalloc exists for callers that cannot allocate device memory
(for example a host framework that keeps the device memory in its own pool, or a
time-critical loop that must not pay for an allocation): it takes all of its
working memory from one static device array of the library.  Here it must give
the same J as rt_create_grid + rt_set_opacity_source + rt_formal_solve, on two
calls in a row that reuse that array with different problems, within the
tolerances the parity tests use (1e-10 for FP64, 1e-5 for the float32 sweep).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_regular_formal_solution(rt, prec):
    problems = [W.random_box(20, 17, 12, seed=41, n_mu=4, bc_lo=(P, P, T), bc_hi=(P, P, V)),
                W.random_box(9, 14, 11, seed=42, n_mu=6, nf=2, bc_lo=(V, P, T), bc_hi=(T, P, V))]
    tol = 1e-10 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(7)
    for p in problems:           # two calls in a row through the shared scratch array
        S = rng.uniform(0.3, 2.0, p.chi.shape)
        g = rt.Grid.from_problem(p, prec=prec)
        g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
        J_ref = g.formal_solve(S)
        J = torch.full(p.chi.shape, float("nan"), dtype=torch.float64, device="cuda")
        rt.formal_solve_noalloc(p.nx, p.ny, p.nz, _dev(p.chi), _dev(S), _dev(p.B), J, n_mu=p.n_mu,
                                nfreq=p.nf, bc_lo=p.bc_lo, bc_hi=p.bc_hi, prec=prec)
        assert _rel(J.cpu().numpy(), J_ref) < tol


def test_noalloc_allocates_no_device_memory(rt):
    # after a first call (which looks up the scratch array's address), further
    # calls on other problems leave the device's free memory as it was
    p1 = W.random_box(16, 12, 10, seed=43, n_mu=4, bc_lo=(P, P, T), bc_hi=(P, P, V))
    p2 = W.random_box(12, 20, 9, seed=44, n_mu=8, nf=2, bc_lo=(V, P, T), bc_hi=(T, P, V))
    args = []
    for p in (p1, p2):
        args.append((p, _dev(p.chi), _dev(p.B), _dev(p.B),
                     torch.empty(p.chi.shape, dtype=torch.float64, device="cuda")))
    def call(p, chi, S, B, J):
        rt.formal_solve_noalloc(p.nx, p.ny, p.nz, chi, S, B, J, n_mu=p.n_mu, nfreq=p.nf,
                                bc_lo=p.bc_lo, bc_hi=p.bc_hi, prec="mixed")
    call(*args[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for a in (args[1], args[0], args[1]):
        call(*a)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0


def test_noalloc_rejects_oversize_and_fixed_faces(rt):
    big = 512
    with pytest.raises(rt.RTError) as e:
        rt.formal_solve_noalloc(big, big, big, None, None, None, None, n_mu=8)
    assert e.value.status == rt.RT_ERR_ARG and "scratch" in str(e.value)
    with pytest.raises(rt.RTError) as e:
        rt.formal_solve_noalloc(8, 8, 8, None, None, None, None, bc_lo=(P, P, 3), bc_hi=(P, P, V))
    assert e.value.status == rt.RT_ERR_ARG
