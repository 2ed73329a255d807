"""Frequency sharding on the GPU (paper_1201_2222_gb300.freqshard with the
library's solver): the bins of a 16^3 x 8-bin atmosphere solved as two blocks
one after the other on this GPU (as two ranks would on two GPUs), against the
single solve of all bins.  FP64: the block holding the slowest bin is the
single solve's to rounding (a block may get another sweep plan, which sums the
rays' J in another grouping) and the iteration count is its count; mixed:
within the mixed path's gates.  Q is the sum of the blocks' heating rates."""
import math

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_blocks_against_the_single_solve(rt, prec):
    from paper_1201_2222_gb300 import freqshard as FS
    p = W.multifrequency_atmosphere(16, nf=8)
    solve = FS.gpu_solver(prec=prec)
    full = solve(p)
    b = FS.bin_blocks(p.nf, 2)
    parts = [solve(FS.sub_problem(p, b[r], b[r + 1])) for r in range(2)]
    iters = max(x["iters"] for x in parts)
    Q = parts[0]["Q"] + parts[1]["Q"]
    S = np.concatenate([x["S"] for x in parts])
    emission = 4 * math.pi * np.sum(p.freq_w[:, None, None, None] * p.eps * p.chi * p.B, axis=0)
    gate = 1e-3 * np.abs(full["Q"]) + 1e-6 * emission
    slow = int(np.argmax([x["iters"] for x in parts]))
    if prec == "fp64":
        assert iters == full["iters"]
        sl = slice(b[slow], b[slow + 1])
        np.testing.assert_allclose(parts[slow]["S"], full["S"][sl], rtol=1e-11)
        np.testing.assert_allclose(parts[slow]["J"], full["J"][sl], rtol=1e-11)
        assert np.max(np.abs(S / full["S"] - 1)) < 20 * p.tol
        assert np.all(np.abs(Q - full["Q"]) <= gate)
    else:
        assert abs(iters - full["iters"]) <= 1
        assert np.max(np.abs(S / full["S"] - 1)) < 1e-3
        assert np.all(np.abs(Q - full["Q"]) <= gate)
