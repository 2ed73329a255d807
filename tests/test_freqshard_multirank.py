"""Frequency sharding (paper_1201_2222_gb300.freqshard): the bins of a
multi-frequency solve split over ranks, each block solved on its own, the
heating rate summed by one all-reduce.  On CPU each block is solved by the
oracle (a stand-in for a rank's GPU), on one process and on two gloo ranks:

* one rank holding every bin is the single solve, bit for bit;
* with two ranks the iteration count (largest over ranks) is the single
  solve's, the rank holding the slowest bin returns its bins as in the single
  solve, the other rank's bins stop earlier within the stopping tolerance, and
  Q is the single solve's within the heating-rate gate.
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1201_2222_gb300 import freqshard as FS  # noqa: E402
from paper_1201_2222_gb300 import workloads as W  # noqa: E402


def oracle_solver(p):
    _, r = O.solve_problem(p, max_iter=20000)
    return dict(S=r["S"], J=r["J"], Q=O.heating_rate(p.chi, p.eps, r["J"], p.B, p.freq_w), iters=r["iters"])


def _problem():
    return W.multifrequency_atmosphere(8, nf=4)


def _reference():
    p = _problem()
    _, r = O.solve_problem(p, max_iter=20000)
    return p, r, O.heating_rate(p.chi, p.eps, r["J"], p.B, p.freq_w)


def test_blocks_and_sub_problems():
    assert FS.bin_blocks(4, 2) == [0, 2, 4]
    assert FS.bin_blocks(7, 3) == [0, 2, 4, 7]
    p = _problem()
    q = FS.sub_problem(p, 1, 3)
    assert q.nf == 2 and np.array_equal(q.chi, p.chi[1:3]) and np.array_equal(q.freq_w, p.freq_w[1:3])
    with pytest.raises(ValueError):
        FS.solve_frequency_sharded(FS.sub_problem(p, 0, 1), comm=_FakeComm(2), solver=oracle_solver)


class _FakeComm:
    def __init__(self, world):
        self.world = world

    def get_world_size(self):
        return self.world

    def get_rank(self):
        return 0


def test_one_rank_is_the_single_solve():
    p, ref, Qref = _reference()
    out = FS.solve_frequency_sharded(p, comm=None, solver=oracle_solver)
    assert out["iters"] == ref["iters"]
    np.testing.assert_array_equal(out["S"], ref["S"])
    np.testing.assert_array_equal(out["Q"], Qref)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = FS.solve_frequency_sharded(_problem(), comm=dist, solver=oracle_solver)
    q.put((rank, out["iters"], out["Q"], out["S"], out["J"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_bins():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, ref, Qref = _reference()
    (r0, it0, Q0, S0, J0), (r1, it1, Q1, S1, J1) = res
    assert it0 == it1 == ref["iters"]
    assert S1 is None and J1 is None                      # gathered on rank 0
    np.testing.assert_array_equal(Q0, Q1)                 # the all-reduced sum on every rank
    # bins 2, 3 (rank 1) hold the slowest bin: as in the single solve
    np.testing.assert_array_equal(S0[2:], ref["S"][2:])
    np.testing.assert_array_equal(J0[2:], ref["J"][2:])
    # bins 0, 1 stopped earlier, within the stopping tolerance
    assert np.max(np.abs(S0[:2] / ref["S"][:2] - 1)) < 20 * p.tol
    emission = 4 * math.pi * np.sum(p.freq_w[:, None, None, None] * p.eps * p.chi * p.B, axis=0)
    assert np.all(np.abs(Q0 - Qref) <= 1e-3 * np.abs(Qref) + 1e-6 * emission)
