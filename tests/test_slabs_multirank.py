"""The slab decomposition's exchange (paper_1201_2222_gb300.slabs, Sec. 3.5) on
CPU: each slab is an oracle-backed stand-in for the library's grid (the
oracle's formal solution with subdomain z faces and the Jacobi update), driven
by the same exchange code as the GPU slabs.

* In one process the driver reproduces the oracle's own ``slab_ali_solve`` bit
  for bit (same S, J and iteration count).
* On two gloo ranks, each owning a block of slabs and exchanging the ghost
  planes by point-to-point messages, the result is the same again.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1201_2222_gb300 import slabs as SL  # noqa: E402
from paper_1201_2222_gb300 import workloads as W  # noqa: E402

P, V, T = O.PERIODIC, O.VACUUM, O.THERMAL


class OracleSlab:
    """A slab as the oracle solves it (the interface of slabs.GridSlab)."""

    def __init__(self, p, z0, z1, ext_lo, ext_hi):
        bl, bh = list(p.bc_lo), list(p.bc_hi)
        if ext_lo:
            bl[2] = O.EXTERNAL
        if ext_hi:
            bh[2] = O.EXTERNAL
        self.g = O.Grid(p.nx, p.ny, z1 - z0, p.n_mu, bc_lo=tuple(bl), bc_hi=tuple(bh),
                        dx=p.dx, dy=p.dy, dz=p.dz)
        self.chi, self.eps, self.B = (np.ascontiguousarray(a[:, z0:z1]) for a in (p.chi, p.eps, p.B))
        self.nf = p.nf
        self.n_angles = self.g.na
        self.face = [dict(), dict()]
        self.ext = (ext_lo, ext_hi)

    def set_face(self, side, chi=None, S=None, B=None, I=None):
        for k, v in (("chi", chi), ("S", S), ("B", B), ("I", I)):
            if v is not None:
                self.face[side][k] = np.array(v)

    def begin(self):
        self.S_ = self.B.copy()
        self.G = [O.init_ghosts(self.g, self.S_[f]) for f in range(self.nf)]
        self.lstar = None
        self.Iz = None

    def iterate(self):
        J = np.empty_like(self.S_)
        first = self.lstar is None
        if first:
            self.lstar = np.empty_like(self.S_)
        Iz = [[], []]
        for f in range(self.nf):
            ext = {}
            for side, key in ((0, "lo"), (1, "hi")):
                if self.ext[side]:
                    x = self.face[side]
                    ext[key] = (x["chi"][f], x["S"][f], x["I"][f], x["B"][f])
            res = O.formal_solution(self.g, self.chi[f], self.S_[f], self.B[f], self.G[f], ext=ext)
            J[f] = res["J"]
            if first:
                self.lstar[f] = res["lstar"]
            self.G[f] = res["G_next"]
            Iz[0].append(res["I_zlo"])
            Iz[1].append(res["I_zhi"])
        self.Iz = [np.stack(Iz[0]), np.stack(Iz[1])]
        self.J_ = J
        e = self.eps
        dS = ((1.0 - e) * J + e * self.B - self.S_) / (1.0 - (1.0 - e) * self.lstar)
        self.S_ = self.S_ + dS
        return O.max_relative_change(dS, self.S_)

    def face_intensity(self, side):
        return self.Iz[side]

    def boundary_S(self, side):
        return np.ascontiguousarray(self.S_[:, 0 if side == 0 else -1])

    def S(self):
        return self.S_

    def J(self):
        return self.J_


def _problem(case):
    if case == "atmosphere":
        return W.stratified_atmosphere(12, nxy=5), 3
    if case == "periodic":
        return W.random_box(5, 4, 8, seed=51, n_mu=4, nf=2, bc_lo=(P, P, P), bc_hi=(P, P, P)), 2
    return W.random_box(4, 5, 9, seed=52, n_mu=4, bc_lo=(T, V, T), bc_hi=(V, T, V)), 4


@pytest.mark.parametrize("case", ["atmosphere", "periodic", "bounded"])
def test_driver_reproduces_the_oracle_slab_solve(case):
    p, nslab = _problem(case)
    tol = 1e-8
    got = SL.slab_ali_solve(p, nslab, tol=tol, max_iter=3000, make_slab=OracleSlab)
    ref = O.slab_ali_solve(O.Grid.from_problem(p), p.chi, p.eps, p.B, nslab, tol=tol, max_iter=3000)
    assert got["iters"] == ref["iters"] and got["converged"]
    np.testing.assert_array_equal(got["S"], ref["S"])
    np.testing.assert_array_equal(got["J"], ref["J"])


def test_slab_layout():
    assert SL.slab_bounds(12, 3) == [0, 4, 8, 12]
    assert SL.slab_bounds(9, 2) == [0, 4, 9]
    assert SL.slab_owner(5, 2) == [0, 0, 0, 1, 1]
    assert SL.slab_owner(4, 4) == [0, 1, 2, 3]
    p = W.random_box(4, 4, 5, seed=1, n_mu=4)
    with pytest.raises(ValueError):
        SL.slab_ali_solve(p, 3, make_slab=OracleSlab)      # slabs of fewer than 2 planes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, nslab = _problem(case)
    out = SL.slab_ali_solve(p, nslab, tol=1e-8, max_iter=3000, comm=dist, make_slab=OracleSlab)
    q.put((rank, out["iters"], out["S"], out["J"]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", ["atmosphere", "periodic"])
def test_two_gloo_ranks_exchange_ghost_planes(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, nslab = _problem(case)
    ref = O.slab_ali_solve(O.Grid.from_problem(p), p.chi, p.eps, p.B, nslab, tol=1e-8, max_iter=3000)
    (r0, it0, S0, J0), (r1, it1, S1, J1) = out
    assert it0 == it1 == ref["iters"]
    assert S1 is None and J1 is None                      # results gathered on rank 0
    np.testing.assert_array_equal(S0, ref["S"])
    np.testing.assert_array_equal(J0, ref["J"])
