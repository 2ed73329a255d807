"""Frequency sharding of a multi-bin solve over ranks (one GPU per rank).

In the Jacobi ALI the frequency bins are independent: J_nu depends on S_nu
only, and S_nu = (1 - eps_nu) J_nu + eps_nu B_nu (Eq. 24).  What couples them is
the stopping rule (Eq. 25, the largest relative change over every cell and bin)
and the heating rate's sum over frequency (Sec. 4).  So each rank solves a
contiguous block of bins on its own grid until its own bins meet Eq. 25; the
heating rate is one all-reduce sum of the ranks' partial sums; the iteration
count reported is the largest over the ranks.

Every bin meets the stopping test.  While each bin's largest change falls
monotonically (as in the benchmark media) the rank holding the slowest bin
takes exactly the single solve's iterations and its bins come out as in the
single solve; the other ranks stop earlier, their bins within the stopping
tolerance of the single solve's.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def bin_blocks(nf: int, world: int) -> list:
    """First bin of each rank's block, and nf: rank r owns bins [b[r], b[r+1])."""
    return [(r * nf) // world for r in range(world + 1)]


def sub_problem(p, f0: int, f1: int):
    """The problem restricted to bins [f0, f1)."""
    return dataclasses.replace(p, name=f"{p.name}_bins{f0}-{f1}", chi=np.ascontiguousarray(p.chi[f0:f1]),
                               eps=np.ascontiguousarray(p.eps[f0:f1]), B=np.ascontiguousarray(p.B[f0:f1]),
                               freq_w=np.ascontiguousarray(p.freq_w[f0:f1]))


def gpu_solver(prec="mixed", max_iter=20000):
    """A solver of a (sub)problem on this process's GPU through the library:
    returns dict(S, J, Q, iters) with Q the bins' part of the heating rate."""
    def solve(p):
        from . import rt
        g = rt.Grid.from_problem(p, prec=prec)
        g.set_opacity_source(p.chi, p.eps, p.B, p.freq_w)
        iters, _, _ = g.ali_solve(tol=p.tol, max_iter=max_iter)
        m = g.moments(want=("J", "Q"))
        out = dict(S=g.get_S(), J=m["J"], Q=m["Q"], iters=iters)
        g.close()
        return out
    return solve


def solve_frequency_sharded(p, comm=None, solver=None):
    """Jacobi ALI of problem ``p`` with its bins shared out over the ranks of
    ``comm`` (a ``torch.distributed`` module with an initialised process group;
    None: one rank).  ``solver(sub_problem) -> dict(S, J, Q, iters)`` solves one
    block (default: ``gpu_solver()``).  Returns, on every rank, Q (summed over
    all bins) and iters (the largest over ranks); on rank 0 also S and J of
    every bin, [nf][nz][ny][nx] (None elsewhere)."""
    solver = solver or gpu_solver()
    world = comm.get_world_size() if comm else 1
    rank = comm.get_rank() if comm else 0
    if p.nf < world:
        raise ValueError("fewer frequency bins than ranks")
    b = bin_blocks(p.nf, world)
    mine = solver(sub_problem(p, b[rank], b[rank + 1]))
    Q = np.ascontiguousarray(mine["Q"], dtype=np.float64)
    iters = int(mine["iters"])
    if not comm:
        return dict(S=mine["S"], J=mine["J"], Q=Q, iters=iters)
    import torch
    tq = torch.from_numpy(Q.copy())
    comm.all_reduce(tq, op=comm.ReduceOp.SUM)          # the one collective of the data path
    ti = torch.tensor([iters], dtype=torch.int64)
    comm.all_reduce(ti, op=comm.ReduceOp.MAX)
    out = dict(Q=tq.numpy(), iters=int(ti.item()), S=None, J=None)
    # S and J of every bin on rank 0
    shape = lambda r: (b[r + 1] - b[r],) + tuple(p.chi.shape[1:])
    if rank == 0:
        S_parts, J_parts = [mine["S"]], [mine["J"]]
        for r in range(1, world):
            bs, bj = torch.empty(shape(r), dtype=torch.float64), torch.empty(shape(r), dtype=torch.float64)
            comm.recv(bs, src=r, tag=20_000 + 2 * r)
            comm.recv(bj, src=r, tag=20_001 + 2 * r)
            S_parts.append(bs.numpy())
            J_parts.append(bj.numpy())
        out["S"] = np.concatenate(S_parts, axis=0)
        out["J"] = np.concatenate(J_parts, axis=0)
    else:
        comm.send(torch.from_numpy(np.ascontiguousarray(mine["S"], dtype=np.float64)), dst=0, tag=20_000 + 2 * rank)
        comm.send(torch.from_numpy(np.ascontiguousarray(mine["J"], dtype=np.float64)), dst=0, tag=20_001 + 2 * rank)
    return out
