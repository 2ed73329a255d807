"""Domain decomposition along z (Sec. 3.5): z slabs solved as grids of their own.

A face between two slabs (and, on a periodic z axis, the wrap) is a subdomain
face (``rt.EXTERNAL``): its one-cell ghost layer holds the neighbouring slab's
opacity, B and current source function on the plane next to the face and, for
the rays entering through it, the neighbour's intensities there from the
previous iteration (before the first, its S, as for lagged periodic ghosts).
Every iteration each slab does one Jacobi step (formal solution + update,
Eq. 24); the stopping rule is the global max |dS|/S (Eq. 25).  Converged slabs
agree with the undecomposed domain to about the stopping tolerance, in a few
more iterations (the lag across the faces).

The exchange is the same on one GPU and across processes: each slab is a
``GridSlab`` (a C-ABI grid on this process's GPU); slabs owned by other ranks
of a ``torch.distributed`` process group receive their ghost planes by
point-to-point messages into their own buffers.  The slab objects only need
``set_face``, ``begin``, ``iterate``, ``face_intensity``, ``boundary_S``, ``S``
and ``J`` (any object with those methods can stand in for one).
"""
from __future__ import annotations

import numpy as np

from . import rt


def slab_bounds(nz: int, nslab: int) -> list:
    """First plane of each slab, and nz: slab d holds planes [z0[d], z0[d+1])."""
    return [(d * nz) // nslab for d in range(nslab + 1)]


def slab_owner(nslab: int, world: int) -> list:
    """Rank owning each slab: contiguous balanced blocks."""
    base, extra = divmod(nslab, world)
    owner = []
    for r in range(world):
        owner += [r] * (base + (1 if r < extra else 0))
    return owner


class GridSlab:
    """One slab as an FP64 grid of the CUDA library with subdomain z faces."""

    def __init__(self, p, z0: int, z1: int, ext_lo: bool, ext_hi: bool):
        bl = list(p.bc_lo)
        bh = list(p.bc_hi)
        if ext_lo:
            bl[2] = rt.EXTERNAL
        if ext_hi:
            bh[2] = rt.EXTERNAL
        self.g = rt.Grid(p.nx, p.ny, z1 - z0, n_mu=p.n_mu, nfreq=p.nf, bc_lo=tuple(bl), bc_hi=tuple(bh),
                         dx=p.dx, dy=p.dy, dz=p.dz, prec=rt.FP64)
        self.g.set_opacity_source(p.chi[:, z0:z1], p.eps[:, z0:z1], p.B[:, z0:z1], p.freq_w)
        self.ext = (ext_lo, ext_hi)
        self.n_angles = self.g.n_angles

    def set_face(self, side, chi=None, S=None, B=None, I=None):
        self.g.set_external_face(side, chi=chi, S=S, B=B, I=I)

    def begin(self):
        self.g.ali_begin(None)

    def iterate(self) -> float:
        return self.g.ali_iterate(1)[1]

    def face_intensity(self, side):
        return self.g.face_intensity(side)

    def boundary_S(self, side):
        S = self.g.get_S()
        return np.ascontiguousarray(S[:, 0 if side == 0 else -1])

    def S(self):
        return self.g.get_S()

    def J(self):
        return self.g.moments(want=("J",))["J"]

    def close(self):
        self.g.close()


def slab_ali_solve(p, nslab: int, tol: float = 1e-6, max_iter: int = 1000, comm=None, make_slab=None):
    """Jacobi ALI of problem ``p`` with its z axis split into ``nslab`` slabs.

    ``comm``: a ``torch.distributed`` module with an initialised process group
    (the slabs are shared out over its ranks in contiguous blocks), or None for
    all slabs in this process.  ``make_slab(p, z0, z1, ext_lo, ext_hi)`` builds a
    slab (default ``GridSlab``).  Returns dict(S, J, iters, resid, converged),
    S and J [nf][nz][ny][nx] on rank 0 (None elsewhere)."""
    make_slab = make_slab or GridSlab
    nx, ny, nz = p.nx, p.ny, p.nz
    if nz < 2 * nslab or p.nz == 1:
        raise ValueError("slabs of at least two planes each split the z axis of a 3D grid")
    if nslab > 1 and rt.FIXED in tuple(p.bc_lo[:2]) + tuple(p.bc_hi[:2]):
        raise ValueError("slabs need x and y faces without fixed incident intensities")
    per_z = p.bc_lo[2] == rt.PERIODIC
    z0 = slab_bounds(nz, nslab)
    world = comm.get_world_size() if comm else 1
    rank = comm.get_rank() if comm else 0
    owner = slab_owner(nslab, world)
    mine = [d for d in range(nslab) if owner[d] == rank]
    below = lambda d: (d - 1) % nslab if (d > 0 or per_z) else None   # slab beyond the low face
    above = lambda d: (d + 1) % nslab if (d < nslab - 1 or per_z) else None
    slabs = {d: make_slab(p, z0[d], z0[d + 1], below(d) is not None, above(d) is not None) for d in mine}
    na = next(iter(slabs.values())).n_angles if slabs else 0

    def exchange(payload):
        """payload[d] = (low-plane data, high-plane data) of each slab this rank
        owns; returns for each owned slab (data of the slab below's high plane,
        data of the slab above's low plane), by point-to-point messages where
        the neighbour lives on another rank."""
        got = {}
        reqs = []
        if comm:
            import torch
        for d in mine:
            lo_nb, hi_nb = below(d), above(d)
            pair = [None, None]
            for k, nb, want in ((0, lo_nb, 1), (1, hi_nb, 0)):
                if nb is None:
                    continue
                if owner[nb] == rank:
                    pair[k] = payload[nb][want]
                else:
                    buf = torch.empty(payload[d][0].shape, dtype=torch.float64)
                    reqs.append(comm.irecv(buf, src=owner[nb], tag=2 * nb + want))
                    pair[k] = buf
            got[d] = pair
        if comm:
            for d in mine:   # send this slab's planes to neighbours on other ranks
                for nb, side in ((below(d), 0), (above(d), 1)):
                    if nb is not None and owner[nb] != rank:
                        t = torch.from_numpy(np.ascontiguousarray(payload[d][side]))
                        reqs.append(comm.isend(t, dst=owner[nb], tag=2 * d + side))
            for r in reqs:
                r.wait()
            for d in got:
                got[d] = [x.numpy() if hasattr(x, "numpy") else x for x in got[d]]
        return got

    # static ghost layers (chi, B) once; then every iteration S and the intensities
    lay = lambda a, z: np.ascontiguousarray(a[:, z])
    stat = exchange({d: (np.stack([lay(p.chi, z0[d]), lay(p.B, z0[d])]),
                         np.stack([lay(p.chi, z0[d + 1] - 1), lay(p.B, z0[d + 1] - 1)])) for d in mine})
    for d in mine:
        for side in (0, 1):
            if stat[d][side] is not None:
                slabs[d].set_face(side, chi=stat[d][side][0], B=stat[d][side][1])
        slabs[d].begin()
    Sb = {d: (slabs[d].boundary_S(0), slabs[d].boundary_S(1)) for d in mine}
    nbS = exchange(Sb)
    # before the first iteration the incoming intensities are the neighbour plane's S
    Iin = {d: [None if x is None else np.repeat(x[:, None], na, axis=1) for x in nbS[d]] for d in mine}
    r = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        rl = 0.0
        for d in mine:
            for side in (0, 1):
                if nbS[d][side] is not None:
                    slabs[d].set_face(side, S=nbS[d][side], I=Iin[d][side])
            rl = max(rl, slabs[d].iterate())
        if comm:
            import torch
            t = torch.tensor([rl], dtype=torch.float64)
            comm.all_reduce(t, op=comm.ReduceOp.MAX)
            rl = float(t.item())
        r = rl
        # the neighbours' new boundary S and this formal solution's face intensities
        nbS = exchange({d: (slabs[d].boundary_S(0), slabs[d].boundary_S(1)) for d in mine})
        faces = exchange({d: (slabs[d].face_intensity(0) if below(d) is not None else np.zeros((p.nf, na, ny, nx)),
                              slabs[d].face_intensity(1) if above(d) is not None else np.zeros((p.nf, na, ny, nx)))
                          for d in mine})
        Iin = {d: faces[d] for d in mine}
        if r <= tol:
            break
    S_loc = {d: slabs[d].S() for d in mine}
    J_loc = {d: slabs[d].J() for d in mine}
    for s in slabs.values():
        if hasattr(s, "close"):
            s.close()
    if comm:
        import torch
        if rank == 0:
            for d in range(nslab):
                if owner[d] != 0:
                    shape = (p.nf, z0[d + 1] - z0[d], ny, nx)
                    bs, bj = torch.empty(shape, dtype=torch.float64), torch.empty(shape, dtype=torch.float64)
                    comm.recv(bs, src=owner[d], tag=10_000 + 2 * d)
                    comm.recv(bj, src=owner[d], tag=10_001 + 2 * d)
                    S_loc[d], J_loc[d] = bs.numpy(), bj.numpy()
        else:
            for d in mine:
                comm.send(torch.from_numpy(np.ascontiguousarray(S_loc[d])), dst=0, tag=10_000 + 2 * d)
                comm.send(torch.from_numpy(np.ascontiguousarray(J_loc[d])), dst=0, tag=10_001 + 2 * d)
            return dict(S=None, J=None, iters=it, resid=r, converged=r <= tol)
    S = np.concatenate([S_loc[d] for d in range(nslab)], axis=1)
    J = np.concatenate([J_loc[d] for d in range(nslab)], axis=1)
    return dict(S=S, J=J, iters=it, resid=r, converged=r <= tol)
