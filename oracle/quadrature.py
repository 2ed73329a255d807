"""Angle quadrature for the oracle (paper Sec. 3.2).

The paper discretises each octant identically (Carlson type-A / Bruls et al.
1999 App. B), with n_a = n_mu (n_mu + 2) rays in 3D and half of them in 2D.
The node construction is not reproduced in the paper, so this oracle uses the
level-symmetric LQ_n family, which satisfies the paper's constraints
(octant-identical, invariant under 90-degree rotations about the axes):

* the direction-cosine levels obey mu_i^2 = mu_1^2 + (i - 1) 2 (1 - 3 mu_1^2)/(n_mu - 2),
  i = 1 .. n_mu/2;
* the nodes of one octant are (mu_i, mu_j, mu_l) with i + j + l = n_mu/2 + 2;
* nodes that are permutations of each other share one weight;
* mu_1 and the class weights are fixed by sum(w) = 1 and the even moments
  sum(w mu_z^2p) = 1/(2p + 1) for p = 2 .. n_classes + 1 (p = 1 holds by symmetry).

n_mu = 2 is the two-stream set: one ray per octant along the cell diagonal.
In 2D (nz == 1) the rays with mu_z > 0 are kept and their weights doubled.

Angle order (shared contract with the library, because user boundary arrays
are indexed by angle): octant o = 0..7 with signs
(sx, sy, sz) = (-1 if o & 1 else +1, -1 if o & 2 else +1, -1 if o & 4 else +1);
inside an octant, i = 1..n_mu/2 outer, j inner, l = n_mu/2 + 2 - i - j.
Weights sum to 1 over the sphere (Eq. 17 has no 4 pi).

Parity: pinned by tests/test_oracle_quadrature.py (moment identities, the closed
form of LQ4, published LQ6/LQ8 tables, exact integration of low-order
polynomials over the sphere).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _octant_nodes(n_mu: int):
    half = n_mu // 2
    nodes = []
    for i in range(1, half + 1):
        for j in range(1, half + 1):
            l = half + 2 - i - j
            if l >= 1:
                nodes.append((i, j, l))
    return nodes


def _levels(a: float, n_mu: int) -> np.ndarray:
    half = n_mu // 2
    i = np.arange(1, half + 1, dtype=np.float64)
    return a + (i - 1.0) * 2.0 * (1.0 - 3.0 * a) / (n_mu - 2)


def _moment_system(a: float, n_mu: int):
    """Rows of the linear system in the class weights for fixed mu_1^2 = a:
    sum w = 1 and sum w mu_z^(2p) = 1/(2p+1), p = 2 .. n_classes + 1."""
    nodes = _octant_nodes(n_mu)
    classes = sorted({tuple(sorted(n)) for n in nodes})
    mu2 = _levels(a, n_mu)
    nc = len(classes)
    M = np.zeros((nc + 1, nc))
    b = np.zeros(nc + 1)
    for n in nodes:
        c = classes.index(tuple(sorted(n)))
        M[0, c] += 1.0
        for p in range(2, nc + 2):
            M[p - 1, c] += mu2[n[2] - 1] ** p
    b[0] = 1.0
    for p in range(2, nc + 2):
        b[p - 1] = 1.0 / (2 * p + 1)
    return classes, M, b


def _consistency(a: float, n_mu: int) -> float:
    """det of the augmented matrix [M | b]: zero where the moment equations admit
    a weight vector (the equations outnumber the weights by one)."""
    _, M, b = _moment_system(a, n_mu)
    return float(np.linalg.det(np.column_stack([M, b])))


def _class_weights(a: float, n_mu: int):
    classes, M, b = _moment_system(a, n_mu)
    w, *_ = np.linalg.lstsq(M, b, rcond=None)
    return classes, w, float(np.abs(M @ w - b).max())


def level_symmetric(n_mu: int, two_d: bool = False):
    """Return (mu [n_a, 3], w [n_a]) for the LQ_n set in the documented order."""
    if n_mu == 2:
        m = 1.0 / math.sqrt(3.0)
        octant = [((m, m, m), 1.0)]
    else:
        if n_mu % 2 or n_mu < 4 or n_mu > 12:
            raise ValueError("n_mu must be 2, 4, 6, 8, 10 or 12")
        f = lambda a: _consistency(a, n_mu)
        grid = np.linspace(1e-6, 1.0 / 3.0 - 1e-6, 4001)
        vals = np.array([f(a) for a in grid])
        roots = []
        for k in range(len(grid) - 1):
            if vals[k] == 0.0 or vals[k] * vals[k + 1] < 0:
                roots.append(brentq(f, grid[k], grid[k + 1], xtol=1e-15, rtol=1e-15))
        good = []
        for a in roots:
            classes, w, res = _class_weights(a, n_mu)
            if res < 1e-12 and np.all(w > 0) and np.all(_levels(a, n_mu) > 0):
                good.append((a, classes, w))
        if not good:
            raise ValueError(f"no positive level-symmetric set for n_mu={n_mu}")
        a, classes, wcls = good[0]
        mu = np.sqrt(_levels(a, n_mu))
        octant = []
        for n in _octant_nodes(n_mu):
            octant.append(((mu[n[0] - 1], mu[n[1] - 1], mu[n[2] - 1]),
                           float(wcls[classes.index(tuple(sorted(n)))])))
    mus, ws = [], []
    for o in range(8):
        sx = -1.0 if o & 1 else 1.0
        sy = -1.0 if o & 2 else 1.0
        sz = -1.0 if o & 4 else 1.0
        if two_d and sz < 0:
            continue
        for (mx, my, mz), w in octant:
            mus.append((sx * mx, sy * my, sz * mz))
            ws.append(w / 8.0 * (2.0 if two_d else 1.0))
    return np.array(mus), np.array(ws)


def angle_count(n_mu: int, two_d: bool = False) -> int:
    na = 8 if n_mu == 2 else n_mu * (n_mu + 2)
    return na // 2 if two_d else na
