"""Pins for the oracle's angle quadrature (paper Sec. 3.2).

The quadrature must integrate the low even moments of the unit sphere exactly
((1/4pi) int mu_i^2 dOmega = 1/3, (1/4pi) int mu_i^4 dOmega = 1/5, ...), be identical in
every octant and invariant under 90-degree rotations, and have n_mu (n_mu + 2)
rays (half in 2D).  The LQ4 level has a closed form; the LQ6 and LQ8 sets are
compared with the published level-symmetric tables (Lathrop & Carlson 1964,
also in Lewis & Miller, "Computational Methods of Neutron Transport", Table 4-1).
"""
import itertools
import math

import numpy as np
import pytest

from oracle.quadrature import angle_count, level_symmetric


@pytest.mark.parametrize("n_mu", [2, 4, 6, 8, 10, 12])
@pytest.mark.parametrize("two_d", [False, True])
def test_count_and_normalisation(n_mu, two_d):
    mu, w = level_symmetric(n_mu, two_d)
    assert len(w) == angle_count(n_mu, two_d)
    if n_mu > 2:
        assert len(w) == n_mu * (n_mu + 2) // (2 if two_d else 1)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(w > 0)
    np.testing.assert_allclose(np.sum(mu ** 2, axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("n_mu", [2, 4, 6, 8, 10, 12])
def test_sphere_moments(n_mu):
    mu, w = level_symmetric(n_mu)
    # first and odd moments vanish; second moment is delta_ij / 3
    np.testing.assert_allclose(w @ mu, 0.0, atol=1e-15)
    M2 = np.einsum("k,ki,kj->ij", w, mu, mu)
    np.testing.assert_allclose(M2, np.eye(3) / 3.0, atol=1e-14)
    M3 = np.einsum("k,ki,kj,kl->ijl", w, mu, mu, mu)
    np.testing.assert_allclose(M3, 0.0, atol=1e-15)
    # exact even moments of mu_z: 1/(2p+1) for p up to the number of weight classes + 1
    nclass = {2: 0, 4: 1, 6: 2, 8: 3, 10: 4, 12: 5}[n_mu]
    for p in range(1, nclass + 2):
        for a in range(3):
            assert abs(np.sum(w * mu[:, a] ** (2 * p)) - 1.0 / (2 * p + 1)) < 1e-13, (p, a)
    # mixed fourth moment <mu_x^2 mu_y^2> = 1/15 whenever <mu^4> = 1/5
    if n_mu >= 4:
        assert abs(np.sum(w * mu[:, 0] ** 2 * mu[:, 1] ** 2) - 1.0 / 15.0) < 1e-14


def test_two_stream_is_cell_diagonal():
    mu, w = level_symmetric(2)
    np.testing.assert_allclose(np.abs(mu), 1.0 / math.sqrt(3.0), rtol=1e-15)
    np.testing.assert_allclose(w, 1.0 / 8.0)


def test_lq4_closed_form():
    # 6 a^2 - 4 a + 2/5 = 0 from <mu^4> = 1/5 with a single weight class
    a = (4.0 - math.sqrt(16.0 - 9.6)) / 12.0
    mu, w = level_symmetric(4)
    levels = np.unique(np.round(np.abs(mu), 14))
    np.testing.assert_allclose(levels, [math.sqrt(a), math.sqrt(1 - 2 * a)], rtol=1e-13)
    np.testing.assert_allclose(w, 1.0 / 24.0, rtol=1e-14)


@pytest.mark.parametrize("n_mu,levels,weights", [
    # the level-symmetric S6 / S8 sets as tabulated in E. E. Lewis & W. F. Miller,
    # Computational Methods of Neutron Transport (Wiley 1984), Table 4-1 (weights
    # normalised to 1 per octant); they are the Carlson sets (Sec. 3.2 cites
    # Carlson 1963 for the construction)
    (6, [0.2666355, 0.6815076, 0.9261808], [0.1761263, 0.1572071]),
    (8, [0.2182179, 0.5773503, 0.7867958, 0.9511897], [0.1209877, 0.0907407, 0.0925926]),
])
def test_published_tables(n_mu, levels, weights):
    mu, w = level_symmetric(n_mu)
    got = np.unique(np.round(np.abs(mu), 12))
    np.testing.assert_allclose(got, levels, atol=2e-7)
    per_octant = np.unique(np.round(w * 8.0, 12))
    np.testing.assert_allclose(sorted(per_octant), sorted(weights), atol=3e-7)


@pytest.mark.parametrize("n_mu", [4, 6, 8])
def test_octant_and_rotation_symmetry(n_mu):
    mu, w = level_symmetric(n_mu)
    table = {tuple(np.round(m, 12)): wk for m, wk in zip(mu, w)}
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            for m, wk in zip(mu, w):
                img = tuple(np.round(np.array(signs) * m[list(perm)], 12))
                assert img in table and abs(table[img] - wk) < 1e-14


def test_order_contract():
    # octant o has signs (-1 if o&1, -1 if o&2, -1 if o&4); nodes i outer, j inner
    mu, _ = level_symmetric(4)
    assert mu.shape == (24, 3)
    for o in range(8):
        block = mu[3 * o:3 * o + 3]
        assert np.all(np.sign(block[:, 0]) == (-1 if o & 1 else 1))
        assert np.all(np.sign(block[:, 1]) == (-1 if o & 2 else 1))
        assert np.all(np.sign(block[:, 2]) == (-1 if o & 4 else 1))
    # first octant: (1,1,2), (1,2,1), (2,1,1) in level indices
    lo, hi = np.unique(np.round(np.abs(mu[:3]), 12))
    np.testing.assert_allclose(mu[0], [lo, lo, hi])
    np.testing.assert_allclose(mu[1], [lo, hi, lo])
    np.testing.assert_allclose(mu[2], [hi, lo, lo])


def test_2d_set_is_upper_hemisphere_doubled():
    mu3, w3 = level_symmetric(6)
    mu2, w2 = level_symmetric(6, two_d=True)
    up = mu3[:, 2] > 0
    np.testing.assert_allclose(mu2, mu3[up])
    np.testing.assert_allclose(w2, 2 * w3[up])
