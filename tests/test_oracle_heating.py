"""Pins of the oracle's heating-rate forms (Sec. 4): Q^int, Q^dif = -4 pi div H and
the chi dx switch between them.

The discrete divergence is pinned by closed forms of centred differences
(sinusoids on periodic axes, linear fields on bounded ones) and by the
telescoping sum on a periodic box; the sign, the 4 pi and the link between H and
J by the zeroth moment of the transfer equation (Eq. 8 integrated over angle:
div H = chi (S - J), so Q^dif -> Q^int as the grid is refined).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

P, V = O.PERIODIC, O.VACUUM


def _grid(n, per=(True, True, True), d=(1.0, 1.0, 1.0), n_mu=4):
    lo = tuple(P if p else V for p in per)
    return O.Grid(*n, n_mu=n_mu, bc_lo=lo, bc_hi=lo, dx=d[0], dy=d[1], dz=d[2])


def test_divergence_of_sinusoids_is_the_centred_difference_closed_form():
    nx, ny, nz = 12, 10, 8
    dx, dy, dz = 0.7, 1.3, 0.9
    g = _grid((nx, ny, nz), d=(dx, dy, dz))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ax, ay, az = 2 * math.pi * 2 / nx, 2 * math.pi * 3 / ny, 2 * math.pi / nz
    H = np.stack([np.sin(ax * i), np.cos(ay * j), np.sin(az * k + 0.3)])
    # (sin(a(i+1)) - sin(a(i-1))) / 2h = cos(a i) sin(a) / h, and likewise for cos
    want = (np.cos(ax * i) * math.sin(ax) / dx - np.sin(ay * j) * math.sin(ay) / dy
            + np.cos(az * k + 0.3) * math.sin(az) / dz)
    np.testing.assert_allclose(O.divergence(g, H), want, atol=1e-13)


def test_divergence_of_linear_fields_on_bounded_axes_is_exact_at_every_cell():
    g = _grid((6, 5, 7), per=(False, False, False), d=(0.5, 2.0, 1.5))
    k, j, i = np.meshgrid(np.arange(7), np.arange(5), np.arange(6), indexing="ij")
    H = np.stack([1.0 + 0.25 * (i * 0.5), -2.0 + 1.5 * (j * 2.0), 3.0 - 0.75 * (k * 1.5)])
    np.testing.assert_allclose(O.divergence(g, H), 0.25 + 1.5 - 0.75, atol=1e-13)


def test_divergence_sums_to_zero_on_a_periodic_box():
    g = _grid((9, 7, 5), d=(1.0, 1.0, 1.0))
    H = np.random.default_rng(3).normal(size=(3, 5, 7, 9))
    assert abs(O.divergence(g, H).sum()) < 1e-11


def test_divergence_is_zero_along_an_axis_of_one_cell():
    g = _grid((6, 5, 1), per=(True, True, True))
    H = np.zeros((3, 1, 5, 6))
    H[2] = np.random.default_rng(4).normal(size=(1, 5, 6))   # z component varies only in x, y
    np.testing.assert_array_equal(O.divergence(g, H), 0.0)


def _qdif_qint_gap(N):
    # LTE (eps = 1, S = B) in a uniform medium, B varying along x: one wavelength
    # across a box of unit length and optical depth 2 pi
    dx = 1.0 / N
    chi0 = 2 * math.pi
    g = _grid((N, 2, 2), d=(dx, dx, dx), n_mu=6)
    x = (np.arange(N) + 0.5) * dx
    B = np.broadcast_to(1.0 + 0.5 * np.sin(2 * math.pi * x), (1, 2, 2, N)).copy()
    chi = np.full_like(B, chi0)
    eps = np.ones_like(B)
    r = O.ali_solve(g, chi, eps, B, tol=1e-12, max_iter=500, nthreads=O.max_threads())
    q_int = O.heating_rate(chi, eps, r["J"], B, [1.0])
    q_dif = O.heating_rate_dif(g, r["H"], [1.0])
    return np.max(np.abs(q_dif - q_int)) / np.max(np.abs(q_int))


def test_differential_heating_converges_to_the_integral_form():
    e16, e32, e64 = (_qdif_qint_gap(n) for n in (16, 32, 64))
    assert e64 < 0.05
    assert e32 < 0.6 * e16 and e64 < 0.6 * e32


def _medium(g, nf, chi_dx):
    rng = np.random.default_rng(7)
    shape = (nf,) + g.shape
    chi = np.full(shape, chi_dx / O.cell_width(g))
    return (chi, rng.uniform(0.1, 1.0, shape), rng.uniform(0.5, 2.0, shape),
            rng.uniform(0.5, 2.0, shape), rng.normal(size=(nf, 3) + g.shape))


@pytest.mark.parametrize("chi_dx", [0.3, 1.0])
def test_switch_takes_the_integral_form_where_cells_are_thin(chi_dx):
    g = _grid((5, 4, 3), d=(1.0, 0.5, 0.25))
    chi, eps, J, B, H = _medium(g, 2, chi_dx)
    fw = [0.4, 0.6]
    np.testing.assert_allclose(O.heating_rate_switch(g, chi, eps, J, B, H, fw),
                               O.heating_rate(chi, eps, J, B, fw), rtol=1e-14, atol=1e-14)


def test_switch_takes_the_differential_form_where_cells_are_thick():
    g = _grid((5, 4, 3), d=(1.0, 0.5, 0.25))
    chi, eps, J, B, H = _medium(g, 2, 1.5)
    fw = [0.4, 0.6]
    np.testing.assert_allclose(O.heating_rate_switch(g, chi, eps, J, B, H, fw),
                               O.heating_rate_dif(g, H, fw), rtol=1e-15, atol=1e-15)


def test_switch_decides_per_cell_and_frequency():
    g = _grid((6, 1, 1), per=(True, True, True))
    chi, eps, J, B, H = _medium(g, 2, 0.5)
    chi[0, 0, 0, 3:] = 4.0    # frequency 0: thick in the right half
    fw = [1.0, 1.0]
    q = O.heating_rate_switch(g, chi, eps, J, B, H, fw)
    q_int = O.heating_rate(chi, eps, J, B, [1.0, 1.0])
    q_int1 = O.heating_rate(chi[1:], eps[1:], J[1:], B[1:], [1.0])
    q_dif0 = O.heating_rate_dif(g, H[:1], [1.0])
    np.testing.assert_allclose(q[..., :3], q_int[..., :3], rtol=1e-14)
    np.testing.assert_allclose(q[..., 3:], (q_dif0 + q_int1)[..., 3:], rtol=1e-14)
