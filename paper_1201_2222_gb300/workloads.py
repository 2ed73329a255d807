"""Seeded synthetic inputs shaped like the paper's radiative-transfer test problems.

This module only builds input fields (opacity, photon-destruction probability,
thermal source function, frequency weights and boundary settings).  It holds none
of the transfer method's arithmetic, so both the CPU oracle and the CUDA path can
draw their inputs from it.

Every field is returned in the layout the library expects: ``[nf][nz][ny][nx]``
float64, C-contiguous, with ``x`` the fastest index.

Workloads (sizes are the defaults; every builder also takes a smaller ``n`` so the
same structure can be run at sizes a slow CPU reference finishes quickly):

* ``stratified_atmosphere``: the paper's uniform-temperature non-LTE atmosphere
  (Sec. 5.1, Eq. 30 and the 3D variant with periodic horizontal boundaries):
  plane-parallel exponential atmosphere whose vertical optical depth runs
  log-spaced from 1e-4 at the top to 1e3 at the bottom, constant epsilon, B = 1,
  vacuum at the top and I = B at the bottom.
* ``turbulent_box``: a fully periodic box with a log-normal density drawn from a
  Gaussian random field with a k^(-11/3) spectrum, a log-normal temperature,
  absorption proportional to rho^2 T^-3.5 plus scattering proportional to rho,
  B = T^4 (the kind of structure of the paper's shearing-box snapshot, Sec. 5.3).
* ``multifrequency_atmosphere``: the stratified atmosphere with a horizontal
  temperature perturbation and free-free-like absorption over log-spaced
  frequency bins plus grey scattering (the multi-frequency spectra test, Sec. 5.1).
* ``large_stratified_turbulent``: the turbulent density on top of the stratified
  profile at 256^3 with epsilon = 1e-3.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC, VACUUM, THERMAL, FIXED = 0, 1, 2, 3


@dataclasses.dataclass
class Problem:
    """A complete transfer problem: grid, boundaries, angle order and fields."""

    name: str
    nx: int
    ny: int
    nz: int
    n_mu: int
    chi: np.ndarray          # total opacity chi_tot, [nf][nz][ny][nx]
    eps: np.ndarray          # photon destruction probability, same shape
    B: np.ndarray            # thermal source function, same shape
    freq_w: np.ndarray       # frequency quadrature weights, [nf]
    bc_lo: tuple = (PERIODIC, PERIODIC, THERMAL)
    bc_hi: tuple = (PERIODIC, PERIODIC, VACUUM)
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    tol: float = 1e-6
    recipe: str = ""

    @property
    def nf(self) -> int:
        return int(self.chi.shape[0])

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_angles(self) -> int:
        if self.n_mu == 2:
            na = 8
        else:
            na = self.n_mu * (self.n_mu + 2)
        return na // 2 if self.nz == 1 else na


def gaussian_random_field(n: int, seed: int, slope: float = -11.0 / 3.0) -> np.ndarray:
    """Unit-variance periodic Gaussian random field with power spectrum k^slope.

    White noise from ``numpy.random.default_rng(seed)`` is Fourier transformed,
    multiplied by |k|^(slope/2) with the k = 0 mode zeroed, transformed back and
    normalised to zero mean and unit variance.  Returns ``[n][n][n]`` (z, y, x).
    """
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(n) * n
    ky = np.fft.fftfreq(n) * n
    kx = np.fft.rfftfreq(n) * n
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)       # |k|^(slope/2)
    g = np.fft.irfftn(fk * amp, s=(n, n, n))
    g -= g.mean()
    g /= g.std()
    return g


def stratified_profile(nz: int, tau_top: float = 1e-4, tau_bot: float = 1e3, dz: float = 1.0):
    """Exponential atmosphere: chi_k = tau_k ln(r)/dz, with the centre optical depth
    tau_k log-spaced from ``tau_bot`` at k = 0 (bottom) to ``tau_top`` at k = nz-1 (top).
    """
    decades = math.log10(tau_bot / tau_top)
    r = 10.0 ** (decades / (nz - 1))
    k = np.arange(nz, dtype=np.float64)
    tau = tau_top * r ** ((nz - 1) - k)
    return tau * math.log(r) / dz, tau


def stratified_atmosphere(n: int = 32, eps: float = 1e-2, n_mu: int = 4, tol: float = 1e-6,
                          nxy: int | None = None) -> Problem:
    """Scattering atmosphere, 32^3 by default (periodic x, y; I = B below, vacuum above)."""
    nxy = n if nxy is None else nxy
    chi_z, _ = stratified_profile(n)
    shape = (1, n, nxy, nxy)
    chi = np.broadcast_to(chi_z[None, :, None, None], shape).copy()
    return Problem(
        name=f"stratified_atmosphere_{nxy}x{nxy}x{n}_eps{eps:g}_lq{n_mu}",
        nx=nxy, ny=nxy, nz=n, n_mu=n_mu, chi=chi,
        eps=np.full(shape, eps), B=np.ones(shape), freq_w=np.ones(1), tol=tol,
        recipe=("vertical centre optical depth log-spaced 1e-4 (top) .. 1e3 (bottom), "
                f"chi_k = tau_k ln r, eps = {eps:g}, B = 1, grey, periodic x/y, "
                "thermal bottom, vacuum top"))


def _turbulent_fields(n: int, seed_rho: int = 1, seed_T: int = 2):
    g1 = gaussian_random_field(n, seed_rho)
    g2 = gaussian_random_field(n, seed_T)
    rho = np.exp(g1 - 0.5)
    T = np.exp(0.3 * g2 - 0.045)
    return rho, T


def turbulent_box(n: int = 128, n_mu: int = 8, tau_box: float = 30.0, tol: float = 1e-6,
                  seed_rho: int = 1, seed_T: int = 2) -> Problem:
    """Fully periodic log-normal turbulent box, 128^3 and 80 angles by default."""
    rho, T = _turbulent_fields(n, seed_rho, seed_T)
    kap_a, kap_s = 0.1, 0.9                      # kappa_a / (kappa_a + kappa_s) = 0.1 at rho = T = 1
    chi_a = kap_a * rho ** 2 * T ** (-3.5)
    chi_s = kap_s * rho
    chi = chi_a + chi_s
    scale = tau_box / (chi.mean() * n)
    chi_a *= scale
    chi *= scale
    eps = chi_a / chi
    B = T ** 4
    shape = (1, n, n, n)
    return Problem(
        name=f"turbulent_box_{n}^3_lq{n_mu}", nx=n, ny=n, nz=n, n_mu=n_mu,
        chi=chi.reshape(shape), eps=eps.reshape(shape), B=B.reshape(shape), freq_w=np.ones(1),
        bc_lo=(PERIODIC, PERIODIC, PERIODIC), bc_hi=(PERIODIC, PERIODIC, PERIODIC), tol=tol,
        recipe=("rho = exp(g1 - 1/2), T = exp(0.3 g2 - 0.045), g1/g2 unit-variance GRFs with "
                f"P(k) ~ k^-11/3 (seeds {seed_rho}, {seed_T}); chi_abs ~ rho^2 T^-3.5, chi_sc ~ rho, "
                f"absorption fraction 0.1 at rho = T = 1, <chi> n = {tau_box:g}; B = T^4; fully periodic"))


def multifrequency_atmosphere(n: int = 64, nf: int = 64, n_mu: int = 4, tol: float = 1e-6,
                              x_lo: float = 0.01, x_hi: float = 30.0, eps_ref: float = 1e-2) -> Problem:
    """Stratified scattering atmosphere with free-free-like absorption in ``nf`` bins."""
    chi_sc_z, _ = stratified_profile(n)
    ix = np.arange(n, dtype=np.float64)
    T2 = 1.0 + 0.2 * np.sin(2 * np.pi * ix[None, :] / n) * np.sin(2 * np.pi * ix[:, None] / n)  # [y][x]
    T = np.broadcast_to(T2[None, :, :], (n, n, n))
    rho = np.broadcast_to((chi_sc_z / chi_sc_z[0])[:, None, None], (n, n, n))
    chi_sc = np.broadcast_to(chi_sc_z[:, None, None], (n, n, n))
    xs = np.exp(np.linspace(math.log(x_lo), math.log(x_hi), nf))
    C = eps_ref / (1.0 - eps_ref) * chi_sc_z[0] / (1.0 - math.exp(-1.0))
    chi = np.empty((nf, n, n, n))
    eps = np.empty_like(chi)
    B = np.empty_like(chi)
    for f, x in enumerate(xs):
        chi_a = C * rho ** 2 * T ** (-0.5) * x ** (-3) * (1.0 - np.exp(-x / T))
        chi[f] = chi_a + chi_sc
        eps[f] = chi_a / chi[f]
        B[f] = x ** 3 / np.expm1(x / T)
    fw = np.zeros(nf)
    if nf > 1:
        dxs = np.diff(xs)
        fw[:-1] += 0.5 * dxs
        fw[1:] += 0.5 * dxs
    else:
        fw[:] = 1.0
    return Problem(
        name=f"multifrequency_atmosphere_{n}^3_nf{nf}_lq{n_mu}", nx=n, ny=n, nz=n, n_mu=n_mu,
        chi=chi, eps=eps, B=B, freq_w=fw, tol=tol,
        recipe=(f"{n}^3, chi_sc from the stratified profile (tau 1e-4..1e3), "
                "T = 1 + 0.2 sin(2 pi x/n) sin(2 pi y/n), "
                f"{nf} bins x log-spaced in [{x_lo:g}, {x_hi:g}], chi_abs = C rho^2 T^-1/2 x^-3 (1 - e^-x/T), "
                "C sets eps = 1e-2 at x = 1, T = 1 in the bottom layer, B = x^3/(e^x/T - 1), "
                "trapezoid weights in x"))


def large_stratified_turbulent(n: int = 256, n_mu: int = 6, eps_scale: float = 1e-3,
                               tol: float = 1e-6) -> Problem:
    """Stratified profile times the turbulent density, epsilon = 1e-3, 48 angles, 256^3."""
    chi_z, _ = stratified_profile(n)
    rho, T = _turbulent_fields(n)
    chi = chi_z[:, None, None] * rho
    shape = (1, n, n, n)
    return Problem(
        name=f"stratified_turbulent_{n}^3_lq{n_mu}", nx=n, ny=n, nz=n, n_mu=n_mu,
        chi=chi.reshape(shape), eps=np.full(shape, eps_scale), B=(T ** 4).reshape(shape),
        freq_w=np.ones(1), tol=tol,
        recipe=("chi = chi_strat(z) * rho(seed 1), eps = 1e-3, B = T^4 (seed 2), "
                "periodic x/y, thermal bottom, vacuum top"))


def uniform_box(n: int, chi: float, eps: float, B: float, n_mu: int = 4, nf: int = 1,
                bc=PERIODIC, nz: int | None = None) -> Problem:
    """Homogeneous box, every face the same boundary type (small tests)."""
    nz = n if nz is None else nz
    shape = (nf, nz, n, n)
    return Problem(name=f"uniform_{n}x{n}x{nz}", nx=n, ny=n, nz=nz, n_mu=n_mu,
                   chi=np.full(shape, float(chi)), eps=np.full(shape, float(eps)),
                   B=np.full(shape, float(B)), freq_w=np.ones(nf),
                   bc_lo=(bc, bc, bc), bc_hi=(bc, bc, bc))


def random_box(nx: int, ny: int, nz: int, seed: int, n_mu: int = 4, nf: int = 1,
               bc_lo=(PERIODIC, PERIODIC, THERMAL), bc_hi=(PERIODIC, PERIODIC, VACUUM),
               chi_range=(1e-3, 3.0), eps_range=(1e-2, 1.0)) -> Problem:
    """Log-uniform random opacity, epsilon and B on an arbitrary (ragged) grid."""
    rng = np.random.default_rng(seed)
    shape = (nf, nz, ny, nx)
    lo, hi = np.log(chi_range[0]), np.log(chi_range[1])
    chi = np.exp(rng.uniform(lo, hi, shape))
    elo, ehi = np.log(eps_range[0]), np.log(eps_range[1])
    eps = np.exp(rng.uniform(elo, ehi, shape))
    B = rng.uniform(0.5, 2.0, shape)
    return Problem(name=f"random_{nx}x{ny}x{nz}_s{seed}", nx=nx, ny=ny, nz=nz, n_mu=n_mu,
                   chi=chi, eps=eps, B=B, freq_w=np.full(nf, 1.0 / nf), bc_lo=tuple(bc_lo),
                   bc_hi=tuple(bc_hi))


def build_request(d: dict, tol: float = 1e-6) -> Problem:
    """The transfer problem of one ``serving_stream`` descriptor.

    3D sizes: the turbulent box's fields (density and temperature from the
    request's seed), box optical depth 30, fully periodic; ``nf`` bins with
    chi_nu = chi (1 + nu/nf) and B_nu = T^4 (1 + nu/nf)^-1, eps the request's
    value everywhere.  2D (512 x 512 x 1): a y-stratified atmosphere (the
    stratified optical-depth profile along y), x periodic, I = B below, vacuum
    above, T from the request's seed on the plane."""
    nx, ny, nz = d["shape"]
    nf, eps0, seed = int(d["nf"]), float(d["eps"]), int(d["seed"])
    if nz > 1:
        n = max(nx, ny, nz)   # fields of the enclosing cube, cut to the grid
        rho, T = _turbulent_fields(n, seed, seed + 1)
        rho, T = rho[:nz, :ny, :nx], T[:nz, :ny, :nx]
        chi0 = rho * (0.1 * rho * T ** (-3.5) + 0.9)
        chi0 = chi0 * (30.0 / (chi0.mean() * n))
        bc_lo = bc_hi = (PERIODIC, PERIODIC, PERIODIC)
    else:
        prof, _ = stratified_profile(ny)
        rng = np.random.default_rng(seed)
        T = np.exp(0.1 * rng.standard_normal((1, ny, nx)))
        chi0 = np.broadcast_to(prof[None, :, None], (1, ny, nx)) * T ** (-1.0)
        bc_lo, bc_hi = (PERIODIC, THERMAL, PERIODIC), (PERIODIC, VACUUM, PERIODIC)
    shape = (nf, nz, ny, nx)
    scale = 1.0 + np.arange(nf, dtype=np.float64) / nf
    chi = np.ascontiguousarray(np.broadcast_to(chi0.reshape((1, nz, ny, nx)), shape) * scale[:, None, None, None])
    B = np.ascontiguousarray(np.broadcast_to((T ** 4).reshape((1, nz, ny, nx)), shape) / scale[:, None, None, None])
    return Problem(name=f"request_{seed}_{nx}x{ny}x{nz}_nf{nf}_lq{d['n_mu']}", nx=nx, ny=ny, nz=nz,
                   n_mu=int(d["n_mu"]), chi=chi, eps=np.full(shape, eps0), B=B,
                   freq_w=np.full(nf, 1.0 / nf), bc_lo=bc_lo, bc_hi=bc_hi, tol=tol,
                   recipe="serving request: turbulent fields (3D) or y-stratified plane (2D), see build_request")


def serving_stream(n_requests: int = 1024, seed: int = 7, rate: float = 1.0):
    """Request descriptors for a mixed-size request stream (Poisson arrivals).

    Returns a list of dicts with ``t_arrival``, ``shape``, ``nf``, ``n_mu`` and
    ``eps`` and ``seed``; fields are built on demand with ``build_request``.
    """
    rng = np.random.default_rng(seed)
    sizes = [(32, 32, 32), (48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 128, 128), (512, 512, 1)]
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    out = []
    for i in range(n_requests):
        out.append(dict(t_arrival=float(t[i]), shape=sizes[int(rng.integers(len(sizes)))],
                        nf=int(rng.choice([1, 4, 16])), n_mu=int(rng.choice([4, 6, 8])),
                        eps=float(10 ** rng.uniform(-4, 0)), seed=1000 + i))
    return out
