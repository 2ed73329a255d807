"""Thin Python binding of the C ABI in ``include/rt_sc.h`` (argument marshalling only).

Arrays may be NumPy (host memory, ``on_device = 0``) or CUDA ``torch`` tensors
(device memory on the grid's device, ``on_device = 1``, run on torch's current
stream).  Outputs come back in the kind of memory the inputs were in.  Every
computation happens in the CUDA library; if ``librtsc.so`` is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PERIODIC, VACUUM, THERMAL, FIXED, EXTERNAL = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1
HEAT_INTEGRAL, HEAT_DIFFERENTIAL, HEAT_SWITCH = 0, 1, 2
INTERP_LINEAR, INTERP_QUADRATIC = 1, 2
ITER_JACOBI, ITER_GAUSS_SEIDEL = 0, 1

RT_OK = 0
RT_ERR_ARG = -1
RT_ERR_OOM = -2
RT_ERR_CUDA = -3
RT_ERR_NOT_CONVERGED = -4
RT_ERR_TIMEOUT = -5
RT_ERR_STATE = -6


class rt_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("n_mu", ctypes.c_int), ("nfreq", ctypes.c_int),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("prec", ctypes.c_int)]


class rt_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class rt_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("resid", ctypes.c_double), ("sweep_ms", ctypes.c_double),
                ("sweep_launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("updates", ctypes.c_longlong),
                ("graph_launches", ctypes.c_longlong), ("first_fp64", ctypes.c_int),
                ("fp64_anchors", ctypes.c_int), ("shared_launches", ctypes.c_longlong)]


class rt_server_opts(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_longlong), ("workers", ctypes.c_int), ("shared_cluster", ctypes.c_int)]


class rt_request(ctypes.Structure):
    _fields_ = [("desc", rt_grid_desc), ("interp", ctypes.c_int), ("chi", ctypes.c_void_p),
                ("eps", ctypes.c_void_p), ("B", ctypes.c_void_p), ("freq_w", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("iteration", ctypes.c_int)]


class rt_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("resid", ctypes.c_double), ("queue_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("footprint", ctypes.c_longlong)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


class RTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rt status {status}: {msg}")
        self.status = status


# symbol -> (restype, argtypes); mirrors include/rt_sc.h
_VP = ctypes.c_void_p
_SIGS = {
    "rt_create_grid": (ctypes.c_int, [ctypes.POINTER(rt_grid_desc), ctypes.POINTER(_VP)]),
    "rt_destroy_grid": (ctypes.c_int, [_VP]),
    "rt_num_angles": (ctypes.c_int, [_VP]),
    "rt_get_angles": (ctypes.c_int, [_VP, _VP, _VP]),
    "rt_set_opacity_source": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rt_set_boundary_intensity": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "rt_formal_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts)]),
    "rt_ali_solve": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "rt_moments": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int,
                                  ctypes.POINTER(rt_solve_opts)]),
    "rt_get_S": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts)]),
    "rt_enable_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rt_set_heating_form": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rt_set_interpolation": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rt_set_iteration": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rt_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(rt_stats)]),
    "rt_set_sweep_config": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "rt_get_sweep_plan": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "rt_autotune": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "rt_angle_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "rt_formal_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(rt_grid_desc), _VP, _VP, _VP, _VP, _VP]),
    "rt_grid_footprint": (ctypes.c_int, [ctypes.POINTER(rt_grid_desc), ctypes.POINTER(ctypes.c_longlong)]),
    "rt_server_create": (ctypes.c_int, [ctypes.POINTER(rt_server_opts), ctypes.POINTER(_VP)]),
    "rt_server_destroy": (ctypes.c_int, [_VP]),
    "rt_server_shared_launches": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "rt_ali_solve_many": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts), _VP, _VP, _VP]),
    "rt_submit": (ctypes.c_int, [_VP, ctypes.POINTER(rt_request), ctypes.POINTER(ctypes.c_longlong)]),
    "rt_poll": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.POINTER(rt_request_info)]),
    "rt_wait": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(rt_request_info)]),
    "rt_fetch": (ctypes.c_int, [_VP, ctypes.c_longlong, _VP, _VP, _VP]),
    "rt_measure_rates": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rt_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "rt_set_fp64_anchors": (ctypes.c_int, [_VP, ctypes.c_double]),
    "rt_set_fp64_bin_limit": (ctypes.c_int, [_VP, ctypes.c_double]),
    "rt_set_external_face": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int,
                                            ctypes.POINTER(rt_solve_opts)]),
    "rt_get_face_intensity": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int,
                                             ctypes.POINTER(rt_solve_opts)]),
    "rt_ali_begin": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts)]),
    "rt_ali_iterate": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(rt_solve_opts),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "rt_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.lib_path(debug=os.environ.get("RT_SC_DEBUG", "0") == "1")


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: build it with "
                               "paper_1201_2222_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st):
    if st != RT_OK:
        raise RTError(st, load().rt_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch") and hasattr(x, "data_ptr")


def _torch():
    import torch
    return torch


def angle_table(n_mu, two_d=False):
    """The library's angle table (mu [n][3], w [n]) computed on the host."""
    lib = load()
    n = lib.rt_angle_table(n_mu, 1 if two_d else 0, None, None)
    if n < 0:
        _check(n)
    mu = np.empty((n, 3))
    w = np.empty(n)
    lib.rt_angle_table(n_mu, 1 if two_d else 0, mu.ctypes.data, w.ctypes.data)
    return mu, w


RATE_NAMES = ("fp32_fma_flops", "fp32x2_fma_flops", "mufu_ex2_per_s", "mufu_rcp_per_s", "fp64_fma_flops")


def measure_rates():
    """Measured arithmetic rates of the current CUDA device (rt_measure_rates)."""
    lib = load()
    out = np.zeros(len(RATE_NAMES))
    _check(lib.rt_measure_rates(out.ctypes.data, len(RATE_NAMES)))
    return dict(zip(RATE_NAMES, (float(x) for x in out)))


NOALLOC_SCRATCH_BYTES = 64 << 20


def formal_solve_noalloc(nx, ny, nz, chi, S, B, J_out, n_mu=4, nfreq=1,
                         bc_lo=(PERIODIC, PERIODIC, THERMAL), bc_hi=(PERIODIC, PERIODIC, VACUUM),
                         dx=1.0, dy=1.0, dz=1.0, prec=MIXED):
    """J = Lambda[S] with no device allocation (see rt_formal_solve_noalloc).

    chi, S, B, J_out: CUDA float64 torch tensors [nf][nz][ny][nx]; runs on torch's
    current stream."""
    lib = load()
    if isinstance(prec, str):
        prec = {"fp64": FP64, "mixed": MIXED}[prec.lower()]
    d = rt_grid_desc(nx, ny, nz, dx, dy, dz, n_mu, nfreq, (ctypes.c_int * 3)(*bc_lo),
                     (ctypes.c_int * 3)(*bc_hi), prec)
    ptr = lambda t: None if t is None else t.data_ptr()
    stream = _torch().cuda.current_stream().cuda_stream
    _check(lib.rt_formal_solve_noalloc(ctypes.byref(d), ptr(chi), ptr(S), ptr(B), ptr(J_out), stream))
    return J_out


class Grid:
    """A transfer problem on the GPU: grid, angle set, medium and solver state."""

    def __init__(self, nx, ny, nz, n_mu=4, nfreq=1, bc_lo=(PERIODIC, PERIODIC, THERMAL),
                 bc_hi=(PERIODIC, PERIODIC, VACUUM), dx=1.0, dy=1.0, dz=1.0, prec=MIXED):
        lib = load()
        if isinstance(prec, str):
            prec = {"fp64": FP64, "mixed": MIXED}[prec.lower()]
        d = rt_grid_desc(nx, ny, nz, dx, dy, dz, n_mu, nfreq, (ctypes.c_int * 3)(*bc_lo),
                         (ctypes.c_int * 3)(*bc_hi), prec)
        h = _VP()
        _check(lib.rt_create_grid(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.shape = (nfreq, nz, ny, nx)
        self.cells = nx * ny * nz
        self.nfreq = nfreq
        self.prec = prec
        self.n_angles = lib.rt_num_angles(h)

    @classmethod
    def from_problem(cls, p, prec=MIXED):
        return cls(p.nx, p.ny, p.nz, p.n_mu, p.nf, p.bc_lo, p.bc_hi, p.dx, p.dy, p.dz, prec)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().rt_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers
    def _in(self, x, n=None):
        """(pointer, on_device, keepalive) for an input array of n float64 values."""
        n = int(np.prod(self.shape)) if n is None else n
        if _is_torch(x):
            torch = _torch()
            if not x.is_cuda:
                x = x.detach().numpy()
            else:
                if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != n:
                    raise ValueError("device inputs must be contiguous float64 with the grid's size")
                return x.data_ptr(), 1, x
        a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        if a.size != n:
            raise ValueError(f"expected {n} values, got {a.size}")
        return a.ctypes.data, 0, a

    def _opts(self, tol=1e-6, max_iter=1000, check_every=0, on_device=False):
        s = None
        if on_device:
            s = _torch().cuda.current_stream().cuda_stream
        return rt_solve_opts(tol, max_iter, check_every, s)

    def _out(self, shape, on_device):
        if on_device:
            torch = _torch()
            return torch.empty(shape, dtype=torch.float64, device="cuda")
        return np.empty(shape, dtype=np.float64)

    @staticmethod
    def _ptr(a):
        return a.data_ptr() if _is_torch(a) else a.ctypes.data

    # -- API
    def angles(self):
        mu = np.empty((self.n_angles, 3))
        w = np.empty(self.n_angles)
        _check(load().rt_get_angles(self._h, mu.ctypes.data, w.ctypes.data))
        return mu, w

    def set_sweep_config(self, angles_per_group=0, cluster_ctas=0, threads=0, variant=0):
        _check(load().rt_set_sweep_config(self._h, angles_per_group, cluster_ctas, threads, variant))

    def autotune(self):
        v = (ctypes.c_int * 7)()
        _check(load().rt_autotune(self._h, v))
        return dict(zip(("variant", "groups", "rays_per_group", "cluster", "threads", "smem", "fp64_bins"),
                        list(v)))

    def sweep_plan(self):
        v = (ctypes.c_int * 7)()
        _check(load().rt_get_sweep_plan(self._h, v))
        return dict(zip(("variant", "groups", "rays_per_group", "cluster", "threads", "smem", "fp64_bins"),
                        list(v)))

    def set_opacity_source(self, chi, eps, B, freq_w=None):
        pc, dc, kc = self._in(chi)
        pe, de, ke = self._in(eps)
        pb, db, kb = self._in(B)
        if len({dc, de, db}) != 1:
            raise ValueError("chi, eps and B must all be host or all be device arrays")
        pw = None
        kw = None
        if freq_w is not None:
            pw, dw, kw = self._in(freq_w, self.nfreq)
            if dw != dc:
                raise ValueError("freq_w must live where chi lives")
        if dc:
            _torch().cuda.current_stream().synchronize()
        _check(load().rt_set_opacity_source(self._h, pc, pe, pb, pw, dc))
        del kc, ke, kb, kw

    def set_boundary_intensity(self, face, I):
        a = np.ascontiguousarray(I, dtype=np.float64).reshape(-1)
        _check(load().rt_set_boundary_intensity(self._h, int(face), a.ctypes.data))

    def formal_solve(self, S=None, want_lstar=False, on_device=None):
        ps, ds, ks = (None, 0, None) if S is None else self._in(S)
        dev = bool(ds) if on_device is None else bool(on_device)
        J = self._out(self.shape, dev)
        L = self._out(self.shape, dev) if want_lstar else None
        o = self._opts(on_device=dev)
        _check(load().rt_formal_solve(self._h, ps, self._ptr(J), None if L is None else self._ptr(L),
                                      1 if dev else 0, ctypes.byref(o)))
        if dev:
            _torch().cuda.current_stream().synchronize()
        return (J, L) if want_lstar else J

    def ali_solve(self, S_init=None, tol=1e-6, max_iter=1000, check_every=0, raise_on_fail=True):
        ps, ds, ks = (None, 0, None) if S_init is None else self._in(S_init)
        o = self._opts(tol, max_iter, check_every, on_device=bool(ds))
        it = ctypes.c_int(0)
        r = ctypes.c_double(0.0)
        st = load().rt_ali_solve(self._h, ps, ds, ctypes.byref(o), ctypes.byref(it), ctypes.byref(r))
        if st != RT_OK and (raise_on_fail or st != RT_ERR_NOT_CONVERGED):
            _check(st)
        return it.value, r.value, st

    def moments(self, on_device=False, want=("J", "H", "K", "f", "Q"), out=None):
        """J, H, K, f = K/J and Q of the last formal solution (rt_moments).

        ``want``: the outputs to return (the others are not copied); ``out``: a dict
        of caller arrays to fill instead of new ones (e.g. pinned host tensors)."""
        nf = self.nfreq
        sp = self.shape[1:]
        shapes = dict(J=(nf,) + sp, H=(nf, 3) + sp, K=(nf, 6) + sp, f=(nf, 6) + sp, Q=sp)
        res = {k: (out[k] if out and k in out else self._out(shapes[k], on_device)) for k in want}
        ptr = lambda k: self._ptr(res[k]) if k in res else None
        o = self._opts(on_device=on_device)
        _check(load().rt_moments(self._h, ptr("J"), ptr("H"), ptr("K"), ptr("f"), ptr("Q"),
                                 1 if on_device else 0, ctypes.byref(o)))
        return res

    def set_external_face(self, side, chi=None, S=None, B=None, I=None):
        """Ghost layer of a subdomain z face (rt_set_external_face): chi, S, B
        [nf][ny][nx] and the rays' incoming intensities I [nf][na][ny][nx] (host)."""
        lay = self.nfreq * self.shape[2] * self.shape[3]
        keep = []
        def ptr(x, n):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
            if a.size != n:
                raise ValueError(f"expected {n} values, got {a.size}")
            keep.append(a)
            return a.ctypes.data
        o = self._opts()
        _check(load().rt_set_external_face(self._h, int(side), ptr(chi, lay), ptr(S, lay), ptr(B, lay),
                                           ptr(I, lay * self.n_angles), 0, ctypes.byref(o)))

    def face_intensity(self, side):
        """Intensities of the last formal solution on the first (0) or last (1) z
        plane, [nf][na][ny][nx] (rt_get_face_intensity)."""
        I = np.empty((self.nfreq, self.n_angles) + self.shape[2:])
        o = self._opts()
        _check(load().rt_get_face_intensity(self._h, int(side), I.ctypes.data, 0, ctypes.byref(o)))
        return I

    def ali_begin(self, S_init=None):
        """Start a Jacobi ALI solve taken one step at a time (rt_ali_begin)."""
        ps, ds, ks = (None, 0, None) if S_init is None else self._in(S_init)
        o = self._opts(on_device=bool(ds))
        _check(load().rt_ali_begin(self._h, ps, ds, ctypes.byref(o)))

    def ali_iterate(self, n=1):
        """n more iterations (rt_ali_iterate): (iterations since begin, last max |dS|/S)."""
        it = ctypes.c_int(0)
        r = ctypes.c_double(0.0)
        o = self._opts()
        _check(load().rt_ali_iterate(self._h, int(n), ctypes.byref(o), ctypes.byref(it), ctypes.byref(r)))
        return it.value, r.value

    def get_S(self, on_device=False):
        S = self._out(self.shape, on_device)
        o = self._opts(on_device=on_device)
        _check(load().rt_get_S(self._h, self._ptr(S), 1 if on_device else 0, ctypes.byref(o)))
        return S

    def set_iteration(self, scheme):
        """ALI scheme: ITER_JACOBI / "jacobi" or ITER_GAUSS_SEIDEL / "gauss_seidel"."""
        if isinstance(scheme, str):
            scheme = {"jacobi": ITER_JACOBI, "gauss_seidel": ITER_GAUSS_SEIDEL}[scheme.lower()]
        _check(load().rt_set_iteration(self._h, int(scheme)))

    def set_fp64_anchors(self, drop):
        """Residual drop between FP64 iterations of mixed Jacobi solves (rt_set_fp64_anchors)."""
        _check(load().rt_set_fp64_anchors(self._h, float(drop)))

    def set_fp64_bin_limit(self, limit):
        """Roundoff/eps limit above which a bin is solved in FP64 (rt_set_fp64_bin_limit);
        applies from the next set_opacity_source."""
        _check(load().rt_set_fp64_bin_limit(self._h, float(limit)))

    def set_wait_limit(self, polls):
        """Polls before a Gauss-Seidel grid-barrier wait gives up (rt_set_wait_limit)."""
        _check(load().rt_set_wait_limit(self._h, int(polls)))

    def set_interpolation(self, order):
        """Face interpolation: INTERP_LINEAR / "linear" or INTERP_QUADRATIC / "quadratic"."""
        if isinstance(order, str):
            order = {"linear": INTERP_LINEAR, "quadratic": INTERP_QUADRATIC}[order.lower()]
        _check(load().rt_set_interpolation(self._h, int(order)))

    def set_heating_form(self, form):
        """Form of Q returned by ``moments``: HEAT_INTEGRAL, HEAT_DIFFERENTIAL or
        HEAT_SWITCH (or their names: "integral", "differential", "switch")."""
        if isinstance(form, str):
            form = {"integral": HEAT_INTEGRAL, "differential": HEAT_DIFFERENTIAL,
                    "switch": HEAT_SWITCH}[form.lower()]
        _check(load().rt_set_heating_form(self._h, int(form)))

    def enable_timing(self, on=True):
        _check(load().rt_enable_timing(self._h, 1 if on else 0))

    def stats(self):
        s = rt_stats()
        _check(load().rt_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in rt_stats._fields_}


def _desc_of(p, prec):
    if isinstance(prec, str):
        prec = {"fp64": FP64, "mixed": MIXED}[prec.lower()]
    return rt_grid_desc(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.n_mu, p.nf, (ctypes.c_int * 3)(*p.bc_lo),
                        (ctypes.c_int * 3)(*p.bc_hi), prec)


def grid_footprint(p, prec=MIXED):
    """Estimated device bytes of a grid for problem ``p`` (rt_grid_footprint)."""
    out = ctypes.c_longlong(0)
    _check(load().rt_grid_footprint(ctypes.byref(_desc_of(p, prec)), ctypes.byref(out)))
    return out.value


def ali_solve_many(grids, tol=1e-6, max_iter=1000, check_every=0, raise_on_fail=True):
    """Jacobi ALI solves of several Grids together, their sweeps merged into shared
    launches (rt_ali_solve_many); returns per grid (iters, resid, status)."""
    n = len(grids)
    hs = (_VP * max(1, n))(*[g._h for g in grids])
    it = (ctypes.c_int * max(1, n))()
    rs = (ctypes.c_double * max(1, n))()
    sts = (ctypes.c_int * max(1, n))()
    o = rt_solve_opts(tol, max_iter, check_every, None)
    st = load().rt_ali_solve_many(ctypes.cast(hs, _VP), n, ctypes.byref(o), ctypes.cast(it, _VP),
                                  ctypes.cast(rs, _VP), ctypes.cast(sts, _VP))
    if st != RT_OK and (raise_on_fail or st != RT_ERR_NOT_CONVERGED):
        _check(st)
    return [(it[i], rs[i], sts[i]) for i in range(n)]


class Server:
    """Request server (rt_server_*): queued ALI solves on worker threads, admitted
    by estimated device footprint; results come back as host arrays."""

    def __init__(self, workers=2, device_bytes=0, shared_cluster=0):
        self._h = _VP()
        opts = rt_server_opts(int(device_bytes), int(workers), int(shared_cluster))
        _check(load().rt_server_create(ctypes.byref(opts), ctypes.byref(self._h)))
        self._shapes = {}
        self._keep = {}

    def close(self):
        if self._h:
            load().rt_server_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, p, prec=MIXED, tol=None, max_iter=1000, interp=INTERP_LINEAR, iteration=ITER_JACOBI):
        """Queue an ALI solve of the workloads.Problem ``p``; returns its id."""
        if isinstance(interp, str):
            interp = {"linear": INTERP_LINEAR, "quadratic": INTERP_QUADRATIC}[interp.lower()]
        if isinstance(iteration, str):
            iteration = {"jacobi": ITER_JACOBI, "gauss_seidel": ITER_GAUSS_SEIDEL}[iteration.lower()]
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.chi, p.eps, p.B, p.freq_w)]
        req = rt_request(_desc_of(p, prec), int(interp), *[a.ctypes.data for a in arrs],
                         float(p.tol if tol is None else tol), int(max_iter), int(iteration))
        rid = ctypes.c_longlong(0)
        _check(load().rt_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        self._shapes[rid.value] = (p.nf, p.nz, p.ny, p.nx)
        return rid.value

    def shared_launches(self):
        """Shared sweep launches issued so far (rt_server_shared_launches)."""
        n = ctypes.c_longlong(0)
        _check(load().rt_server_shared_launches(self._h, ctypes.byref(n)))
        return n.value

    @staticmethod
    def _info(i):
        return {k: getattr(i, k) for k, _ in rt_request_info._fields_}

    def poll(self, rid):
        i = rt_request_info()
        _check(load().rt_poll(self._h, ctypes.c_longlong(rid), ctypes.byref(i)))
        return self._info(i)

    def wait(self, rid, timeout=600.0):
        """Info once the request is done; raises RTError(RT_ERR_TIMEOUT) after ``timeout`` s."""
        i = rt_request_info()
        _check(load().rt_wait(self._h, ctypes.c_longlong(rid), float(timeout), ctypes.byref(i)))
        return self._info(i)

    def fetch(self, rid, raise_on_fail=True):
        """(J, S, Q) host arrays of a finished request, and its status."""
        nf, nz, ny, nx = self._shapes.pop(rid)
        J = np.empty((nf, nz, ny, nx))
        S = np.empty_like(J)
        Q = np.empty((nz, ny, nx))
        st = load().rt_fetch(self._h, ctypes.c_longlong(rid), J.ctypes.data, S.ctypes.data, Q.ctypes.data)
        if st != RT_OK and (raise_on_fail or st not in (RT_ERR_NOT_CONVERGED,)):
            _check(st)
        return J, S, Q, st
