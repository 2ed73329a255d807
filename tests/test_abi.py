"""The C-ABI library loads without a GPU and exports every entry point of include/*.h.

No compute call is made here except the host-only angle table, which is compared
with the oracle's quadrature (both follow Sec. 3.2; they share no code).
"""
import glob
import os
import re

import numpy as np
import pytest

from paper_1201_2222_gb300 import build as B
from paper_1201_2222_gb300 import rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(rt_[A-Za-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rt.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(rt._SIGS), "binding signatures must mirror the header"


def test_angle_table_matches_oracle(lib):
    from oracle.quadrature import level_symmetric
    for n_mu in (2, 4, 6, 8, 10, 12):
        for two_d in (False, True):
            m1, w1 = rt.angle_table(n_mu, two_d)
            m2, w2 = level_symmetric(n_mu, two_d)
            np.testing.assert_allclose(m1, m2, atol=5e-14)
            np.testing.assert_allclose(w1, w2, atol=5e-15)


def test_bad_angle_count_is_an_error(lib):
    assert lib.rt_angle_table(5, 0, None, None) == rt.RT_ERR_ARG
    assert lib.rt_angle_table(14, 0, None, None) == rt.RT_ERR_ARG
    assert b"n_mu" in lib.rt_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(rt, "_lib", None)
    monkeypatch.setattr(B, "lib_path", lambda debug=False: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        rt.load()


def test_grid_footprint_is_host_only_and_grows_with_the_problem():
    from paper_1201_2222_gb300 import rt, workloads as W
    small = rt.grid_footprint(W.random_box(8, 8, 8, seed=1, n_mu=4))
    big = rt.grid_footprint(W.random_box(16, 16, 16, seed=1, n_mu=4))
    more_rays = rt.grid_footprint(W.random_box(8, 8, 8, seed=1, n_mu=8))
    fp64 = rt.grid_footprint(W.random_box(8, 8, 8, seed=1, n_mu=4), prec="fp64")
    assert 0 < small < more_rays
    # a mixed grid also holds the internal FP64 grid of its FP64 iterations
    assert 0.5 * fp64 < small < 2 * fp64
    assert 6 * small < big < 9 * small      # cells x 8, faces (ghosts) x 4


def test_grid_footprint_rejects_bad_descriptions():
    import dataclasses
    from paper_1201_2222_gb300 import rt, workloads as W
    p = W.random_box(4, 4, 4, seed=1, n_mu=4)
    with pytest.raises(rt.RTError):
        rt.grid_footprint(dataclasses.replace(p, n_mu=5))
    with pytest.raises(rt.RTError):
        rt.grid_footprint(dataclasses.replace(p, nx=0))
