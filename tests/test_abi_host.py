"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol include/mgmc.h declares; host-only helpers and argument validation
(no kernel is launched by these tests)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2407_12149_gb300 import build, inputs, mgmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mgmc.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mgmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgmc_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "mgmc_create" in declared and "mgmc_sample" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(mgmc.EXPORTS)


def test_point_obs_rows_match_input_generator(lib):
    for dim, n in ((2, 31), (2, 1023), (3, 15)):
        xyz = inputs.obs_locations(20, dim, 3)
        s1, w1 = inputs.point_obs_rows(n, dim, xyz)
        s2, w2 = mgmc.mgmc_point_obs_rows(dim, n, xyz)
        assert np.array_equal(s1, s2)
        assert np.array_equal(w1, w2)


def test_point_obs_rows_rejects_outside_points(lib):
    with pytest.raises(mgmc.MGMCError) as e:
        mgmc.mgmc_point_obs_rows(2, 15, np.array([[0.5, 1.5]]))
    assert e.value.code == 1


@pytest.mark.parametrize("kw,msg", [(dict(dim=4, n=7), "dim"), (dict(dim=2, n=30), "2^k - 1"),
                                    (dict(dim=2, n=7, n_levels=9), "n_levels"),
                                    (dict(dim=2, n=7, precision=5), "precision")])
def test_create_rejects_bad_config(lib, kw, msg):
    cfg = mgmc.mgmc_config(kw.get("dim", 2), kw.get("n", 7), kw.get("n_levels", 0), 1, 1, kw.get("precision", 0), 1, 0)
    h = ctypes.c_void_p()
    rc = lib.mgmc_create(ctypes.byref(cfg), None, None, None, 10.0, 0, None, None, 1, None, None, 0, None, None,
                         ctypes.byref(h))
    assert rc == 1
    assert msg in lib.mgmc_last_error().decode()
    assert not h.value


def test_create_rejects_too_many_observations(lib):
    cfg = mgmc.mgmc_config(2, 7, 0, 1, 1, 0, 1, 0)
    h = ctypes.c_void_p()
    rc = lib.mgmc_create(ctypes.byref(cfg), None, None, None, 10.0, mgmc.MGMC_MAX_OBS + 1, None, None, 1, None, None,
                         0, None, None, ctypes.byref(h))
    assert rc == 1


def test_sample_rejects_null_handle(lib):
    rc = lib.mgmc_sample(None, 1, 0, 0, 0, None, None, None)
    assert rc == 1


def test_stats_rejects_short_series(lib):
    out = mgmc.mgmc_stats()
    assert lib.mgmc_qoi_stats(None, 10, 0, 1.5, ctypes.byref(out), None) == 1
