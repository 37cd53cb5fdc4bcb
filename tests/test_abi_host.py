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
                                    (dict(dim=2, n=7, precision=5), "precision"),
                                    (dict(dim=2, n=7, band_min_n=-1), "band_min_n"),
                                    (dict(dim=2, n=7, disc=2, precision=1), "FP64"),
                                    (dict(dim=2, n=7, gamma=3), "gamma"),
                                    (dict(dim=2, n=16383, gamma=2, nu=16), "noise slots")])
def test_create_rejects_bad_config(lib, kw, msg):
    nu = kw.get("nu", 1)
    cfg = mgmc.mgmc_config(kw.get("dim", 2), kw.get("n", 7), kw.get("n_levels", 0), nu, nu, kw.get("precision", 0), 1,
                           0)
    cfg.band_min_n = kw.get("band_min_n", 0)
    cfg.disc = kw.get("disc", 0)
    cfg.gamma = kw.get("gamma", 0)
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


@pytest.mark.parametrize("dim,n,disc,scale_hd,var", [(2, 15, 0, 1, True), (2, 7, 0, 0, False), (3, 7, 0, 1, True),
                                                     (2, 15, 1, 1, False), (2, 7, 1, 0, False), (3, 7, 1, 1, False),
                                                     (2, 1, 2, 1, False), (2, 15, 2, 1, False), (2, 31, 2, 0, False)])
def test_fine_operator_matches_oracle(lib, dim, n, disc, scale_hd, var):
    """mgmc_fine_operator (host only) returns the oracle's finest stencil (FD, Q1 and the
    13-point squared shifted Laplacian, assembled there as a stencil product)."""
    import oracle
    p = inputs.make_problem("op", dim, n, kappa2_seed=4 if var else None, kappa2_const=37.0, scale_hd=scale_hd,
                            disc=disc)
    got = mgmc.mgmc_fine_operator(p)
    o = oracle.Oracle(dim, n, 1, kappa2=p.kappa2, kappa2_const=37.0, scale_hd=scale_hd, disc=disc)
    ref = o.stencil(0)
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def test_fine_operator_rejects_bad_input(lib):
    p = inputs.make_problem("op", 2, 7, kappa2_seed=4)
    p.disc = 1
    with pytest.raises(mgmc.MGMCError):
        mgmc.mgmc_fine_operator(p)
    p = inputs.make_problem("op", 2, 7)
    p.n = 8
    with pytest.raises(mgmc.MGMCError):
        mgmc.mgmc_fine_operator(p)
    p = inputs.make_problem("op", 3, 7)
    p.disc = 2
    with pytest.raises(mgmc.MGMCError):
        mgmc.mgmc_fine_operator(p)
