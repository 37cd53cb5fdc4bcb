"""The allocation-free statistics entry point against the allocating one.

mgmc_qoi_stats_noalloc serves callers that cannot allocate device memory while
they run (a device whose memory another framework's pool holds, or a loop that
must not wait on an allocator); it keeps its scratch in one fixed array inside
the library.  This file is collected last so that a stop at the first failure
has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _series(seed, n, phi):
    from scipy.signal import lfilter
    e = np.random.default_rng(seed).normal(size=n)
    return 0.3 + lfilter([np.sqrt(1 - phi * phi)], [1.0, -phi], e)


def test_noalloc_stats_match_allocating_entry_point_twice():
    import torch
    from paper_2407_12149_gb300 import build, mgmc
    build.build()
    L = mgmc.load()
    for call, (seed, n, burn, phi) in enumerate([(1, 20000, 100, 0.6), (2, 4001, 0, 0.2)]):
        q = torch.tensor(_series(seed, n, phi), dtype=torch.float64, device="cuda")
        ref = mgmc.mgmc_stats()
        got = mgmc.mgmc_stats()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert L.mgmc_qoi_stats(ctypes.c_void_p(q.data_ptr()), n, burn, 1.5, ctypes.byref(ref), stream) == 0
        assert L.mgmc_qoi_stats_noalloc(ctypes.c_void_p(q.data_ptr()), n, burn, 1.5, ctypes.byref(got),
                                        stream) == 0, f"call {call}"
        for k in ("mean", "var", "tau_int", "tau_err", "ess"):
            assert getattr(got, k) == pytest.approx(getattr(ref, k), rel=1e-10, abs=1e-14), (call, k)
        assert got.window == ref.window and got.n_used == ref.n_used == n - burn


def test_noalloc_stats_reject_series_beyond_the_limit():
    from paper_2407_12149_gb300 import build, mgmc
    build.build()
    L = mgmc.load()
    out = mgmc.mgmc_stats()
    n = mgmc.MGMC_NOALLOC_MAX_SERIES + 2
    assert L.mgmc_qoi_stats_noalloc(ctypes.c_void_p(1 << 20), n, 0, 1.5, ctypes.byref(out), None) == 1
    assert b"MGMC_NOALLOC_MAX_SERIES" in L.mgmc_last_error()
