"""The streaming band kernels of the 9-point Galerkin grids (FP32, stream9.cu).

mgmc_config.band_min_n decides which 9-point grids below the finest run in the
band kernels and which in the shared-memory tile kernels; both evaluate the same
site arithmetic, noise and sums in the same order, so whole cycles agree bit for
bit.  The band path is also compared with the FP64 CPU oracle at the FP32
tolerance, and its bounded waits report MGMC_ERR_TIMEOUT like every other kernel.
"""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs

pytestmark = pytest.mark.gpu

TILES_ONLY = 1 << 20
MGMC_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _orc(p):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const, scale_hd=p.scale_hd,
                         obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                         qoi_w=p.qoi_w)


def _run_batch(torch, ps, band_min_n, steps, seed):
    from paper_2407_12149_gb300.mgmc import BatchSampler
    b = BatchSampler(ps, precision="fp32", coarse_max_n=31, band_min_n=band_min_n)
    xs = b.zeros()
    q = torch.zeros(len(ps) * steps, dtype=torch.float64, device="cuda")
    b.sample(xs, steps, seed, step_offset=3, qoi=q)
    torch.cuda.synchronize()
    b.close()
    return xs, q


def test_band_kernels_equal_tile_kernels_mixed_batch(torch_mod):
    """Grids of 63^2 .. 511^2 below the finest (one to eight bands, ragged last band,
    runs that cross bands and chains), with observations and without."""
    torch = torch_mod
    ps = []
    for c, n in enumerate([127, 255, 511, 1023, 255, 127]):
        m = 0 if c == 4 else 6 + 3 * c
        ps.append(inputs.make_problem(f"s9_{c}", 2, n, kappa2_seed=500 + c, m=m, obs_seed=600 + c,
                                      qoi_cells=(n + 1) // 4))
    xb, qb = _run_batch(torch, ps, 63, 6, 71)
    xt, qt = _run_batch(torch, ps, TILES_ONLY, 6, 71)
    for c in range(len(ps)):
        assert torch.equal(xb[c], xt[c]), f"chain {c}"
    assert torch.equal(qb, qt)


def test_band_kernels_equal_tile_kernels_many_runs_per_cta(torch_mod):
    """Ten 511^2 chains: the 255^2 grids (default threshold) span many strips per CTA."""
    torch = torch_mod
    ps = [inputs.make_problem(f"s9w{c}", 2, 511, kappa2_seed=700 + c, m=8 + c, obs_seed=800 + c, qoi_cells=64)
          for c in range(10)]
    xb, qb = _run_batch(torch, ps, 0, 4, 5)
    xt, qt = _run_batch(torch, ps, TILES_ONLY, 4, 5)
    for c in range(len(ps)):
        assert torch.equal(xb[c], xt[c]), f"chain {c}"
    assert torch.equal(qb, qt)


def test_band_kernels_fp32_parity_after_100_cycles(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import Sampler
    p = inputs.make_problem("s9p", 2, 255, kappa2_seed=9, m=16, obs_seed=3, qoi_cells=64)
    s = Sampler(p, precision="fp32", coarse_max_n=31, band_min_n=63)
    x = s.zeros()
    q = torch.zeros(100, dtype=torch.float64, device="cuda")
    s.sample(x, 100, 2468, qoi=q)
    torch.cuda.synchronize()
    s.close()
    xo, qo = _orc(p).sample(100, 2468)
    rms = np.sqrt(np.mean(xo ** 2))
    assert np.abs(x.double().cpu().numpy() - xo).max() <= 2e-4 * rms
    assert np.abs(q.cpu().numpy() - qo).max() <= 2e-4 * rms


def test_band_kernel_wait_that_gives_up_reports_timeout(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import MGMCError, Sampler
    p = inputs.make_problem("s9t", 2, 255, kappa2_seed=4, m=8, obs_seed=5, qoi_cells=24)
    s = Sampler(p, precision="fp32", coarse_max_n=31, band_min_n=63)
    s.set_wait_limit(-1)
    with pytest.raises(MGMCError) as e:
        s.sample(s.zeros().cpu(), 2, 7)
    assert e.value.code == MGMC_ERR_TIMEOUT
    s.set_wait_limit(0)
    s.check_status()
    x = s.zeros().cpu()
    s.sample(x, 10, 7)
    s.close()
    xo, _ = _orc(p).sample(10, 7)
    assert np.abs(x.double().numpy() - xo).max() <= 2e-4 * np.sqrt(np.mean(xo ** 2))


def test_coarse_kernel_thread_count_does_not_change_the_states(torch_mod):
    """mgmc_set_coarse_threads (an autotuned launch setting) leaves the arithmetic alone."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    ps = [inputs.make_problem(f"ct{c}", 2, n, kappa2_seed=900 + c, m=8, obs_seed=910 + c, qoi_cells=16)
          for c, n in enumerate([127, 255, 127, 63])]
    out = []
    for threads in (0, 128, 256, 1024):
        b = BatchSampler(ps, precision="fp32", coarse_threads=threads)
        xs = b.zeros()
        q = torch.zeros(len(ps) * 5, dtype=torch.float64, device="cuda")
        b.sample(xs, 5, 13, qoi=q)
        torch.cuda.synchronize()
        out.append((xs, q))
        b.close()
    for xs, q in out[1:]:
        assert all(torch.equal(a, c) for a, c in zip(xs, out[0][0]))
        assert torch.equal(q, out[0][1])
