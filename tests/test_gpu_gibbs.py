"""The plain Gibbs sampler (mgmc_config.gibbs = 1, Sec. 5.1.3) on the GPU against the
oracle's Gibbs sampler, per site, with the tolerances of the MGMC parity tests."""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs
from tests.test_gpu_parity import TOL32, _check32, _check64, _orc, _run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _gibbs(p, precision="fp64"):
    from paper_2407_12149_gb300.mgmc import Sampler
    return Sampler(p, precision=precision, gibbs=True)


@pytest.mark.parametrize("dim,n,m", [(2, 63, 8), (2, 127, 0), (3, 15, 4), (3, 31, 12)])
def test_fp64_gibbs_parity(torch_mod, dim, n, m):
    p = inputs.make_problem("t", dim, n, kappa2_seed=13, m=m, obs_seed=9, qoi_cells=(n + 1) // 4)
    o = _orc(p)
    s = _gibbs(p)
    xo, qo = o.sample(15, 555, gibbs=True)
    xg, qg = _run_gpu(torch_mod, s, p, 15, 555)
    _check64(xg, xo)
    _check64(qg, qo)
    s.close()


@pytest.mark.parametrize("dim,n,m", [(2, 255, 16), (3, 31, 16)])
def test_fp32_gibbs_parity_after_100_steps(torch_mod, dim, n, m):
    p = inputs.make_problem("t", dim, n, kappa2_seed=7, m=m, obs_seed=2, qoi_cells=(n + 1) // 4)
    o = _orc(p)
    s = _gibbs(p, "fp32")
    xo, qo = o.sample(100, 4321, gibbs=True)
    xg, qg = _run_gpu(torch_mod, s, p, 100, 4321)
    _check32(xg, xo)
    assert np.abs(qg - qo).max() <= TOL32 * np.sqrt(np.mean(xo ** 2))
    s.close()


def test_gibbs_continues_bit_exactly(torch_mod):
    """Two calls of 4 and 6 steps (step_offset 4) equal one call of 10 steps."""
    torch = torch_mod
    p = inputs.make_problem("t", 2, 63, kappa2_seed=3, m=5, obs_seed=4)
    s = _gibbs(p)
    x1, _ = _run_gpu(torch, s, p, 10, 21)
    xa, _ = _run_gpu(torch, s, p, 4, 21)
    xb, _ = _run_gpu(torch, s, p, 6, 21, x0=xa, step_offset=4)
    assert np.array_equal(x1, xb)
    s.close()


def test_gibbs_rejects_one_grid_and_batches(torch_mod, monkeypatch):
    from paper_2407_12149_gb300 import mgmc as M
    p = inputs.make_problem("t", 2, 31, n_levels=1, kappa2_seed=1, m=2, obs_seed=1)
    with pytest.raises(M.MGMCError):
        _gibbs(p)
    # a batch whose chain configuration asks for the Gibbs sampler
    lib = M.load()

    class AsGibbs:
        def __getattr__(self, name):
            return getattr(lib, name)

        def mgmc_create_batch(self, n, cfgs, *rest):
            for c in range(n):
                cfgs[c].gibbs = 1
            return lib.mgmc_create_batch(n, cfgs, *rest)

    monkeypatch.setattr(M, "load", lambda: AsGibbs())
    q = inputs.make_problem("t", 2, 31, kappa2_seed=1, m=2, obs_seed=1)
    with pytest.raises(M.MGMCError):
        M.BatchSampler([q])
