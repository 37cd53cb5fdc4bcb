"""Batched chains (mgmc_create_batch / mgmc_sample_batch) against solo runs and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _problems():
    ps = []
    for c, n in enumerate([63, 127, 255, 63, 127, 255, 511]):
        m = 0 if c == 3 else 8 + 4 * (c % 3)
        ps.append(inputs.make_problem(f"b{c}", 2, n, kappa2_seed=100 + c, m=m, obs_seed=200 + c,
                                      qoi_cells=(n + 1) // 4))
    return ps


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_chains_equal_solo_runs(torch_mod, precision):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler, Sampler
    ps = _problems()
    b = BatchSampler(ps, precision=precision)
    xs = b.zeros()
    n_steps = 7
    q = torch.zeros(len(ps) * n_steps, dtype=torch.float64, device="cuda")
    b.sample(xs, n_steps, 31, step_offset=5, qoi=q)
    torch.cuda.synchronize()
    for c, p in enumerate(ps):
        s = Sampler(p, precision=precision, coarse_max_n=31)
        x = s.zeros()
        qs = torch.zeros(n_steps, dtype=torch.float64, device="cuda")
        s.sample(x, n_steps, 31, step_offset=5, chain=c, qoi=qs)
        torch.cuda.synchronize()
        assert torch.equal(x, xs[c]), f"chain {c}"
        assert torch.equal(qs, q[c * n_steps:(c + 1) * n_steps]), f"chain {c} qoi"
        s.close()


def test_batch_chain_matches_oracle(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    ps = _problems()[:3]
    b = BatchSampler(ps, precision="fp64")
    xs = b.zeros()
    b.sample(xs, 4, 77)
    torch.cuda.synchronize()
    for c, p in enumerate(ps):
        o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w,
                          Gamma=p.Gamma, y=p.y)
        xo = o.sample(4, 77, chain=c, qoi=False)
        xg = xs[c].cpu().numpy()
        rms = np.sqrt(np.mean(xo ** 2))
        assert np.all(np.abs(xg - xo) <= 1e-11 * np.maximum(np.abs(xo), rms))
