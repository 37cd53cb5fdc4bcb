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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_persistent_tiles_span_chains(torch_mod, precision):
    """A batch with many more tiles than resident CTAs (each CTA walks a range of
    tiles across chain boundaries, with staged copies of the next tile in flight)
    equals the solo runs bit for bit."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler, Sampler
    ps = [inputs.make_problem(f"w{c}", 2, 511, kappa2_seed=300 + c, m=8 + c, obs_seed=400 + c, qoi_cells=64)
          for c in range(10)]
    b = BatchSampler(ps, precision=precision)
    xs = b.zeros()
    b.sample(xs, 3, 17, step_offset=2)
    torch.cuda.synchronize()
    for c in (0, 4, 9):
        s = Sampler(ps[c], precision=precision, coarse_max_n=31)
        x = s.zeros()
        s.sample(x, 3, 17, step_offset=2, chain=c)
        torch.cuda.synchronize()
        assert torch.equal(x, xs[c]), f"chain {c}"
        s.close()


def test_fp32_batch_with_galerkin_tiles_matches_oracle(torch_mod):
    """FP32 batched chains whose 9-point grids 127^2 and 63^2 run in tile kernels,
    per site against the FP64 oracle after 60 cycles (tolerance 2e-4 of the RMS)."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    ps = [inputs.make_problem(f"g{c}", 2, 255, kappa2_seed=500 + c, m=12, obs_seed=600 + c, qoi_cells=64)
          for c in range(2)]
    b = BatchSampler(ps, precision="fp32")
    xs = b.zeros()
    b.sample(xs, 60, 23)
    torch.cuda.synchronize()
    for c, p in enumerate(ps):
        o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w,
                          Gamma=p.Gamma, y=p.y)
        xo = o.sample(60, 23, chain=c, qoi=False)
        xg = xs[c].cpu().numpy().astype(np.float64)
        rms = np.sqrt(np.mean(xo ** 2))
        assert np.abs(xg - xo).max() <= 2e-4 * rms, f"chain {c}"


def test_resume_and_get_state_reproduce_one_run(torch_mod):
    """x = None continues from the held state: split runs equal one run bit for bit."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler, Sampler
    ps = _problems()[:4]
    b1, b2 = BatchSampler(ps, precision="fp32"), BatchSampler(ps, precision="fp32")
    xa, xb = b1.zeros(), b2.zeros()
    qa = torch.zeros(len(ps) * 5, dtype=torch.float64, device="cuda")
    b1.sample(xa, 5, 9, step_offset=3, qoi=qa)
    b2.sample(xb, 2, 9, step_offset=3)
    qb = torch.zeros(len(ps) * 3, dtype=torch.float64, device="cuda")
    b2.sample(None, 3, 9, step_offset=5, qoi=qb)
    for c, p in enumerate(ps):
        got = torch.empty(p.N, dtype=torch.float32, device="cuda")
        b2.get_state(c, got)
        torch.cuda.synchronize()
        assert torch.equal(got, xa[c]), f"chain {c}"
        assert torch.equal(qb[c * 3:(c + 1) * 3], qa[c * 5 + 2:(c + 1) * 5]), f"chain {c} qoi"
        host = torch.empty(p.N, dtype=torch.float32)
        b2.get_state(c, host)
        assert torch.equal(host, xa[c].cpu())
    # single-chain handle
    p = ps[1]
    s1, s2 = Sampler(p, precision="fp64"), Sampler(p, precision="fp64")
    x1, x2 = s1.zeros(), s2.zeros()
    s1.sample(x1, 4, 5, chain=2)
    s2.sample(x2, 1, 5, chain=2)
    s2.sample(None, 3, 5, step_offset=1, chain=2)
    y = torch.empty_like(x1)
    s2.get_state(y)
    torch.cuda.synchronize()
    assert torch.equal(y, x1)


@pytest.mark.parametrize("precision,m", [("fp64", 40), ("fp64", 16), ("fp32", 40)])
def test_uniform_batch_low_rank_tails_match_oracle(torch_mod, precision, m):
    """Chains of one size get CTA groups of their own in the tile launches; the
    low-rank step after each sweep (Alg. 3) takes its register form at m = 16 and
    its general form at m = 40."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    ps = [inputs.make_problem(f"u{c}", 2, 127, kappa2_seed=700 + c, m=m, obs_seed=800 + c, qoi_cells=32)
          for c in range(3)]
    b = BatchSampler(ps, precision=precision)
    xs = b.zeros()
    n_steps = 6 if precision == "fp64" else 40
    b.sample(xs, n_steps, 41)
    torch.cuda.synchronize()
    for c, p in enumerate(ps):
        o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w,
                          Gamma=p.Gamma, y=p.y)
        xo = o.sample(n_steps, 41, chain=c, qoi=False)
        xg = xs[c].cpu().numpy().astype(np.float64)
        rms = np.sqrt(np.mean(xo ** 2))
        if precision == "fp64":
            assert np.all(np.abs(xg - xo) <= 1e-11 * np.maximum(np.abs(xo), rms)), f"chain {c}"
        else:
            assert np.abs(xg - xo).max() <= 2e-4 * rms, f"chain {c}"
