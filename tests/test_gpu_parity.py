"""GPU parity of the CUDA sampler (through the C ABI) against the FP64 CPU oracle.

Tolerances (per site i, after the stated number of V-cycles, same seed and
Philox counters on both sides):
  FP64 path: |x_gpu - x_orc|_i <= 1e-11 * max(|x_orc,i|, rms(x_orc))
  FP32 path: |x_gpu - x_orc|_i <= 2e-4 * rms(x_orc)
"""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 2e-4


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


def _gpu(p, precision="fp64", **kw):
    from paper_2407_12149_gb300.mgmc import Sampler
    return Sampler(p, precision=precision, **kw)


def _run_gpu(torch, s, p, n_steps, seed, x0=None, step_offset=0, chain=0):
    x = s.zeros()
    if x0 is not None:
        x.copy_(torch.as_tensor(x0, dtype=x.dtype))
    q = torch.zeros(max(n_steps, 1), dtype=torch.float64, device=x.device)
    s.sample(x, n_steps, seed, step_offset=step_offset, chain=chain, qoi=q)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), q[:n_steps].cpu().numpy()


def _check64(xg, xo, tol=TOL64):
    rms = np.sqrt(np.mean(xo ** 2))
    bound = tol * np.maximum(np.abs(xo), rms)
    err = np.abs(xg - xo)
    assert np.all(err <= bound), f"max rel err {np.max(err / np.maximum(np.abs(xo), rms)):.3e}"


def _check32(xg, xo, tol=TOL32):
    rms = np.sqrt(np.mean(xo ** 2))
    err = np.abs(xg - xo).max()
    assert err <= tol * rms, f"max err / rms = {err / rms:.3e}"


@pytest.mark.parametrize("coarse_max_n", [0, 3])
def test_fp64_config1_parity(torch_mod, coarse_max_n):
    """Plain 31^2 problem, kappa^2 = 10, 4 grids, seed 1234, x0 = 0."""
    p = inputs.config1()
    o = _orc(p)
    s = _gpu(p, coarse_max_n=coarse_max_n)
    for n_steps in (1, 7, 300):
        xo, qo = o.sample(n_steps, 1234)
        xg, qg = _run_gpu(torch_mod, s, p, n_steps, 1234)
        _check64(xg, xo)
        _check64(qg, qo)


@pytest.mark.parametrize("dim,n,m,coarse_max_n", [(2, 63, 8, 0), (2, 127, 16, 7), (2, 63, 5, 1), (3, 15, 8, 0),
                                                  (3, 31, 12, 3), (3, 15, 4, 1)])
def test_fp64_bayes_parity(torch_mod, dim, n, m, coarse_max_n):
    p = inputs.make_problem("t", dim, n, kappa2_seed=11, m=m, obs_seed=5, qoi_cells=(n + 1) // 4)
    o = _orc(p)
    s = _gpu(p, coarse_max_n=coarse_max_n)
    xo, qo = o.sample(12, 99)
    xg, qg = _run_gpu(torch_mod, s, p, 12, 99)
    _check64(xg, xo)
    _check64(qg, qo)


@pytest.mark.parametrize("dim,n,m,coarse_max_n", [(2, 127, 16, 0), (2, 255, 16, 7), (3, 31, 16, 3)])
def test_fp32_parity_after_100_cycles(torch_mod, dim, n, m, coarse_max_n):
    p = inputs.make_problem("t", dim, n, kappa2_seed=7, m=m, obs_seed=2, qoi_cells=(n + 1) // 4)
    o = _orc(p)
    s = _gpu(p, precision="fp32", coarse_max_n=coarse_max_n)
    xo, qo = o.sample(100, 4321)
    xg, qg = _run_gpu(torch_mod, s, p, 100, 4321)
    _check32(xg, xo)
    assert np.abs(qg - qo).max() <= TOL32 * np.sqrt(np.mean(xo ** 2))


def test_config2_full_size_parity(torch_mod):
    """1023^2, non-stationary kappa^2, 16 observations, 10 grids, in the launch
    configuration the benchmark times (FP32), plus the FP64 path."""
    p = inputs.config2()
    o = _orc(p)
    xo, qo = o.sample(3, 2024)
    for prec, chk in (("fp64", _check64), ("fp32", _check32)):
        s = _gpu(p, precision=prec)
        xg, qg = _run_gpu(torch_mod, s, p, 3, 2024)
        chk(xg, xo)
        s.close()


def test_config3_full_size_parity(torch_mod):
    """127^3, kappa^2 = 25, 32 observations, coarsest 3^3 (6 grids), FP32 and FP64."""
    p = inputs.config3()
    o = _orc(p)
    xo, qo = o.sample(2, 77)
    for prec, chk in (("fp64", _check64), ("fp32", _check32)):
        s = _gpu(p, precision=prec)
        xg, qg = _run_gpu(torch_mod, s, p, 2, 77)
        chk(xg, xo)
        s.close()


def test_config2_fp32_after_100_cycles_single_chain_and_batch_chain(torch_mod):
    """The tolerance as stated for the FP32 path (2e-4 of the field RMS after 100
    V-cycles) on the benchmarked problem (1023^2, 16 observations, 10 grids): one
    chain, and chain 5 of a batch of 32 chains of it (the benchmark's launch
    configuration); both use Philox chain id 5, so one oracle run serves both."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    p = inputs.config2()
    xo, qo = _orc(p).sample(100, 31, chain=5)
    rms = np.sqrt(np.mean(xo ** 2))
    s = _gpu(p, precision="fp32")
    xg, qg = _run_gpu(torch, s, p, 100, 31, chain=5)
    s.close()
    _check32(xg, xo)
    assert np.abs(qg - qo).max() <= TOL32 * rms
    b = BatchSampler([p] * 32, precision="fp32")
    xs = b.zeros()
    q = torch.zeros(32 * 100, dtype=torch.float64, device="cuda")
    b.sample(xs, 100, 31, qoi=q)
    torch.cuda.synchronize()
    _check32(xs[5].double().cpu().numpy(), xo)
    assert np.abs(q[5 * 100:6 * 100].cpu().numpy() - qo).max() <= TOL32 * rms
    b.close()


@pytest.mark.slow
def test_config3_fp32_after_100_cycles(torch_mod):
    """127^3, kappa^2 = 25, 32 observations, coarsest 3^3: FP32 after 100 V-cycles
    (the oracle needs about 2.8 s per cycle here)."""
    p = inputs.config3()
    xo, qo = _orc(p).sample(100, 55)
    s = _gpu(p, precision="fp32")
    xg, qg = _run_gpu(torch_mod, s, p, 100, 55)
    s.close()
    _check32(xg, xo)
    assert np.abs(qg - qo).max() <= TOL32 * np.sqrt(np.mean(xo ** 2))


def test_config1_fp64_parity_over_10000_cycles(torch_mod):
    """Config 1 (31^2, 4 grids, seed 1234, x0 = 0): every site within 1e-11 after
    10^4 V-cycles, and the whole QoI series."""
    p = inputs.config1()
    xo, qo = _orc(p).sample(10000, 1234)
    s = _gpu(p)
    xg, qg = _run_gpu(torch_mod, s, p, 10000, 1234)
    s.close()
    _check64(xg, xo)
    _check64(qg, qo)


def _mean_qoi(torch, p):
    """F . mu with mu = A~^-1 f from the FP64 noise-free V-cycle (the exact posterior mean of the QoI)."""
    s = _gpu(p)
    x = s.zeros()
    _, rr = s.mean_solve(x, rtol=1e-12, max_cycles=200)
    s.close()
    assert rr <= 1e-12
    mu = x.cpu().numpy()
    return float(np.dot(p.qoi_w, mu[p.qoi_site]))


def test_fp32_batch_qoi_mean_matches_mean_solve(torch_mod):
    """Config 2 has no closed form: the FP32 chains' QoI mean must match F . mu from the
    FP64 mean solve within 3 standard errors (32 independent chains x 1000 cycles after
    100 of burn-in; the standard error from the spread of the 32 chain means)."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler
    p = inputs.config2()
    fmu = _mean_qoi(torch, p)
    nc, n = 32, 1100
    b = BatchSampler([p] * nc, precision="fp32")
    xs = b.zeros()
    q = torch.zeros(nc * n, dtype=torch.float64, device="cuda")
    b.sample(xs, n, 808, qoi=q)
    torch.cuda.synchronize()
    b.close()
    means = q.view(nc, n)[:, 100:].mean(1).cpu().numpy()
    se = means.std(ddof=1) / np.sqrt(nc)
    assert abs(means.mean() - fmu) <= 3.0 * se, (means.mean(), fmu, se)


def test_fp32_3d_qoi_mean_matches_mean_solve(torch_mod):
    """Config 3 (127^3): one FP32 chain of 4000 cycles; standard error from the device
    Wolff estimate of its integrated autocorrelation time; within 3 SE of F . mu."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import mgmc_qoi_stats
    p = inputs.config3()
    fmu = _mean_qoi(torch, p)
    s = _gpu(p, precision="fp32")
    x = s.zeros()
    n = 4000
    q = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.sample(x, n, 909, qoi=q)
    st = mgmc_qoi_stats(q.data_ptr(), n, 100, 1.5)
    s.close()
    se = np.sqrt(st["var"] * st["tau_int"] / st["n_used"])
    assert abs(st["mean"] - fmu) <= 3.0 * se, (st["mean"], fmu, se)


def test_restart_is_bit_exact(torch_mod):
    """Counter-based noise: 2 x 50 cycles == 1 x 100 cycles, bit for bit."""
    p = inputs.make_problem("t", 2, 63, kappa2_seed=3, m=6, obs_seed=1)
    for prec in ("fp32", "fp64"):
        s = _gpu(p, precision=prec)
        a, qa = _run_gpu(torch_mod, s, p, 100, 5)
        b, qb1 = _run_gpu(torch_mod, s, p, 50, 5)
        b, qb2 = _run_gpu(torch_mod, s, p, 50, 5, x0=b, step_offset=50)
        assert np.array_equal(a, b)
        assert np.array_equal(qa, np.concatenate([qb1, qb2]))


def test_chains_are_independent_streams(torch_mod):
    p = inputs.make_problem("t", 2, 31, kappa2_const=10.0, m=0, qoi_cells=8)
    o = _orc(p)
    s = _gpu(p)
    for chain in (1, 65535):
        xo, _ = o.sample(5, 8, chain=chain)
        xg, _ = _run_gpu(torch_mod, s, p, 5, 8, chain=chain)
        _check64(xg, xo)


@pytest.mark.parametrize("dim,n,levels,m", [(2, 1, 1, 0), (2, 3, 2, 2), (2, 7, 1, 3), (3, 3, 2, 3), (3, 7, 3, 0)])
def test_small_and_degenerate_grids(torch_mod, dim, n, levels, m):
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=2, m=m, obs_seed=4)
    o = _orc(p)
    s = _gpu(p)
    xo, _ = o.sample(5, 17)
    xg, _ = _run_gpu(torch_mod, s, p, 5, 17)
    _check64(xg, xo)


def test_nu2_sweeps_and_boundary_observations(torch_mod):
    p = inputs.make_problem("t", 2, 63, kappa2_seed=1, m=3, obs_seed=1)
    xyz = np.array([[0.005, 0.5], [0.999, 0.999], [0.5, 0.25]])
    p.obs_site, p.obs_w = inputs.point_obs_rows(63, 2, xyz)
    o = oracle.Oracle(2, 63, p.n_levels, kappa2=p.kappa2, nu1=2, nu2=2, obs_site=p.obs_site, obs_w=p.obs_w,
                      Gamma=p.Gamma, y=p.y)
    s = _gpu(p, nu1=2, nu2=2, coarse_max_n=7)
    xo = o.sample(4, 3, qoi=False)
    xg, _ = _run_gpu(torch_mod, s, p, 4, 3)
    _check64(xg, xo)


def test_mean_solve_matches_oracle(torch_mod):
    p = inputs.make_problem("t", 2, 127, kappa2_seed=9, m=16, obs_seed=7)
    o = _orc(p)
    xo, co, ro = o.mean_solve(rtol=1e-10, max_cycles=100)
    s = _gpu(p)
    x = s.zeros()
    cyc, rr = s.mean_solve(x, rtol=1e-10, max_cycles=100)
    assert rr <= 1e-10
    xg = x.cpu().numpy()
    assert np.abs(xg - xo).max() <= 1e-8 * np.abs(xo).max()


def test_host_buffers_match_device_buffers(torch_mod):
    torch = torch_mod
    p = inputs.make_problem("t", 2, 127, kappa2_seed=4, m=8, obs_seed=2, qoi_cells=32)
    s = _gpu(p, precision="fp32")
    xd, qd = _run_gpu(torch, s, p, 10, 11)
    xh = torch.zeros(p.N, dtype=torch.float32).pin_memory()
    qh = torch.zeros(10, dtype=torch.float64).pin_memory()
    s.sample(xh, 10, 11, qoi=qh)
    assert np.array_equal(xh.double().numpy(), xd)
    assert np.array_equal(qh.numpy(), qd)


def test_qoi_stats_on_device_match_oracle(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import mgmc_qoi_stats
    p = inputs.config1()
    s = _gpu(p)
    x = s.zeros()
    q = torch.zeros(10000, dtype=torch.float64, device="cuda")
    s.sample(x, 10000, 1234, qoi=q)
    st = mgmc_qoi_stats(q.data_ptr(), 10000, 100, 1.5)
    ref = oracle.chain_stats(q[100:].cpu().numpy())
    for k in ("mean", "var", "tau", "tau_err"):
        kk = "tau_int" if k == "tau" else k
        assert st[kk] == pytest.approx(ref[k], rel=1e-10, abs=1e-14)
    assert st["window"] == ref["window"]
    # exact IACT of this chain (closed form from the iteration matrix): 1.228612
    assert abs(st["tau_int"] - 1.228612) < 3 * st["tau_err"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config1_qoi_moments(torch_mod, precision):
    """A chain of config 1 in either precision: QoI mean 0 and variance
    F^T A^-1 F = 0.18241764732 within 3 SE (the closed-form integrated
    autocorrelation time 1.228612 of this chain, which the iteration matrix fixes)."""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import mgmc_qoi_stats
    p = inputs.config1()
    s = _gpu(p, precision=precision)
    x = s.zeros()
    n = 40000
    q = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.sample(x, n, 99, qoi=q)
    st = mgmc_qoi_stats(q.data_ptr(), n, 100, 1.5)
    var, tau = 0.18241764732, 1.228612
    nn = n - 100
    assert abs(st["mean"]) < 3 * np.sqrt(var * tau / nn)
    assert abs(st["var"] - var) < 3 * var * np.sqrt(2 * tau / nn)
