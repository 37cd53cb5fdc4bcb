"""Pins of the oracle's FP32 site-noise mode (oracle_set_draws32): one Philox4x32-10
block per 8-site span of a grid row and one parity, one 32-bit word per uniform.

The site normals are read back from a chain (one forward sweep of the prior from
theta = 0 leaves theta_i = z_i / sqrt(a_ii) on the sites with i + j even, whose
neighbours are all still zero), then checked for the standard normal law (KS) and
recomputed from the Philox known-answer-pinned block function and the Box-Muller
map; the chain moments and the IACT in this mode are checked against the dense
closed forms as for the FP64 draws.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr


def _oracle(p, **kw):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const,
                         scale_hd=p.scale_hd, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y,
                         qoi_site=p.qoi_site, qoi_w=p.qoi_w, **kw)


def _first_sweep_normals(n, seed, cycle, draws32=True):
    """z on the i + j even sites after one forward sweep of the prior from 0 (kappa^2 = 10)."""
    p = inputs.make_problem("t", 2, n, kappa2_const=10.0)
    o = oracle.Oracle(2, n, p.n_levels, kappa2_const=10.0, nu1=1, nu2=0, draws32=draws32)
    x = o.sample(1, seed, x=np.zeros(p.N), step_offset=cycle, qoi=False, gibbs=True)
    a = np.diag(dr.fd_operator(n, 2, 10.0)).copy()
    z = x * np.sqrt(a)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    even = ((i + j) % 2 == 0).ravel()
    return z, even, p.n_levels - 1


def _expected32(seed, cycle, level, slot, n, i, j):
    """The stated draw: block ((j n_sp + i / 8) * 2 + i % 2, cycle, chain 0, kind 3)."""
    nsp = (n + 7) // 8
    block = ((j * nsp + (i >> 3)) * 2 + (i & 1)) & 0xFFFFFFFF
    w = oracle.philox4x32_10([block, cycle & 0xFFFFFFFF, (cycle >> 32) & 0xFFFF,
                              (3 << 24) | (level << 16) | slot], [seed & 0xFFFFFFFF, seed >> 32])
    h = (i >> 2) & 1
    u1 = (w[2 * h] + 0.5) * 2.0 ** -32
    u2 = (w[2 * h + 1] + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.sin(2 * np.pi * u2) if (i >> 1) & 1 else r * np.cos(2 * np.pi * u2)


def test_draws32_normals_follow_the_stated_map():
    n, seed, cycle = 31, 0x1234_5678_9ABC, 7
    z, even, level = _first_sweep_normals(n, seed, cycle)
    for s in np.flatnonzero(even)[::17]:
        i, j = s % n, s // n
        assert z[s] == pytest.approx(_expected32(seed, cycle, level, 0, n, i, j), rel=1e-12, abs=1e-12)


def test_draws32_normals_are_standard_and_differ_from_fp64_draws():
    vals = []
    for seed in range(12):
        z, even, _ = _first_sweep_normals(31, seed, 3)
        vals.append(z[even])
    v = np.concatenate(vals)
    assert stats.kstest(v, "norm").pvalue > 1e-3
    assert abs(v.mean()) < 4 / np.sqrt(v.size) and abs(v.var() - 1) < 6 * np.sqrt(2 / v.size)
    assert np.unique(v).size == v.size
    z64, even, _ = _first_sweep_normals(31, 0, 3, draws32=False)
    assert not np.allclose(z64[even], vals[0])


def test_draws32_chain_iact_matches_closed_form():
    """The config-1 chain (31^2, kappa^2 = 10, 4 grids) with the FP32 draws: Wolff's IACT
    equals the closed form of Eq. tau_int (1.228612) within 3 errors; QoI mean and variance
    within 4 SE of 0 and F^T A^-1 F."""
    p = inputs.config1()
    o = _oracle(p, draws32=True)
    H = dr.Hierarchy(p.n, p.dim, p.n_levels, p.kappa2_const, None, None, p.scale_hd)
    X = H.iteration_matrix()
    Ai = np.linalg.inv(H.Atilde(3))
    F = np.zeros(p.N)
    F[p.qoi_site] = p.qoi_w
    var = F @ Ai @ F
    tau_inf, Xs = 1.0, np.eye(p.N)
    for _ in range(100):
        Xs = X @ Xs
        tau_inf += 2 * (F @ Xs @ Ai @ F) / var
    _, q = o.sample(10000, 99)
    st = oracle.chain_stats(q[100:])
    assert abs(st["tau"] - tau_inf) < 3 * st["tau_err"]
    m = q[100:].size
    assert abs(st["mean"]) < 4 * np.sqrt(var * tau_inf / m)
    assert abs(st["var"] - var) < 4 * var * np.sqrt(2 * tau_inf / m)


def test_draws32_posterior_moments_vs_dense_cholesky():
    """Theorem mgmc_invariance with the FP32 draws: 7^2 posterior (4 observations, 3 grids),
    chain started in the target; sample mean and covariance within 5 SE of A~^-1 f, A~^-1."""
    p = inputs.make_problem("t", 2, 7, n_levels=3, kappa2_seed=6, m=4, obs_seed=8)
    o = _oracle(p, draws32=True)
    k2 = p.kappa2
    H = dr.Hierarchy(p.n, 2, 3, k2, dr.B_dense(p.N, p.obs_site, p.obs_w), p.Gamma, p.scale_hd)
    Ai = np.linalg.inv(H.Atilde(2))
    mu = Ai @ o.fine_rhs()
    x = mu + np.linalg.cholesky(Ai) @ np.random.default_rng(5).normal(size=p.N)
    S = 30000
    draws = np.empty((S, p.N))
    for k in range(S):
        x = o.sample(1, 777, x=x, step_offset=k, qoi=False)
        draws[k] = x
    tau = 3.0
    sd = np.sqrt(np.diag(Ai))
    assert np.all(np.abs(draws.mean(0) - mu) <= 5 * sd * np.sqrt(tau / S))
    cov = np.cov(draws.T)
    se = np.sqrt(tau * (Ai ** 2 + np.outer(np.diag(Ai), np.diag(Ai))) / S)
    assert np.all(np.abs(cov - Ai) <= 5 * se)
