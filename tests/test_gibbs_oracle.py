"""Pins of the oracle's plain Gibbs sampler (Sec. 5.1.3, "Gibbs sampler"): one step is
the forward then the backward low-rank Gibbs sweep (Alg. 3) of the finest grid.

Checked against dense linear algebra built from the definitions (tests/dense_ref.py):
the noise-free step is theta -> K theta + (I - K) A~^-1 f with K = S_b S_f,
S_dir = I - M~_dir^-1 A~; the IACT of a long chain equals the closed form of
Eq. tau_int for that K; and the closed form grows with the resolution while the
MGMC V-cycle's does not (the comparison of Table 1 and Fig. autocorrelation).
"""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr


def _oracle(p):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const,
                         scale_hd=p.scale_hd, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y,
                         qoi_site=p.qoi_site, qoi_w=p.qoi_w)


def _hier(p):
    k2 = p.kappa2 if p.kappa2 is not None else p.kappa2_const
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    return dr.Hierarchy(p.n, p.dim, p.n_levels, k2, B, p.Gamma, p.scale_hd)


def _gibbs_K(H):
    l = len(H.A) - 1
    return H.smoother_matrix(l, 1) @ H.smoother_matrix(l, 0)


def _tau_closed_form(K, Ai, F, terms):
    """Eq. tau_int for the chain theta' = K theta + noise at stationarity:
    rho(t) = F^T K^t A~^-1 F / F^T A~^-1 F."""
    var = F @ Ai @ F
    tau, v = 1.0, Ai @ F
    for _ in range(terms):
        v = K @ v
        tau += 2 * (F @ v) / var
    return tau, var


@pytest.mark.parametrize("dim,n,levels,m", [(2, 15, 3, 0), (2, 15, 4, 6), (3, 7, 2, 4)])
def test_noise_free_gibbs_step_is_dense_sgs(dim, n, levels, m):
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=8, m=m, obs_seed=6)
    o = _oracle(p)
    H = _hier(p)
    K = _gibbs_K(H)
    c = o.sample(1, 0, x=np.zeros(p.N), noise=False, qoi=False, gibbs=True)
    Ko = np.zeros((p.N, p.N))
    for j in range(p.N):
        e = np.zeros(p.N)
        e[j] = 1.0
        Ko[:, j] = o.sample(1, 0, x=e, noise=False, qoi=False, gibbs=True) - c
    assert np.allclose(Ko, K, atol=1e-11)
    mu = np.linalg.solve(H.Atilde(levels - 1), o.fine_rhs())
    assert np.allclose(c, (np.eye(p.N) - K) @ mu, atol=1e-9 * max(1.0, abs(mu).max()))


def test_gibbs_and_mgmc_steps_differ_only_by_the_coarse_correction():
    """n_levels = 2 with the coarse grid solved exactly: the MGMC cycle is S_b (coarse
    correction) S_f, the Gibbs step S_b S_f; both start from the same forward sweep, so
    with the same seed the two chains agree after the forward half-step and differ after."""
    p = inputs.make_problem("t", 2, 15, n_levels=2, kappa2_seed=3, m=3, obs_seed=2)
    o = _oracle(p)
    H = _hier(p)
    Xm = H.iteration_matrix()
    K = _gibbs_K(H)
    assert not np.allclose(Xm, K, atol=1e-6)
    x = o.sample(1, 0, x=np.ones(p.N), noise=False, qoi=False, gibbs=True)
    mu = np.linalg.solve(H.Atilde(1), o.fine_rhs())
    assert np.allclose(x, K @ np.ones(p.N) + (np.eye(p.N) - K) @ mu, atol=1e-9)


def test_gibbs_iact_matches_closed_form():
    """31^2, kappa^2 = 10, no observations, QoI central 8x8 cells (the config of the plain
    MGMC pins): Wolff's estimate of a 40 000-step oracle Gibbs chain agrees with the
    closed-form IACT within 3 errors; the QoI mean (exact 0) and variance F^T A^-1 F
    within 4 SE."""
    p = inputs.config1()
    o = _oracle(p)
    H = _hier(p)
    K = _gibbs_K(H)
    Ai = np.linalg.inv(H.Atilde(len(H.A) - 1))
    F = np.zeros(p.N)
    F[p.qoi_site] = p.qoi_w
    tau_inf, var = _tau_closed_form(K, Ai, F, 4000)
    assert 3.0 < tau_inf < 200.0          # far above MGMC's 1.23 on the same problem
    burn = 2000
    _, q = o.sample(40000 + burn, 77, gibbs=True)
    st = oracle.chain_stats(q[burn:])
    assert abs(st["tau"] - tau_inf) < 3 * st["tau_err"], (st["tau"], st["tau_err"], tau_inf)
    n = q[burn:].size
    assert abs(st["mean"]) < 4 * np.sqrt(var * tau_inf / n)
    assert abs(st["var"] - var) < 4 * var * np.sqrt(2 * tau_inf / n)


def test_gibbs_iact_grows_with_resolution_mgmc_does_not():
    """Closed-form IACT of the QoI for n = 7, 15, 31 (kappa^2 = 10, central box of a
    quarter of the domain): the Gibbs sampler's grows by more than 2x per halving of h,
    the MGMC V-cycle's stays within 10% (Thm. IACT; Table 1)."""
    tg, tm = [], []
    for n, cells in ((7, 2), (15, 4), (31, 8)):
        p = inputs.make_problem("t", 2, n, kappa2_const=10.0, qoi_cells=cells)
        H = _hier(p)
        Ai = np.linalg.inv(H.Atilde(len(H.A) - 1))
        F = np.zeros(p.N)
        F[p.qoi_site] = p.qoi_w
        tg.append(_tau_closed_form(_gibbs_K(H), Ai, F, 20000)[0])
        tm.append(_tau_closed_form(H.iteration_matrix(), Ai, F, 200)[0])
    assert tg[1] > 2 * tg[0] and tg[2] > 2 * tg[1], tg
    assert max(tm) < 1.1 * min(tm), tm
    assert max(tm) < tg[0], (tm, tg)


def test_gibbs_needs_two_grids():
    p = inputs.make_problem("t", 2, 7, n_levels=1, kappa2_seed=1, m=2, obs_seed=1)
    o = _oracle(p)
    with pytest.raises(oracle.OracleError):
        o.sample(1, 0, gibbs=True)
