"""Pins of the Sec. 5.3 estimators (paper_2407_12149_gb300/experiments.py).

The law of the chain started at theta^(0) is known in closed form (Lemma
MG-iteration-rep iterated): theta^(m) ~ N((I - X^m) mu, A~^-1 - X^m A~^-1 X^mT)
with X the noise-free V-cycle's iteration matrix (tests/dense_ref.py), and the
lag covariance Cov(theta^(m'), theta^(m)) = X^(m'-m) Cov(theta^(m)) for m' >= m.
Oracle chains on a tiny grid must reproduce the sample means, variances, the
ratios R and Z and the root mean squared error within 3 standard errors.
"""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import experiments as E
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr
from tests.test_oracle_pins import _z_ok


def _dense(p):
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    H = dr.Hierarchy(p.n, p.dim, p.n_levels, p.kappa2 if p.kappa2 is not None else p.kappa2_const, B, p.Gamma,
                     p.scale_hd, disc=p.disc)
    At = H.Atilde(p.n_levels - 1)
    f = B @ np.linalg.solve(p.Gamma, p.y) if p.m else np.zeros(p.N)
    F = np.zeros(p.N)
    np.add.at(F, p.qoi_site, p.qoi_w)
    return H, At, f, F


@pytest.mark.parametrize("disc", [0, 1])
def test_exact_qoi_moments_match_dense_solve(disc):
    p = (inputs.make_problem("e", 2, 15, kappa2_seed=3, m=4, obs_seed=2, qoi_cells=4) if disc == 0 else
         inputs.make_problem("e", 2, 15, kappa2_const=100.0, m=4, obs_seed=2, qoi_cells=4, disc=1))
    _, At, f, F = _dense(p)
    mu, s2 = E.exact_qoi_moments(p)
    assert mu == pytest.approx(F @ np.linalg.solve(At, f), rel=1e-10)
    assert s2 == pytest.approx(F @ np.linalg.solve(At, F), rel=1e-10)


def _chains(p, n_chains, steps, seed):
    """QoI of oracle chains from theta^(0) = 0 at steps 0 .. steps (column 0 = F . 0)."""
    o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const, obs_site=p.obs_site,
                      obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site, qoi_w=p.qoi_w, disc=p.disc)
    z = np.zeros((n_chains, steps + 1))
    for c in range(n_chains):
        _, q = o.sample(steps, seed, x=np.zeros(p.N), chain=c)
        z[c, 1:] = q
    return z


def _law(H, At, f, F, steps):
    """exact mean and variance of z^(m) for theta^(0) = 0, and Cov(z^(m), z^(m'))."""
    X = H.iteration_matrix()
    Sig = np.linalg.inv(At)
    mu = Sig @ f
    N = At.shape[0]
    Xm = [np.eye(N)]
    for _ in range(steps):
        Xm.append(X @ Xm[-1])
    mean = np.array([F @ ((np.eye(N) - Xm[m]) @ mu) for m in range(steps + 1)])
    cov_state = [Sig - Xm[m] @ Sig @ Xm[m].T for m in range(steps + 1)]
    var = np.array([F @ cov_state[m] @ F for m in range(steps + 1)])
    C = np.zeros((steps + 1, steps + 1))
    for m in range(steps + 1):
        for mp in range(m, steps + 1):
            C[m, mp] = C[mp, m] = F @ Xm[mp - m] @ cov_state[m] @ F
    return mean, var, C, F @ mu, F @ Sig @ F


def test_convergence_estimators_against_the_closed_form_law():
    p = inputs.make_problem("e", 2, 7, n_levels=3, kappa2_seed=6, m=3, obs_seed=4, qoi_cells=4)
    H, At, f, F = _dense(p)
    steps, n = 6, 4000
    mean, var, _, mu, s2 = _law(H, At, f, F, steps)
    z = _chains(p, n, steps, 31)
    r = E.convergence_ratios(z, mu, s2)
    m = np.arange(1, steps + 1)
    assert _z_ok(r["mean"][m], mean[m], np.sqrt(var[m] / n))
    assert _z_ok(r["var"][m], var[m], var[m] * np.sqrt(2.0 / (n - 1)))
    # the ratios against their exact values (theta^(0) = 0: mu^(0) = 0, sigma^(0) = 0)
    R_exact = np.abs(mean - mu) / abs(mu)
    Z_exact = np.abs(var - s2) / s2
    assert _z_ok(r["R"][m], R_exact[m], r["R_err"][m])
    assert _z_ok(r["Z"][m], Z_exact[m], r["Z_err"][m])
    assert r["R"][0] == 1.0 and r["Z"][0] == 1.0


def test_rmse_estimator_against_the_closed_form_law():
    p = inputs.make_problem("e", 2, 7, n_levels=3, kappa2_seed=6, m=3, obs_seed=4, qoi_cells=4)
    H, At, f, F = _dense(p)
    steps, n = 8, 4000
    mean, var, C, mu, _ = _law(H, At, f, F, steps)
    z = _chains(p, n, steps, 57)
    Ms = [1, 2, 4, 8]
    got = E.rmse(z, mu, Ms)
    for M, d in zip(Ms, got):
        bias = mu - mean[:M].mean()
        v = C[:M, :M].sum() / M ** 2
        mse = bias ** 2 + v
        se = np.sqrt((2.0 * v ** 2 + 4.0 * bias ** 2 * v) / n)      # of the mean of (mu - zbar)^2
        assert abs(d ** 2 - mse) <= 3.0 * se, (M, d ** 2, mse, se)


def test_rate_takes_the_last_step_within_ten_percent():
    R = np.array([1.0, 0.3, 0.09, 0.027, 0.0081, 0.002])
    err = np.array([0.0, 0.003, 0.003, 0.003, 0.003, 0.003])    # relative: 1 %, 3 %, 11 %, ...
    rho, m_star = E.rate(R, err)
    assert m_star == 2 and rho == pytest.approx(0.09 ** 0.5)
    rho, m_star = E.rate(np.array([1.0, 0.01]), np.array([0.0, 0.005]))
    assert m_star == 1 and rho == pytest.approx(0.01)


@pytest.mark.parametrize("n", [31, 127])
def test_ball_rows_average_constants_and_linear_functions(n):
    """The ball-average rows (inputs.ball_rows) of a ball inside the domain reproduce
    the average of a constant (weights sum to 1) and of the coordinates (the centre):
    the multilinear interpolant of a linear function is the function itself."""
    centres = np.array([[0.31, 0.52], [0.7, 0.27]])
    site, w = inputs.ball_rows(n, 2, centres, 0.025)
    assert np.all(w >= 0.0)
    idx = np.arange(n * n)
    xy = np.stack([(idx % n + 1) / (n + 1), (idx // n + 1) / (n + 1)], axis=1)
    for k in range(2):
        ok = site[k] >= 0
        assert w[k][ok].sum() == pytest.approx(1.0, abs=1e-12)
        centre = (w[k][ok][:, None] * xy[site[k][ok]]).sum(0)
        # the midpoint rule resolves the disc to one sub-cell (h / 8): a wrong vertex
        # index or a transposed axis would be off by about h
        assert np.allclose(centre, centres[k], atol=1.0 / (n + 1) / 8)


def test_ball_rows_near_the_boundary_lose_the_outside_part():
    """Next to x = 0 the interior hat functions sum to clip(x / h, 0, 1): the row's weight
    sum is the ball average of that function (reference: a 64x finer midpoint rule)."""
    n, c, R = 63, np.array([0.01, 0.5]), 0.025
    site, w = inputs.ball_rows(n, 2, c[None, :], R)
    got = w[0][site[0] >= 0].sum()
    h, d = 1.0 / (n + 1), 1.0 / (n + 1) / 64
    ax = np.arange(np.floor((c[0] - R) / d), np.ceil((c[0] + R) / d)) * d + d / 2
    ay = np.arange(np.floor((c[1] - R) / d), np.ceil((c[1] + R) / d)) * d + d / 2
    X, Y = np.meshgrid(ax, ay, indexing="ij")
    inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 <= R * R
    ref = np.clip(X[inside] / h, 0.0, 1.0).mean()
    assert 0.0 < got < 1.0 and abs(got - ref) <= 0.02, (got, ref)
