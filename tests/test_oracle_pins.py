"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: known-answer
vectors, closed forms, dense linear algebra built from the definitions
(tests/dense_ref.py), or statistics whose exact values follow from the
theorems of the paper (moments, one-cycle law, IACT).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(p, **kw):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const,
                         scale_hd=p.scale_hd, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y,
                         qoi_site=p.qoi_site, qoi_w=p.qoi_w, **kw)


def _hier(p):
    k2 = p.kappa2 if p.kappa2 is not None else p.kappa2_const
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    return dr.Hierarchy(p.n, p.dim, p.n_levels, k2, B, p.Gamma, p.scale_hd)


def _stencil_to_dense(st, n, d):
    """Dense matrix of a full W^d stencil (W = 3, or 5 for radius-2 stencils)."""
    N = n ** d
    W = int(round(st.shape[1] ** (1.0 / d)))
    R = W // 2
    A = np.zeros((N, N))
    for s in range(N):
        c = [s % n, (s // n) % n] + ([s // (n * n)] if d == 3 else [])
        for o in range(W ** d):
            off = [o % W - R, (o // W) % W - R] + ([o // (W * W) - R] if d == 3 else [])
            cc = [c[a] + off[a] for a in range(d)]
            if all(0 <= v < n for v in cc):
                t = cc[0] + n * cc[1] + (n * n * cc[2] if d == 3 else 0)
                A[s, t] += st[s, o]
    return A


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert rows
    for r in rows:
        v = [int(t, 16) for t in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_box_muller_normals():
    z = []
    for c in range(20000):
        z.extend(oracle.normal_pair(99, c, 5, 0, 0))
    z = np.array(z)
    assert abs(z.mean()) < 4 * 1 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two members of a pair are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 4 / np.sqrt(z.size / 2)


def test_site_noise_quads_are_independent_standard_normals():
    """The four normals of a site-noise block (two Box-Muller pairs from 32-bit
    uniforms): each member N(0, 1) (moments, Kolmogorov-Smirnov), the six pairs of
    members uncorrelated, and the squares uncorrelated (a wrong angle or a shared
    radius between the two pairs would correlate them)."""
    q = np.array([oracle.normal_quad(7, c, 11, 3 << 16, 2) for c in range(40000)])
    m = q.shape[0]
    for k in range(4):
        z = q[:, k]
        assert abs(z.mean()) < 4 / np.sqrt(m)
        assert abs(z.var() - 1) < 4 * np.sqrt(2 / m)
        assert stats.kstest(z, "norm").pvalue > 1e-3
    for a in range(4):
        for b in range(a + 1, 4):
            assert abs(np.corrcoef(q[:, a], q[:, b])[0, 1]) < 4 / np.sqrt(m)
    assert abs(np.corrcoef(q[:, 0] ** 2, q[:, 2] ** 2)[0, 1]) < 4 / np.sqrt(m)
    # a pair's radius is shared by its members: r^2 = z0^2 + z1^2 ~ chi^2_2 (exponential, mean 2)
    r2 = q[:, 0] ** 2 + q[:, 1] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-3


# --------------------------------------------------------------------------
# hierarchy (Eq. A_ell_1_B_ell_1, Sec. 5.1.3)
# --------------------------------------------------------------------------

def test_galerkin_closed_form_2d():
    """Constant kappa^2, h^d scaling: P^T A P = Laplacian part + kappa^2 h^2 (P1^T P1 x P1^T P1).

    Derivation: the 5-point part times h^2 is the stencil [0 -1 0; -1 4 -1; 0 -1 0];
    its bilinear Galerkin product is [-1 -2 -1; -2 12 -2; -1 -2 -1]/4, and the
    mass part is kappa^2 h^2 times the tensor square of tridiag(1/4, 3/2, 1/4).
    """
    p = inputs.config1()
    o = _oracle(p)
    st = o.stencil(2)                      # 15 x 15 level
    h = 1 / 32
    lap = np.array([[-1, -2, -1], [-2, 12, -2], [-1, -2, -1]]) / 4.0
    m1 = np.array([0.25, 1.5, 0.25])
    expect = lap + 10.0 * h * h * np.outer(m1, m1)
    s = 7 + 15 * 7
    assert np.allclose(st[s].reshape(3, 3), expect, rtol=0, atol=1e-14)
    assert st[s][4] == pytest.approx(3.02197266, abs=1e-8)


@pytest.mark.parametrize("dim,n,levels,var_kappa", [(2, 15, 3, True), (2, 31, 4, False), (3, 7, 2, True),
                                                    (3, 15, 3, False)])
def test_galerkin_equals_dense_PtAP(dim, n, levels, var_kappa):
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=5 if var_kappa else None,
                            kappa2_const=25.0, m=3, obs_seed=4)
    o = _oracle(p)
    H = _hier(p)
    for l in range(levels):
        A = _stencil_to_dense(o.stencil(l), o.level_n(l), dim)
        assert np.allclose(A, H.A[l], rtol=1e-13, atol=1e-13 * abs(H.A[l]).max())
        assert np.allclose(o.B_dense(l), H.B[l], rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# smoother (Alg. 3, Eq. M_lowrank_gibbs / lowrank_gibbs_two_steps)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,levels", [(2, 15, 3), (3, 7, 2)])
@pytest.mark.parametrize("direction", [0, 1])
def test_alg3_equals_generic_random_smoother(dim, n, levels, direction):
    """theta' of Alg. 3 == theta + M~^-1 (f + xi - A~ theta), xi = D^1/2 z + B L_G^-T z',
    for f = fd + B Gamma^-1 d (the split the oracle evaluates)."""
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=3, m=5, obs_seed=2)
    p.Gamma = np.diag(np.linspace(1e-4, 3e-4, 5)) + 2e-5  # non-diagonal SPD Gamma
    o = _oracle(p)
    H = _hier(p)
    rng = np.random.default_rng(0)
    for l in range(1, levels):
        N = o.level_N(l)
        theta = rng.normal(size=N)
        fd = rng.normal(size=N)
        d = rng.normal(size=5) * 3.0
        zd = rng.normal(size=N)
        zl = rng.normal(size=5)
        got = o.smoother_step_given(l, direction, theta, fd, zd, zl, d=d)
        D = np.diag(np.diag(H.A[l]))
        LG = np.linalg.cholesky(p.Gamma)
        f = fd + H.B[l] @ np.linalg.solve(p.Gamma, d)
        xi = np.sqrt(D) @ zd + H.B[l] @ np.linalg.solve(LG.T, zl)
        M = H.splitting(l, direction)
        want = theta + np.linalg.solve(M, f + xi - H.Atilde(l) @ theta)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * abs(want).max())


def test_smoother_noise_covariance_identity_and_naive_split():
    """M~ + M~^T - A~ = D + B Gamma^-1 B^T (Eq. low_rank_smoother_covariance) and the naive
    D + L splitting gives the indefinite D - B Gamma^-1 B^T (end of Sec. 3.4)."""
    p = inputs.make_problem("t", 2, 15, n_levels=3, kappa2_const=10.0, m=8, obs_seed=1)
    H = _hier(p)
    l = 2
    M = H.splitting(l, 0)
    lhs = M + M.T - H.Atilde(l)
    rhs = np.diag(np.diag(H.A[l])) + H.B[l] @ H.Gi @ H.B[l].T
    assert np.allclose(lhs, rhs, atol=1e-9)
    naive = np.diag(np.diag(H.A[l])) - H.B[l] @ H.Gi @ H.B[l].T
    assert np.linalg.eigvalsh(naive).min() < 0


def test_lowrank_G_matches_definition():
    """G = M^-1 B (Gamma + B^T M^-1 B)^-1 with M = D + L (Eq. Bellstar_definition)."""
    p = inputs.make_problem("t", 2, 15, n_levels=3, kappa2_seed=1, m=6, obs_seed=9)
    o = _oracle(p)
    H = _hier(p)
    for l in (1, 2):
        for direction in (0, 1):
            M = H.splitting(l, direction) - H.B[l] @ H.Gi @ H.B[l].T
            C = np.linalg.solve(M, H.B[l])
            G = C @ np.linalg.inv(p.Gamma + H.B[l].T @ C)
            assert np.allclose(o.G_dense(l, direction), G, rtol=1e-10, atol=1e-12 * abs(G).max())


# --------------------------------------------------------------------------
# cycle (Alg. 1) -- deterministic part
# --------------------------------------------------------------------------

def _oracle_X(o, N):
    """Columns X e_j of the affine noise-free cycle theta -> X theta + c."""
    c = o.sample(1, 0, x=np.zeros(N), noise=False, qoi=False)
    X = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        X[:, j] = o.sample(1, 0, x=e, noise=False, qoi=False) - c
    return X


@pytest.mark.parametrize("dim,n,levels,m", [(2, 15, 3, 0), (2, 15, 4, 6), (3, 7, 2, 4), (2, 7, 1, 3)])
def test_noise_free_cycle_is_dense_multigrid(dim, n, levels, m):
    """With all noise zeroed, one MGMC cycle is theta -> X theta + (I - X) A~^-1 f."""
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=8, m=m, obs_seed=6)
    o = _oracle(p)
    H = _hier(p)
    X = H.iteration_matrix()
    Xo = _oracle_X(o, p.N)
    assert np.allclose(Xo, X, atol=1e-11)
    mu = np.linalg.solve(H.Atilde(levels - 1), o.fine_rhs())
    if m:
        assert np.allclose(o.fine_rhs(), H.B[-1] @ np.linalg.solve(p.Gamma, p.y), atol=1e-9)
    x1 = o.sample(1, 0, x=np.zeros(p.N), noise=False, qoi=False)
    assert np.allclose(x1, (np.eye(p.N) - X) @ mu, atol=1e-9 * max(1, abs(mu).max()))


def test_contraction_config1_and_grid_independence():
    """||X||_A of the noise-free V-cycle (config 1: 31^2, kappa^2 = 10, 4 grids), and the same
    cycle on finer grids (Thm. moments-conv: the bound is independent of L)."""
    p = inputs.config1()
    o = _oracle(p)
    H = _hier(p)
    X = _oracle_X(o, p.N)
    rho31 = dr.a_norm(X, H.Atilde(3))
    assert rho31 == pytest.approx(dr.a_norm(H.iteration_matrix(), H.Atilde(3)), abs=1e-10)
    assert 0.2 < rho31 < 0.3
    # power iteration on finer grids (X is A-self-adjoint: ||X||_A = spectral radius)
    rhos = [rho31]
    for n, L in ((63, 5), (127, 6)):
        oo = oracle.Oracle(2, n, L, kappa2_const=10.0)     # f = 0: the cycle is linear
        v = np.random.default_rng(1).normal(size=n * n)
        lam = 0
        for _ in range(40):
            w = oo.sample(1, 0, x=v, noise=False, qoi=False)
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        rhos.append(lam)
    assert max(rhos) - min(rhos) < 0.02


def test_mean_solve_matches_dense_solve():
    p = inputs.make_problem("t", 2, 31, n_levels=4, kappa2_seed=2, m=8, obs_seed=3)
    o = _oracle(p)
    H = _hier(p)
    mu = np.linalg.solve(H.Atilde(3), o.fine_rhs())
    x, cyc, rr = o.mean_solve(rtol=1e-12, max_cycles=200)
    assert rr <= 1e-12 and cyc < 200
    assert np.allclose(x, mu, atol=1e-9 * abs(mu).max())


def test_coarsest_operator_is_galerkin_posterior():
    p = inputs.make_problem("t", 3, 7, n_levels=2, kappa2_const=25.0, m=5, obs_seed=3)
    o = _oracle(p)
    H = _hier(p)
    assert np.allclose(o.coarsest_dense(), H.Atilde(0), atol=1e-12)


# --------------------------------------------------------------------------
# cycle (Alg. 1) -- the law of the random iteration
# --------------------------------------------------------------------------

def _z_ok(est, exact, se):
    """Every estimate within 3 standard errors, read at the family-wise level of a
    3-sigma test: with M estimates the two-sided 3-sigma tail (0.27 %) is shared
    over all of them (Bonferroni: |z| <= Phi^-1(1 - 0.0027 / 2M)), and the count of
    estimates beyond 3 SE must be within the 99.73 % quantile of Binomial(M, 0.0027).
    (M individual 3-SE tests fail somewhere with probability 1 - 0.9973^M.)"""
    z = np.abs(np.asarray(est) - np.asarray(exact)).ravel() / (np.asarray(se).ravel() + 1e-300)
    M = z.size
    return (np.all(z <= stats.norm.ppf(1.0 - 0.0027 / (2 * M)))
            and np.count_nonzero(z > 3.0) <= stats.binom.ppf(0.9973, M, 0.0027))


def _stationary_lag_covariances(X, Sigma, tol=1e-14):
    """C_t = Cov(theta_{k+t}, theta_k) = X^t Sigma of the stationary chain
    theta_{k+1} = X theta_k + c + noise (Lemma MG-iteration-rep), t = 0, 1, ...
    until it has decayed below tol relative to Sigma."""
    C = [Sigma]
    while np.abs(C[-1]).max() > tol * np.abs(Sigma).max() and len(C) < 2000:
        C.append(X @ C[-1])
    return C


@pytest.mark.parametrize("dim,n,levels,m", [(2, 7, 3, 3), (3, 7, 2, 4)])
def test_one_cycle_law(dim, n, levels, m):
    """Lemma MG-iteration-rep: theta' ~ N(X theta0 + (I - X) mu, A~^-1 - X A~^-1 X^T)."""
    p = inputs.make_problem("t", dim, n, n_levels=levels, kappa2_seed=4, m=m, obs_seed=5)
    o = _oracle(p)
    H = _hier(p)
    At = H.Atilde(levels - 1)
    X = H.iteration_matrix()
    Ai = np.linalg.inv(At)
    mu = Ai @ o.fine_rhs()
    rng = np.random.default_rng(3)
    theta0 = rng.normal(size=p.N) * 0.5
    mean_exact = X @ theta0 + (np.eye(p.N) - X) @ mu
    cov_exact = Ai - X @ Ai @ X.T
    S = 12000
    draws = np.empty((S, p.N))
    for c in range(S):
        draws[c] = o.sample(1, 777, x=theta0, chain=c, qoi=False)
    mean = draws.mean(0)
    cov = np.cov(draws.T)
    sd = np.sqrt(np.diag(cov_exact))
    # independent chains: the standard errors are exact
    assert _z_ok(mean, mean_exact, sd / np.sqrt(S))
    se_cov = np.sqrt((cov_exact ** 2 + np.outer(np.diag(cov_exact), np.diag(cov_exact))) / S)
    iu = np.triu_indices(p.N)
    assert _z_ok(cov[iu], cov_exact[iu], se_cov[iu])


@pytest.mark.parametrize("levels", [1, 3])
def test_invariance_moments_vs_dense_cholesky(levels):
    """Theorem mgmc_invariance: started in N(mu, A~^-1) the chain stays there; the sample
    moments of a long chain match mu = A~^-1 f and A~^-1 (dense Cholesky) within 3 SE.
    The standard errors use each coordinate's own integrated autocorrelation in closed
    form from the exact iteration matrix X (Sec. 4: the lag-t covariance of the
    stationary chain is X^t A~^-1): Var(mean_i) = Sigma_ii tau_i / S with
    tau_i = 1 + 2 sum_t (X^t Sigma)_ii / Sigma_ii, and for the sample covariance (Isserlis)
    Var(c_ij) = (1/S) sum_t [C_t,ii C_t,jj + C_t,ij C_t,ji] over all lags t."""
    p = inputs.make_problem("t", 2, 7, n_levels=levels, kappa2_seed=6, m=4, obs_seed=8)
    o = _oracle(p)
    H = _hier(p)
    At = H.Atilde(levels - 1)
    Ai = np.linalg.inv(At)
    mu = Ai @ o.fine_rhs()
    Lc = np.linalg.cholesky(Ai)
    x0 = mu + Lc @ np.random.default_rng(2).normal(size=p.N)      # exact draw from the target
    S = 40000
    draws = np.empty((S, p.N))
    x = x0
    for k in range(0, S, 1000):
        # record every cycle: chunked so the state carries over
        for j in range(1000):
            x = o.sample(1, 4242, x=x, step_offset=k + j, qoi=False)
            draws[k + j] = x
    C = _stationary_lag_covariances(H.iteration_matrix(), Ai)
    d = np.diag(Ai)
    tau = 1.0 + 2.0 * sum(np.diag(c) for c in C[1:]) / d
    assert np.all(tau >= 1.0 - 1e-12) and tau.max() < 5.0
    var_cov = (np.outer(d, d) + Ai ** 2
               + 2.0 * sum(np.outer(np.diag(c), np.diag(c)) + c * c.T for c in C[1:]))
    mean = draws.mean(0)
    cov = np.cov(draws.T)
    assert np.all(np.abs(mean - mu) <= 3.0 * np.sqrt(d * tau / S))      # each coordinate at 3 SE
    assert _z_ok(mean, mu, np.sqrt(d * tau / S))
    iu = np.triu_indices(p.N)
    assert _z_ok(cov[iu], Ai[iu], np.sqrt(var_cov[iu] / S))


def test_iact_config1_matches_closed_form():
    """Eq. tau_int: tau_inf = 1 + 2 sum_s F^T X^s A^-1 F / F^T A^-1 F for config 1; the oracle
    chain (10^4 cycles, seed 1234, x0 = 0) and Wolff's estimator must agree within 3 errors,
    and the QoI mean (exact 0) and variance F^T A^-1 F within 3-4 SE."""
    p = inputs.config1()
    o = _oracle(p)
    H = _hier(p)
    X = H.iteration_matrix()
    Ai = np.linalg.inv(H.Atilde(3))
    F = np.zeros(p.N)
    F[p.qoi_site] = p.qoi_w
    var = F @ Ai @ F
    tau_inf, Xs = 1.0, np.eye(p.N)
    for _ in range(100):
        Xs = X @ Xs
        tau_inf += 2 * (F @ Xs @ Ai @ F) / var
    assert tau_inf == pytest.approx(1.228612, abs=2e-6)
    assert var == pytest.approx(0.18241764732, abs=1e-10)
    x, q = o.sample(10000, 1234)
    st = oracle.chain_stats(q[100:])
    assert abs(st["tau"] - tau_inf) < 3 * st["tau_err"]
    n = q[100:].size
    assert abs(st["mean"]) < 4 * np.sqrt(var * tau_inf / n)
    assert abs(st["var"] - var) < 4 * var * np.sqrt(2 * tau_inf / n)


# --------------------------------------------------------------------------
# chain statistics (Sec. 5.3.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("phi", [0.0, 0.5, 0.8])
def test_wolff_on_ar1(phi):
    """AR(1): rho(t) = phi^t, so tau = (1 + phi) / (1 - phi)."""
    from scipy.signal import lfilter
    rng = np.random.default_rng(11)
    n = 200000
    e = rng.normal(size=n)
    z = lfilter([np.sqrt(1 - phi * phi)], [1.0, -phi], e)
    st = oracle.chain_stats(z)
    exact = (1 + phi) / (1 - phi)
    assert abs(st["tau"] - exact) < 3 * st["tau_err"] + 1e-3
    assert st["ess"] == pytest.approx(n / st["tau"])


def test_chain_stats_degenerate():
    st = oracle.chain_stats(np.full(100, 3.0))
    assert st["tau"] == 1.0 and st["var"] == 0.0 and st["mean"] == 3.0


# --------------------------------------------------------------------------
# inputs and argument checking
# --------------------------------------------------------------------------

def test_qoi_weights_config1():
    p = inputs.config1()
    W = np.zeros(p.N)
    W[p.qoi_site] = p.qoi_w
    W = W.reshape(31, 31)
    assert W.sum() == pytest.approx(1.0)
    assert W[15, 15] == pytest.approx(1 / 64) and W[11, 15] == pytest.approx(1 / 128)
    assert W[11, 11] == pytest.approx(1 / 256) and W[10, 15] == 0.0


def test_point_obs_rows_interpolate_bilinear():
    n = 15
    xyz = np.array([[0.3, 0.71], [0.01, 0.53], [0.99, 0.99]])
    site, w = inputs.point_obs_rows(n, 2, xyz)
    h = 1 / (n + 1)
    # B^T applied to a bilinear function reproduces it (interpolation is exact)
    X, Y = np.meshgrid((np.arange(n) + 1) * h, (np.arange(n) + 1) * h)
    fgrid = (2 * X + 3 * Y + X * Y).ravel()
    fgrid_exact = lambda x, y: 2 * x + 3 * y + x * y
    got = np.array([sum(ww * fgrid[s] for s, ww in zip(site[k], w[k]) if s >= 0) for k in range(3)])
    assert got[0] == pytest.approx(fgrid_exact(0.3, 0.71))
    # near the boundary the missing vertex carries value 0 (Dirichlet), so weights sum < 1
    assert w[1].sum() < 1 and (site[1] == -1).sum() == 2


def test_oracle_rejects_bad_sizes():
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(2, 30, 3)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(2, 7, 4)
