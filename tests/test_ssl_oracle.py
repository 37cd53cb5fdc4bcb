"""Pins of the oracle's squared shifted Laplacian (Eq. squared_shifted_laplace,
13-point finite differences with u = du/dn = 0, Sec. 5.1.1) and of its W-cycle
(Alg. 1 with gamma = 2, Sec. 5.1.3), against constructions that do not use the
oracle's stencil code: the matrix square of the shifted 5-point operator plus
the clamped-boundary diagonal (tests/dense_ref.py), the closed-form spectrum of
that square, the ghost-point rows written out by hand, dense Galerkin products,
dense V- and W-cycle iteration matrices, and the law of one W-cycle."""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr
from tests.test_oracle_pins import _oracle_X, _stencil_to_dense, _z_ok


def _problem(n, levels, m, seed=4):
    return inputs.make_problem("ssl", 2, n, n_levels=levels, kappa2_const=100.0, m=m, obs_seed=seed, disc=2)


def _oracle(p, gamma=2):
    return oracle.Oracle(2, p.n, p.n_levels, kappa2_const=p.kappa2_const, scale_hd=p.scale_hd,
                         obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                         qoi_w=p.qoi_w, disc=2, gamma=gamma)


def _hier(p, gamma=2):
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    return dr.Hierarchy(p.n, 2, p.n_levels, p.kappa2_const, B, p.Gamma, p.scale_hd, disc=2, gamma=gamma)


@pytest.mark.parametrize("n,scale_hd", [(1, 1), (2, 1), (5, 0), (7, 1), (8, 0)])
def test_ssl_operator_is_clamped_square(n, scale_hd):
    """13-point stencil with mirror ghosts == s [(kappa^2 + L)^2 + 2 h^-4 E]."""
    o = oracle.Oracle(2, n, 1, kappa2_const=37.0, scale_hd=scale_hd, disc=2)
    A = _stencil_to_dense(o.stencil(0), n, 2)
    ref = dr.ssl_operator(n, 37.0, scale_hd)
    assert np.allclose(A, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0


def test_ssl_spectrum_closed_form():
    """Without the boundary diagonal the matrix is (kappa^2 + L)^2, whose eigenvalues are
    (kappa^2 + lambda_a + lambda_b)^2, lambda_a = 4 h^-2 sin^2(a pi h / 2), a = 1..n."""
    n, k2 = 9, 100.0
    h = 1.0 / (n + 1)
    o = oracle.Oracle(2, n, 1, kappa2_const=k2, scale_hd=0, disc=2)
    A = _stencil_to_dense(o.stencil(0), n, 2)
    idx = np.arange(n * n)
    i, j = idx % n, idx // n
    E = (i == 0).astype(float) + (i == n - 1) + (j == 0) + (j == n - 1)
    got = np.sort(np.linalg.eigvalsh(A - np.diag(2.0 * E / h ** 4)))
    lam = 4.0 / h ** 2 * np.sin(np.arange(1, n + 1) * np.pi * h / 2.0) ** 2
    want = np.sort(((k2 + lam[:, None] + lam[None, :]) ** 2).ravel())
    assert np.allclose(got, want, rtol=1e-12)


def test_ssl_rows_written_out():
    """Rows of the 13-point stencil (Bjorstad's discretisation) by hand, h = 1/8,
    kappa^2 = 100, no scaling: deep inside 20 / -8 / 2 / 1 (times h^-4) plus
    2 kappa^2 (4, -1) h^-2 + kappa^4; next to one boundary the mirror ghost adds h^-4
    to the centre (21), at a corner twice (22); couplings onto the boundary vanish."""
    n, k2 = 7, 100.0
    h = 1.0 / 8
    i4, i2 = h ** -4, h ** -2
    st = oracle.Oracle(2, n, 1, kappa2_const=k2, scale_hd=0, disc=2).stencil(0)
    o = lambda dx, dy: (dx + 2) + 5 * (dy + 2)
    deep = st[3 + 7 * 3]
    assert deep[o(0, 0)] == pytest.approx(20 * i4 + 8 * k2 * i2 + k2 ** 2, rel=1e-15)
    assert deep[o(1, 0)] == pytest.approx(-8 * i4 - 2 * k2 * i2, rel=1e-15)
    assert deep[o(1, 1)] == pytest.approx(2 * i4, rel=1e-15)
    assert deep[o(0, -2)] == pytest.approx(i4, rel=1e-15)
    assert deep[o(2, 1)] == 0.0 and deep[o(2, 2)] == 0.0
    edge = st[0 + 7 * 3]                      # i = 0: left boundary at distance 1
    assert edge[o(0, 0)] == pytest.approx(21 * i4 + 8 * k2 * i2 + k2 ** 2, rel=1e-15)
    assert edge[o(-1, 0)] == 0.0 and edge[o(-2, 0)] == 0.0 and edge[o(-1, 1)] == 0.0
    assert edge[o(2, 0)] == pytest.approx(i4, rel=1e-15)
    corner = st[0]
    assert corner[o(0, 0)] == pytest.approx(22 * i4 + 8 * k2 * i2 + k2 ** 2, rel=1e-15)
    assert np.count_nonzero(corner) == 6      # centre, (1,0), (0,1), (1,1), (2,0), (0,2)


@pytest.mark.parametrize("n,levels", [(15, 3), (31, 4)])
def test_ssl_galerkin_equals_dense_PtAP(n, levels):
    p = _problem(n, levels, 4)
    o = _oracle(p)
    H = _hier(p)
    for l in range(levels):
        A = _stencil_to_dense(o.stencil(l), o.level_n(l), 2)
        assert np.allclose(A, H.A[l], rtol=1e-12, atol=1e-12 * np.abs(H.A[l]).max())
        np.testing.assert_allclose(o.B_dense(l), H.B[l], atol=1e-14)


def test_nine_colours_decouple_every_level():
    """Sites of one class (i mod 3, j mod 3) are never coupled on any level, so the
    colour-ordered sweep is a Gauss-Seidel sweep in one fixed order."""
    p = _problem(31, 4, 0)
    o = _oracle(p)
    for l in range(4):
        nl = o.level_n(l)
        A = _stencil_to_dense(o.stencil(l), nl, 2)
        idx = np.arange(nl * nl)
        code = (idx % nl) % 3 + 3 * ((idx // nl) % 3)
        for c in range(9):
            sub = A[np.ix_(code == c, code == c)]
            assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0


@pytest.mark.parametrize("direction", [0, 1])
def test_ssl_alg3_equals_generic_random_smoother(direction):
    """Alg. 3 on radius-2 levels == theta + M~^-1 (f + xi - A~ theta), the nine-colour
    splitting (Eq. M_lowrank_gibbs)."""
    p = _problem(15, 3, 5, seed=2)
    o = _oracle(p)
    H = _hier(p)
    rng = np.random.default_rng(0)
    for l in (1, 2):
        N = o.level_N(l)
        theta, fd, zd = rng.normal(size=N), rng.normal(size=N), rng.normal(size=N)
        d, zl = rng.normal(size=5) * 3.0, rng.normal(size=5)
        got = o.smoother_step_given(l, direction, theta, fd, zd, zl, d=d)
        D = np.diag(np.diag(H.A[l]))
        LG = np.linalg.cholesky(p.Gamma)
        f = fd + H.B[l] @ np.linalg.solve(p.Gamma, d)
        xi = np.sqrt(D) @ zd + H.B[l] @ np.linalg.solve(LG.T, zl)
        want = theta + np.linalg.solve(H.splitting(l, direction), f + xi - H.Atilde(l) @ theta)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * abs(want).max())


@pytest.mark.parametrize("disc,n,levels,m", [(2, 15, 3, 0), (2, 15, 4, 5), (0, 15, 4, 4), (0, 31, 4, 0)])
def test_w_cycle_noise_free_is_dense_multigrid(disc, n, levels, m):
    """gamma = 2: one noise-free cycle is X_W theta + (I - X_W) mu with the dense W-cycle
    matrix, which differs from the V-cycle's from four grids on (with three, the second
    call is the exact coarsest solve again)."""
    if disc == 2:
        p = _problem(n, levels, m, seed=6)
    else:
        p = inputs.make_problem("sl", 2, n, n_levels=levels, kappa2_seed=8, m=m, obs_seed=6)
    o = oracle.Oracle(2, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const, obs_site=p.obs_site,
                      obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, disc=disc, gamma=2)
    k2 = p.kappa2 if p.kappa2 is not None else p.kappa2_const
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    H = dr.Hierarchy(p.n, 2, levels, k2, B, p.Gamma, p.scale_hd, disc=disc, gamma=2)
    XW = H.iteration_matrix()
    Xo = _oracle_X(o, p.N)
    assert np.allclose(Xo, XW, atol=1e-11)
    HV = dr.Hierarchy(p.n, 2, levels, k2, B, p.Gamma, p.scale_hd, disc=disc, gamma=1)
    if levels >= 4:
        assert np.abs(XW - HV.iteration_matrix()).max() > 1e-6
    else:
        assert np.allclose(XW, HV.iteration_matrix(), atol=1e-12)
    mu = np.linalg.solve(H.Atilde(levels - 1), o.fine_rhs())
    x1 = o.sample(1, 0, x=np.zeros(p.N), noise=False, qoi=False)
    assert np.allclose(x1, (np.eye(p.N) - XW) @ mu, atol=1e-9 * max(1, abs(mu).max()))


def test_ssl_w_cycle_contracts_grid_independently():
    """||X_W||_A of the noise-free W-cycle stays below 1 and nearly constant under
    refinement (Thm. moments-conv), by power iteration (f = 0: the cycle is linear)."""
    rhos = []
    for n, L in ((15, 3), (31, 4), (63, 5)):
        o = oracle.Oracle(2, n, L, kappa2_const=100.0, disc=2, gamma=2)
        v = np.random.default_rng(1).normal(size=n * n)
        lam = 0.0
        for _ in range(40):
            w = o.sample(1, 0, x=v, noise=False, qoi=False)
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        rhos.append(lam)
    assert max(rhos) < 0.9
    assert max(rhos) - min(rhos) < 0.15


def test_ssl_mean_solve_matches_dense_solve():
    p = _problem(31, 4, 6, seed=3)
    o = _oracle(p)
    H = _hier(p)
    mu = np.linalg.solve(H.Atilde(3), o.fine_rhs())
    x, cyc, rr = o.mean_solve(rtol=1e-11, max_cycles=400)
    assert rr <= 1e-11 and cyc < 400
    assert np.allclose(x, mu, atol=1e-8 * abs(mu).max())


def test_w_cycle_one_cycle_law():
    """Lemma MG-iteration-rep for the W-cycle: theta' ~ N(X theta0 + (I - X) mu,
    A~^-1 - X A~^-1 X^T).  Each visit of a coarse grid must draw its own numbers: a
    second visit that reused the first one's would give the wrong covariance (four
    grids: the middle grid is visited twice)."""
    p = _problem(15, 4, 3, seed=5)
    o = _oracle(p)
    H = _hier(p)
    At = H.Atilde(3)
    X = H.iteration_matrix()
    Ai = np.linalg.inv(At)
    mu = Ai @ o.fine_rhs()
    theta0 = np.random.default_rng(3).normal(size=p.N) * 0.5 * np.sqrt(np.diag(Ai))
    mean_exact = X @ theta0 + (np.eye(p.N) - X) @ mu
    cov_exact = Ai - X @ Ai @ X.T
    S = 12000
    draws = np.empty((S, p.N))
    for c in range(S):
        draws[c] = o.sample(1, 991, x=theta0, chain=c, qoi=False)
    mean = draws.mean(0)
    cov = np.cov(draws.T)
    sd = np.sqrt(np.diag(cov_exact))
    assert _z_ok(mean, mean_exact, sd / np.sqrt(S))
    se_cov = np.sqrt((cov_exact ** 2 + np.outer(np.diag(cov_exact), np.diag(cov_exact))) / S)
    iu = np.triu_indices(p.N)
    assert _z_ok(cov[iu], cov_exact[iu], se_cov[iu])


def test_gamma_validation():
    p = _problem(7, 3, 0)
    with pytest.raises(oracle.OracleError):
        _oracle(p, gamma=3)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(3, 7, 2, disc=2)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(2, 7, 2, kappa2=np.ones(49), disc=2)
