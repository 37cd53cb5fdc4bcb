"""Pins of the oracle's Q1 finite-element option (lowest-order conforming
multilinear elements for kappa^2 - Delta, Sec. 5.1.1) against constructions
written from the definition: cell-by-cell assembly with Gauss quadrature
(tests/dense_ref.py), the nesting of the Q1 spaces (V_{l-1} in V_l makes the
Galerkin product P^T A_l P the Q1 matrix of the coarse grid), dense
multigrid, and the moments of the posterior from a dense Cholesky factor."""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs
from tests import dense_ref as dr
from tests.test_oracle_pins import _oracle_X, _stationary_lag_covariances, _stencil_to_dense, _z_ok


def _q1_problem(dim, n, levels, m, kappa2=100.0, seed=3):
    p = inputs.make_problem("q1", dim, n, n_levels=levels, kappa2_const=kappa2, m=m, obs_seed=seed)
    return p


def _oracle(p):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2_const=p.kappa2_const, scale_hd=p.scale_hd,
                         obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                         qoi_w=p.qoi_w, disc=1)


def _hier(p):
    B = dr.B_dense(p.N, p.obs_site, p.obs_w) if p.m else None
    return dr.Hierarchy(p.n, p.dim, p.n_levels, p.kappa2_const, B, p.Gamma, p.scale_hd, disc=1)


@pytest.mark.parametrize("dim,n,scale_hd", [(2, 7, 1), (2, 7, 0), (3, 3, 1), (3, 5, 0)])
def test_q1_fine_operator_equals_quadrature_assembly(dim, n, scale_hd):
    o = oracle.Oracle(dim, n, 1, kappa2_const=37.0, scale_hd=scale_hd, disc=1)
    A = _stencil_to_dense(o.stencil(0), n, dim)
    ref = dr.q1_operator(n, dim, 37.0, scale_hd)
    assert np.allclose(A, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    # the textbook 2D stencil: stiffness (1/3)[-1 -1 -1; -1 8 -1; -1 -1 -1], mass (h^2/36)[1 4 1; 4 16 4; 1 4 1]
    if dim == 2 and scale_hd == 1:
        h2 = 1.0 / (n + 1) ** 2
        c = n // 2 * (n + 1)    # the centre site
        assert A[c, c] == pytest.approx(8.0 / 3.0 + 37.0 * 16.0 * h2 / 36.0, rel=1e-14)
        assert A[c, c + 1] == pytest.approx(-1.0 / 3.0 + 37.0 * 4.0 * h2 / 36.0, rel=1e-14)
        assert A[c, c + n + 1] == pytest.approx(-1.0 / 3.0 + 37.0 * h2 / 36.0, rel=1e-14)


@pytest.mark.parametrize("dim,n,levels", [(2, 15, 3), (3, 7, 2)])
def test_q1_galerkin_levels_are_coarse_q1_matrices(dim, n, levels):
    """Nested Q1 spaces: the oracle's Galerkin grids equal the Q1 matrix of each coarse grid."""
    o = oracle.Oracle(dim, n, levels, kappa2_const=100.0, disc=1)
    nn = n
    for l in range(levels - 1, -1, -1):
        A = _stencil_to_dense(o.stencil(l), nn, dim)
        ref = dr.q1_operator(nn, dim, 100.0)
        assert np.allclose(A, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), l
        nn = (nn - 1) // 2


@pytest.mark.parametrize("dim,n,levels,m", [(2, 15, 3, 4), (3, 7, 2, 3)])
def test_q1_noise_free_cycle_is_dense_multigrid(dim, n, levels, m):
    p = _q1_problem(dim, n, levels, m)
    o = _oracle(p)
    H = _hier(p)
    assert np.allclose(_oracle_X(o, p.N), H.iteration_matrix(), atol=1e-11)


def test_q1_contraction_is_grid_independent():
    """||X||_A of the noise-free Q1 V-cycle (kappa^-1 = 0.1) is bounded independently of h
    (Thm. moments-conv): it rises while kappa^2 h^2 is not small (the mass term helps
    the smoother) and levels off -- 0.117, 0.164, 0.196, 0.209, 0.216 for 15^2 .. 255^2."""
    rhos = []
    for n, L in ((15, 3), (31, 4)):
        p = _q1_problem(2, n, L, 0)
        H = _hier(p)
        rhos.append(dr.a_norm(H.iteration_matrix(), H.Atilde(L - 1)))
    for n, L in ((63, 5), (127, 6), (255, 7)):
        oo = oracle.Oracle(2, n, L, kappa2_const=100.0, disc=1)     # f = 0: the cycle is linear
        v = np.random.default_rng(1).normal(size=n * n)
        lam = 0.0
        for _ in range(40):
            w = oo.sample(1, 0, x=v, noise=False, qoi=False)
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        rhos.append(lam)
    assert max(rhos) < 0.25, rhos
    assert np.all(np.diff(rhos) >= -1e-3) and rhos[-1] - rhos[-2] < 0.01, rhos


def test_q1_invariance_moments_vs_dense_cholesky():
    """Started in N(mu, A~^-1) the Q1 chain stays there: sample mean and covariance
    within 3 SE (each coordinate's closed-form integrated autocorrelation time)."""
    p = _q1_problem(2, 7, 3, 4, seed=8)
    o = _oracle(p)
    H = _hier(p)
    Ai = np.linalg.inv(H.Atilde(2))
    mu = Ai @ o.fine_rhs()
    x = mu + np.linalg.cholesky(Ai) @ np.random.default_rng(5).normal(size=p.N)
    S = 40000
    draws = np.empty((S, p.N))
    for k in range(S):
        x = o.sample(1, 77, x=x, step_offset=k, qoi=False)
        draws[k] = x
    C = _stationary_lag_covariances(H.iteration_matrix(), Ai)
    d = np.diag(Ai)
    tau = 1.0 + 2.0 * sum(np.diag(c) for c in C[1:]) / d
    var_cov = np.outer(d, d) + Ai ** 2 + 2.0 * sum(np.outer(np.diag(c), np.diag(c)) + c * c.T for c in C[1:])
    mean = draws.mean(0)
    assert np.all(np.abs(mean - mu) <= 3.0 * np.sqrt(d * tau / S))
    iu = np.triu_indices(p.N)
    assert _z_ok(np.cov(draws.T)[iu], Ai[iu], np.sqrt(var_cov[iu] / S))


def test_q1_rejects_variable_kappa():
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(2, 7, 2, kappa2=np.full(49, 3.0), disc=1)
