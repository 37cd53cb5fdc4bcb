"""GPU parity of the W-cycle (Alg. 1, gamma = 2) and of the squared shifted
Laplacian (Eq. squared_shifted_laplace, 13-point finite differences, Sec. 5.1.1)
against the FP64 CPU oracle, through the C ABI, same seeds and Philox counters.

Tolerance, per site i after the stated number of cycles:
  |x_gpu - x_orc|_i <= tol * max(|x_orc,i|, rms(x_orc)),
  tol = max(1e-11, 20 eps cond),  cond = ((kappa^2 + 8 h^-2) / (kappa^2 + 2 pi^2))^2
for the squared operator (its condition number: largest over smallest eigenvalue
of (kappa^2 - Delta_h)^2).  The library and the oracle assemble the operator by
different routes (stencil product vs ghost-point stencil) and the Galerkin
products in different orders, so the entries differ by rounding (eps = 2^-52
relative); a relative perturbation eps of the operator moves the smooth modes of
the state by up to cond * eps.  1e-11 for the 5-point operator, as in the other
FP64 parity tests."""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs
from tests.test_gpu_parity import _check64, _run_gpu

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _tol(p):
    if p.disc != 2:
        return 1e-11
    h2 = 1.0 / (p.n + 1) ** 2
    cond = ((p.kappa2_const + 8.0 / h2) / (p.kappa2_const + 2.0 * np.pi ** 2)) ** 2
    return max(1e-11, 20.0 * EPS * cond)


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _orc(p, gamma):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const, scale_hd=p.scale_hd,
                         obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                         qoi_w=p.qoi_w, disc=p.disc, gamma=gamma)


def _gpu(p, gamma, **kw):
    from paper_2407_12149_gb300.mgmc import Sampler
    return Sampler(p, precision="fp64", gamma=gamma, **kw)


@pytest.mark.parametrize("n,gamma,cmax", [(31, 2, 0), (63, 2, 0), (63, 1, 0), (127, 2, 0), (127, 2, 1)])
def test_ssl_parity(torch_mod, n, gamma, cmax):
    """The Table 1c posterior (squared shifted Laplacian, 8 ball observations), per site
    after 1, 5 and 40 cycles, QoI series included; 63^2 also as a V-cycle.  cmax = 0: the
    grids up to 63^2 in the one-CTA kernel; 1: every grid on its own launches."""
    p = inputs.table1c(n)
    o = _orc(p, gamma)
    s = _gpu(p, gamma, coarse_max_n=cmax)
    tol = _tol(p)
    for n_steps in (1, 5, 40):
        xo, qo = o.sample(n_steps, 77)
        xg, qg = _run_gpu(torch_mod, s, p, n_steps, 77)
        _check64(xg, xo, tol)
        _check64(qg, qo, tol)
    s.close()


@pytest.mark.parametrize("n,m,nu", [(63, 8, 1), (31, 5, 2), (127, 16, 1)])
def test_sl_w_cycle_parity(torch_mod, n, m, nu):
    """The W-cycle on the 5-point shifted Laplacian with a non-stationary kappa^2 (the
    general path with the W-cycle recursion; nu = 2 uses four visit slots per grid)."""
    p = inputs.make_problem("w", 2, n, kappa2_seed=11, m=m, obs_seed=5, qoi_cells=(n + 1) // 4)
    o = oracle.Oracle(2, p.n, p.n_levels, kappa2=p.kappa2, scale_hd=p.scale_hd, nu1=nu, nu2=nu,
                      obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                      qoi_w=p.qoi_w, gamma=2)
    s = _gpu(p, 2, nu1=nu, nu2=nu)
    for n_steps in (1, 30):
        xo, qo = o.sample(n_steps, 5, step_offset=3, chain=2)
        xg, qg = _run_gpu(torch_mod, s, p, n_steps, 5, step_offset=3, chain=2)
        _check64(xg, xo)
        _check64(qg, qo)
    s.close()


def test_w_cycle_parity_3d(torch_mod):
    """The W-cycle in 3D (15^3, four grids, non-stationary kappa^2, observations): the
    general kernels with the recursion, every grid on its own launches."""
    p = inputs.make_problem("w3", 3, 15, kappa2_seed=4, m=4, obs_seed=3, qoi_cells=4)
    o = _orc(p, 2)
    s = _gpu(p, 2)
    for n_steps in (1, 10):
        xo, qo = o.sample(n_steps, 13)
        xg, qg = _run_gpu(torch_mod, s, p, n_steps, 13)
        _check64(xg, xo)
        _check64(qg, qo)
    s.close()


@pytest.mark.parametrize("disc,n,gamma", [(2, 127, 2), (2, 63, 1), (0, 127, 2), (0, 63, 2)])
def test_small_grid_kernel_is_bitwise_per_launch_path(torch_mod, disc, n, gamma):
    """The one-CTA kernel of the small grids evaluates the per-site functions of the
    one-launch-per-phase path (coarse_max_n = 1); the compiler may contract the
    multiply-adds of the same source differently in the two kernels, so the states agree
    to rounding (the parity tolerance), with far fewer launches; 63^2 runs the whole
    cycle in it."""
    if disc == 2:
        p = inputs.table1c(n)
    else:
        p = inputs.make_problem("w", 2, n, kappa2_seed=3, m=6, obs_seed=2, qoi_cells=(n + 1) // 4)
    a = _gpu(p, gamma, coarse_max_n=1)
    b = _gpu(p, gamma)
    xa, qa = _run_gpu(torch_mod, a, p, 12, 31, step_offset=5)
    xb, qb = _run_gpu(torch_mod, b, p, 12, 31, step_offset=5)
    _check64(xb, xa, _tol(p))
    _check64(qb, qa, _tol(p))
    assert b.launches_per_cycle() < a.launches_per_cycle()
    a.close()
    b.close()


def test_ssl_gibbs_and_mean_solve(torch_mod):
    """The plain Gibbs sampler (Sec. 5.1.3) on the squared operator, and the mean solve
    (noise-free W-cycles to rtol) against the oracle's."""
    p = inputs.table1c(63)
    tol = _tol(p)
    o = _orc(p, 2)
    from paper_2407_12149_gb300.mgmc import Sampler
    g = Sampler(p, precision="fp64", gibbs=True)
    xo, qo = o.sample(25, 9, gibbs=True)
    xg, qg = _run_gpu(torch_mod, g, p, 25, 9)
    _check64(xg, xo, tol)
    _check64(qg, qo, tol)
    g.close()
    s = _gpu(p, 2)
    mu_o, cyc_o, rr_o = o.mean_solve(rtol=1e-10, max_cycles=200)
    mu = torch_mod.zeros(p.N, dtype=torch_mod.float64, device="cuda")
    cyc, rr = s.mean_solve(mu, rtol=1e-10, max_cycles=200)
    assert rr <= 1e-10 and rr_o <= 1e-10
    assert abs(cyc - cyc_o) <= 1
    np.testing.assert_allclose(mu.cpu().numpy(), mu_o, rtol=0, atol=1e-8 * np.abs(mu_o).max())
    s.close()


def test_ssl_full_size_511(torch_mod):
    """Table 1c's largest grid (512 x 512 cells, 9 grids, W-cycle): per site after 3 cycles."""
    p = inputs.table1c(511)
    o = _orc(p, 2)
    s = _gpu(p, 2)
    xo, qo = o.sample(3, 2024)
    xg, qg = _run_gpu(torch_mod, s, p, 3, 2024)
    _check64(xg, xo, _tol(p))
    _check64(qg, qo, _tol(p))
    s.close()


def test_w_cycle_rejections(torch_mod):
    from paper_2407_12149_gb300 import mgmc
    p = inputs.table1c(31)
    with pytest.raises(mgmc.MGMCError):
        mgmc.Sampler(p, precision="fp32")
    q = inputs.make_problem("w", 2, 31, kappa2_seed=1, m=4)
    with pytest.raises(mgmc.MGMCError):
        mgmc.Sampler(q, gamma=3)
    with pytest.raises(mgmc.MGMCError):
        mgmc.BatchSampler([p, p], precision="fp64")
