"""Estimators of the paper's convergence and error experiments (Sec. 5.3) on QoI
traces of many independent chains, and the exact posterior moments of the QoI.

Sec. 5.3.1 (convergence to the target): n chains all start from theta^(0) = 0;
z_j^(m) = F(theta_j^(m)) is the QoI of chain j after m steps.  With the sample
mean mu^(m) and variance (sigma^(m))^2 over the chains at step m,
    R^(m) = |mu^(m) - mu_L| / |mu^(0) - mu_L|,
    Z^(m) = |(sigma^(m))^2 - sigma_L^2| / |(sigma^(0))^2 - sigma_L^2|
(Eq. convergence_rate_definition), and the rates rho = (R^(m*))^(1/m*),
zeta = (Z^(m*))^(1/m*) (Eq. convergence_rate_definitions) at the largest m*
whose statistical error is at most 10 % (m* = 1 when there is none).
Sec. 5.3.3 (root mean squared error): zbar_j^(M) = (1/M) sum_{m<M} z_j^(m) and
Delta^(M) = sqrt((1/n) sum_j (mu_L - zbar_j^(M))^2) (Eq. RMSE_estimator).

mu_L = F^T A~^-1 f and sigma_L^2 = F^T A~^-1 F come from a sparse direct solve
(scipy's LU) with the finest operator the library assembles
(mgmc_fine_operator) plus B Gamma^-1 B^T.  Host code: it post-processes QoI
series the CUDA sampler produced; it runs no step of the sampler.
"""
from __future__ import annotations

import numpy as np


def posterior_operator(problem):
    """A~ = A + B Gamma^-1 B^T (scipy CSR), f = B Gamma^-1 y and the QoI vector F."""
    import scipy.sparse as sp
    from . import mgmc
    p = problem
    st = mgmc.mgmc_fine_operator(p)                      # [N, 3^d]
    N, NS = st.shape
    d = p.dim
    idx = np.arange(N)
    c = [idx % p.n, (idx // p.n) % p.n] + ([idx // (p.n * p.n)] if d == 3 else [])
    rows, cols, vals = [], [], []
    for o in range(NS):
        off = [o % 3 - 1, (o // 3) % 3 - 1] + ([o // 9 - 1] if d == 3 else [])
        nb = [c[a] + off[a] for a in range(d)]
        ok = np.ones(N, bool)
        for a in range(d):
            ok &= (nb[a] >= 0) & (nb[a] < p.n)
        ok &= st[:, o] != 0.0
        j = sum(nb[a] * p.n ** a for a in range(d))
        rows.append(idx[ok])
        cols.append(j[ok])
        vals.append(st[ok, o])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    f = np.zeros(N)
    if p.m:
        B = sp.lil_matrix((N, p.m))
        for k in range(p.m):
            for s, w in zip(p.obs_site[k], p.obs_w[k]):
                if s >= 0:
                    B[s, k] += w
        B = B.tocsr()
        Gi = np.linalg.inv(p.Gamma)
        A = A + B @ sp.csr_matrix(Gi) @ B.T
        f = B @ (Gi @ p.y)
    F = np.zeros(N)
    np.add.at(F, p.qoi_site, p.qoi_w)
    return A.tocsr(), f, F


def exact_qoi_moments(problem):
    """(mu_L, sigma_L^2) of the QoI F^T theta under the posterior N(A~^-1 f, A~^-1)."""
    from scipy.sparse.linalg import splu
    A, f, F = posterior_operator(problem)
    lu = splu(A.tocsc())
    return float(F @ lu.solve(f)), float(F @ lu.solve(F))


def convergence_ratios(z, mu, sigma2):
    """z: [n_chains, steps] QoI of every chain at steps 0, 1, ... (column 0: theta^(0)).
    Returns per step the sample mean and variance over the chains, R and Z with
    their one-standard-error statistical errors (the mean's error sqrt(var / n); the
    variance's var sqrt(2 / (n - 1)), Gaussian QoI)."""
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[0]
    mean = z.mean(axis=0)
    var = z.var(axis=0, ddof=1)
    dmu = abs(mean[0] - mu)
    dvar = abs(var[0] - sigma2)
    R = np.abs(mean - mu) / dmu
    Z = np.abs(var - sigma2) / dvar
    R_err = np.sqrt(var / n) / dmu
    Z_err = var * np.sqrt(2.0 / (n - 1)) / dvar
    return {"mean": mean, "var": var, "R": R, "R_err": R_err, "Z": Z, "Z_err": Z_err}


def rate(ratio, err, max_rel_err=0.1):
    """(ratio^(m*))^(1/m*) with m* the last step m >= 1 before the relative statistical
    error first exceeds max_rel_err (m* = 1 if the error exceeds it at m = 1)."""
    ratio = np.asarray(ratio)
    err = np.asarray(err)
    m_star = 1
    for m in range(1, len(ratio)):
        if not (ratio[m] > 0 and err[m] <= max_rel_err * ratio[m]):
            break
        m_star = m
    return float(ratio[m_star] ** (1.0 / m_star)), m_star


def rmse(z, mu, M_values):
    """Delta^(M) = sqrt(mean_j (mu - zbar_j^(M))^2), zbar_j^(M) the mean of the first M
    QoI values of chain j (steps 0 .. M-1), for each M in M_values."""
    z = np.asarray(z, dtype=np.float64)
    cs = np.cumsum(z, axis=1)
    out = []
    for M in M_values:
        zbar = cs[:, M - 1] / M
        out.append(float(np.sqrt(np.mean((mu - zbar) ** 2))))
    return np.array(out)
