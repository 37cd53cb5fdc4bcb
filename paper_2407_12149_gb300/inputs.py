"""Seeded synthetic problem generators for the MGMC sampler.

This module holds none of the sampler's arithmetic: it only produces the
inputs that define a posterior problem (Sec. 5.1 of the paper) -- the
coefficient field kappa^2(x), observation locations and values, the noise
covariance Gamma, the rows of the observation operator B (point evaluation
of the piecewise multilinear grid function, Eq. B_ell_definition) and the
vector F_L of a box-average quantity of interest (Eq. F_matrix).  Both the
CUDA library and the CPU oracle consume these arrays; neither is imported
here.

Grids: a level with n interior points per axis has vertices at (i + 1) h,
i = 0 .. n-1, h = 1 / (n + 1); zero Dirichlet values sit at i = -1 and i = n.
Site index s = i + n (j + n k) (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


def kappa2_field(n: int, dim: int, seed: int, base: float = 10.0, std: float = 0.5,
                 length: float = 0.1, n_features: int = 512) -> np.ndarray:
    """Non-stationary kappa^2(x) = base * exp(g(x)) on the interior vertices.

    g is a random-Fourier-feature approximation (Rahimi & Recht 2007) of a
    centred Gaussian field with squared-exponential covariance
    std^2 exp(-|x-y|^2 / (2 length^2)):
        g(x) = std sqrt(2/K) sum_k cos(w_k . x + b_k),
        w_k ~ N(0, length^-2 I), b_k ~ U[0, 2 pi).
    Evaluated separably through complex exponentials.  Returns float64 [n^dim].
    """
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0 / length, size=(n_features, dim))
    b = rng.uniform(0.0, 2.0 * np.pi, size=n_features)
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1.0) * h
    ph = [np.exp(1j * np.outer(w[:, a], x)) for a in range(dim)]   # [K, n] per axis
    c = np.exp(1j * b) * std * np.sqrt(2.0 / n_features)
    if dim == 2:
        g = np.real((ph[1].T * c) @ ph[0])                            # [y, x]
    else:
        g = np.empty((n, n, n))
        for kz in range(n):
            g[kz] = np.real((ph[1].T * (c * ph[2][:, kz])) @ ph[0])
    return (base * np.exp(g)).ravel()


def obs_locations(m: int, dim: int, seed: int) -> np.ndarray:
    """m observation points, seeded uniform in (0, 1)^dim."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(m, dim))


def obs_values(m: int, seed: int, lo: float = 1.0, hi: float = 4.0) -> np.ndarray:
    """Observed values y_j in [1, 4] as in Sec. 5.1.2 of the paper."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(lo, hi, size=m)


def point_obs_rows(n: int, dim: int, xyz: np.ndarray):
    """Rows of B for point observations: multilinear interpolation weights.

    For each point the 2^dim vertices of the enclosing cell get the product of
    1D hat-function values; a boundary vertex (zero Dirichlet value) is
    reported as site -1 with weight 0.  Returns (site int32 [m, 2^dim],
    weight float64 [m, 2^dim]); corner order: bit a of the corner index
    selects the upper vertex along axis a.
    """
    xyz = np.atleast_2d(np.asarray(xyz, dtype=np.float64))
    m = xyz.shape[0]
    h = 1.0 / (n + 1)
    nc = 1 << dim
    site = np.full((m, nc), -1, dtype=np.int32)
    wts = np.zeros((m, nc), dtype=np.float64)
    for k in range(m):
        cell = np.minimum(np.floor(xyz[k] / h).astype(np.int64), n)   # vertex index of lower corner
        t = xyz[k] / h - cell
        for corner in range(nc):
            w = 1.0
            idx = []
            for a in range(dim):
                up = (corner >> a) & 1
                v = cell[a] + up                 # vertex index 0 .. n+1
                w *= t[a] if up else (1.0 - t[a])
                idx.append(v - 1)                # interior index
            if all(0 <= i < n for i in idx) and w != 0.0:
                s = idx[0] + n * idx[1] + (n * n * idx[2] if dim == 3 else 0)
                site[k, corner] = s
                wts[k, corner] = w
    return site, wts


def ball_rows(n: int, dim: int, centres: np.ndarray, radius: float, sub: int = 8):
    """Rows of B for averages of the field over balls (Sec. 5.1.2, Eq. observations):
    (1/|B|) int_B phi_i dx for the multilinear hat functions phi_i of the interior
    vertices, by the midpoint rule on a sub-grid of spacing h / sub, normalised by the
    rule's own area inside the ball so that constants are averaged exactly (points
    outside the domain count: the field is 0 there).  Returns (site int32 [m, nnz],
    weight float64 [m, nnz]); rows are padded with site -1, weight 0."""
    centres = np.atleast_2d(np.asarray(centres, dtype=np.float64))
    h = 1.0 / (n + 1)
    d = h / sub
    rows = []
    for c in centres:
        lo = np.floor((c - radius) / d).astype(int)
        hi = np.ceil((c + radius) / d).astype(int)
        axes = [(np.arange(lo[a], hi[a]) + 0.5) * d for a in range(dim)]
        pts = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
        pts = pts[np.sum((pts - c) ** 2, axis=1) <= radius ** 2]
        npts = len(pts)
        pts = pts[np.all((pts > 0.0) & (pts < 1.0), axis=1)]
        acc = {}
        for q in pts:
            cell = np.floor(q / h).astype(np.int64)
            t = q / h - cell
            for corner in range(1 << dim):
                w, idx, ok = 1.0, 0, True
                for a in range(dim):
                    up = (corner >> a) & 1
                    w *= t[a] if up else 1.0 - t[a]
                    v = cell[a] + up - 1          # interior index of the vertex
                    ok = ok and 0 <= v < n
                    idx += v * n ** a
                if ok and w > 0.0:
                    acc[idx] = acc.get(idx, 0.0) + w
        rows.append({i: w / npts for i, w in acc.items()})
    nnz = max(1, max(len(r) for r in rows))
    site = np.full((len(rows), nnz), -1, dtype=np.int32)
    wts = np.zeros((len(rows), nnz), dtype=np.float64)
    for k, acc in enumerate(rows):
        for t, (i, w) in enumerate(sorted(acc.items())):
            site[k, t] = i
            wts[k, t] = w
    return site, wts


def qoi_box(n: int, dim: int, c0: int, c1: int):
    """F_L for the average of the multilinear interpolant over the box
    [c0 h, c1 h]^dim (c0 < c1 are vertex indices of grid lines).

    Exact for piecewise multilinear functions: vertex weight = product of 1D
    trapezoid weights (1/2 on the box faces, 1 inside) / (c1 - c0)^dim.
    Returns (site int32, weight float64) over the interior vertices with
    nonzero weight.
    """
    if not (0 <= c0 < c1 <= n + 1):
        raise ValueError("box outside the grid")
    w1 = np.zeros(n)
    for v in range(c0, c1 + 1):
        i = v - 1
        if 0 <= i < n:
            w1[i] = 0.5 if v in (c0, c1) else 1.0
    w1 /= (c1 - c0)
    if dim == 2:
        W = np.outer(w1, w1)                       # [j, i]
    else:
        W = np.einsum("k,j,i->kji", w1, w1, w1)
    flat = W.ravel()
    sites = np.nonzero(flat)[0].astype(np.int32)
    return sites, flat[sites].copy()


def central_box(n: int, cells: int):
    """Vertex-line indices of the central box of `cells` cells per axis."""
    ncell = n + 1
    c0 = (ncell - cells) // 2
    return c0, c0 + cells


@dataclass
class Problem:
    """A posterior problem N(A~^-1 f, A~^-1) on one grid (Sec. 5.1)."""
    name: str
    dim: int
    n: int
    n_levels: int
    kappa2: Optional[np.ndarray]          # float64 [n^dim] or None
    kappa2_const: float = 10.0
    obs_site: Optional[np.ndarray] = None # int32 [m, 2^dim]
    obs_w: Optional[np.ndarray] = None    # float64 [m, 2^dim]
    Gamma: Optional[np.ndarray] = None    # float64 [m, m]
    y: Optional[np.ndarray] = None        # float64 [m]
    qoi_site: Optional[np.ndarray] = None
    qoi_w: Optional[np.ndarray] = None
    scale_hd: int = 1
    disc: int = 0                         # 0 finite differences, 1 Q1 finite elements, 2 squared shifted
                                          # Laplacian (13-point finite differences; 1 and 2 constant kappa^2)
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return 0 if self.obs_site is None else int(self.obs_site.shape[0])

    @property
    def N(self) -> int:
        return self.n ** self.dim


def levels_for(n: int, coarsest: int = 1) -> int:
    """Number of grids n -> (n-1)/2 -> ... down to `coarsest` points per axis."""
    L, nn = 1, n
    while nn > coarsest:
        if (nn - 1) % 2:
            raise ValueError("n must be 2^k - 1")
        nn = (nn - 1) // 2
        L += 1
    if nn != coarsest:
        raise ValueError("coarsest size not reachable")
    return L


def make_problem(name: str, dim: int, n: int, *, n_levels: Optional[int] = None,
                 coarsest: int = 1, kappa2_seed: Optional[int] = None, kappa2_const: float = 10.0,
                 m: int = 0, obs_seed: int = 1, sigma2: float = 1e-4, qoi_cells: Optional[int] = None,
                 scale_hd: int = 1, disc: int = 0, gamma_range: Optional[tuple] = None,
                 ball_radius: Optional[float] = None) -> Problem:
    """Assemble a seeded problem.  kappa2_seed=None gives constant kappa^2.  disc = 1: Q1
    finite elements (constant kappa^2 only).  gamma_range = (lo, hi): Gamma diagonal with
    seeded entries uniform in [lo, hi] instead of sigma2 I.  ball_radius: observations
    and QoI are averages over balls of that radius (the QoI centred in the domain)
    instead of point values and the central box."""
    if disc in (1, 2) and kappa2_seed is not None:
        raise ValueError("the Q1 and squared-operator discretisations take a constant kappa^2")
    if disc == 2 and dim != 2:
        raise ValueError("the squared shifted Laplacian is two-dimensional")
    if n_levels is None:
        n_levels = levels_for(n, coarsest)
    k2 = None if kappa2_seed is None else kappa2_field(n, dim, kappa2_seed)
    p = Problem(name=name, dim=dim, n=n, n_levels=n_levels, kappa2=k2, kappa2_const=kappa2_const,
                scale_hd=scale_hd, disc=disc)
    if m > 0:
        xyz = obs_locations(m, dim, obs_seed)
        if ball_radius is None:
            p.obs_site, p.obs_w = point_obs_rows(n, dim, xyz)
        else:
            p.obs_site, p.obs_w = ball_rows(n, dim, xyz, ball_radius)
        if gamma_range is None:
            p.Gamma = sigma2 * np.eye(m)
        else:
            g = np.random.default_rng(1_000_003 + obs_seed).uniform(gamma_range[0], gamma_range[1], m)
            p.Gamma = np.diag(g)
        p.y = obs_values(m, obs_seed)
        p.meta["obs_xyz"] = xyz
    if ball_radius is not None:
        qs, qw = ball_rows(n, dim, np.full((1, dim), 0.5), ball_radius)
        keep = qs[0] >= 0
        p.qoi_site, p.qoi_w = qs[0][keep], qw[0][keep]
        p.meta["qoi_ball"] = ball_radius
    elif qoi_cells is not None:
        c0, c1 = central_box(n, qoi_cells)
        p.qoi_site, p.qoi_w = qoi_box(n, dim, c0, c1)
        p.meta["qoi_box"] = (c0, c1)
    return p


def config1() -> Problem:
    """Plain MGMC, 31^2, kappa^2 = 10, no observations, 4 grids, QoI central 8x8 cells."""
    return make_problem("plain-2d-31", 2, 31, n_levels=4, kappa2_const=10.0, qoi_cells=8)


def config2(n: int = 1023, n_levels: Optional[int] = None) -> Problem:
    """Bayesian 2D, non-stationary kappa^2, 16 point observations, Gamma = 1e-4 I."""
    return make_problem(f"bayes-2d-{n}", 2, n, n_levels=n_levels, kappa2_seed=2024, m=16, obs_seed=1,
                        qoi_cells=max(2, (46 * (n + 1)) // 1024))


def table1a(n: int, n_levels: Optional[int] = None) -> Problem:
    """The setting of the paper's Table 1a (Sec. 5.1): the Q1 finite-element shifted
    Laplacian with correlation length kappa^-1 = 0.1, 8 observations whose variances are
    uniform in [1e-6, 2e-6], observed values in [1, 4]; the observations are averages over
    balls of radius 0.025 at seeded locations, and the QoI is the
    average over the ball of the same radius at the centre of the domain (Eq.
    measurement_definition)."""
    return make_problem(f"table1a-q1-{n}", 2, n, n_levels=n_levels, kappa2_const=100.0, m=8, obs_seed=11,
                        disc=1, gamma_range=(1e-6, 2e-6), ball_radius=0.025)


def table1c(n: int, n_levels: Optional[int] = None) -> Problem:
    """The setting of the paper's Table 1c (Sec. 5.1): the squared shifted Laplacian
    (kappa^2 - Delta)^2 with kappa^-1 = 0.1 in 2D, 13-point finite differences with
    u = du/dn = 0, and the observations and QoI of Table 1a (8 averages over balls of
    radius 0.025, variances uniform in [1e-6, 2e-6], values in [1, 4]); the paper samples
    it with a W-cycle."""
    return make_problem(f"table1c-ssl-{n}", 2, n, n_levels=n_levels, kappa2_const=100.0, m=8, obs_seed=11,
                        disc=2, gamma_range=(1e-6, 2e-6), ball_radius=0.025)


def config3(n: int = 127, n_levels: Optional[int] = None) -> Problem:
    """Bayesian 3D, kappa^2 = 25, 32 point observations, coarsest 3^3, QoI central 16^3 cells."""
    return make_problem(f"bayes-3d-{n}", 3, n, n_levels=n_levels, coarsest=3 if n_levels is None else 1,
                        kappa2_const=25.0, m=32, obs_seed=3,
                        qoi_cells=max(2, (16 * (n + 1)) // 128))
