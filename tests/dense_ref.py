"""Dense-matrix constructions written from the definitions, used to pin the oracle.

Everything here is built from the problem definition with dense linear
algebra (numpy solves / Cholesky) rather than sweeps or stencils, so that it
shares no code path with the oracle:
  - A_L from the finite-difference formula s (kappa^2 I - Delta_h), or the Q1
    finite-element matrix assembled by quadrature over the cells;
  - P from the coarse hat functions evaluated at the fine vertices (Sec. 5.1.3);
  - A_{l-1} = P^T A_l P and B_{l-1} = P^T B_l (Eq. A_ell_1_B_ell_1);
  - the forward/backward low-rank Gibbs splittings M~ = D + L + B Gamma^-1 B^T
    (Eq. M_lowrank_gibbs) with L the strictly lower part in colour order;
  - the squared shifted Laplacian as the matrix square of the shifted
    5-point operator plus the diagonal boundary term of u = du/dn = 0;
  - the deterministic V- and W-cycle iteration matrices X_L (Lemma
    MG-iteration-rep).
"""
import numpy as np


def fd_operator(n, d, kappa2, scale_hd=1):
    h = 1.0 / (n + 1)
    N = n ** d
    k2 = np.broadcast_to(np.asarray(kappa2, dtype=float), (N,)) if np.ndim(kappa2) == 0 else np.asarray(kappa2)
    s = h ** d if scale_hd else 1.0
    # 1D second-difference matrix and Kronecker sums: -Delta_h = sum_a I x T x I
    T = (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / (h * h)
    I = np.eye(n)
    if d == 2:
        lap = np.kron(I, T) + np.kron(T, I)
    else:
        lap = np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I) + np.kron(np.kron(T, I), I)
    return s * (lap + np.diag(k2))


def ssl_operator(n, kappa2, scale_hd=1):
    """Squared shifted Laplacian (kappa^2 - Delta)^2 in 2D with u = du/dn = 0, as a matrix
    product: s [(kappa^2 I + L)^2 + 2 h^-4 E] with L = -Delta_h the 5-point Dirichlet matrix
    and E the diagonal that counts, per vertex, the boundary sides it is adjacent to
    (the clamped-plate correction of the 13-point stencil: the mirror ghost behind a
    boundary vertex adds h^-4 where L^2 lacks h^-4 from the dropped boundary row)."""
    h = 1.0 / (n + 1)
    L = fd_operator(n, 2, 0.0, scale_hd=0)
    K = kappa2 * np.eye(n * n) + L
    idx = np.arange(n * n)
    i, j = idx % n, idx // n
    E = np.diag((i == 0).astype(float) + (i == n - 1) + (j == 0) + (j == n - 1))
    s = h * h if scale_hd else 1.0
    return s * (K @ K + 2.0 / h ** 4 * E)


def q1_operator(n, d, kappa2, scale_hd=1):
    """Q1 finite-element matrix of kappa^2 - Delta (constant kappa^2, zero Dirichlet
    values) assembled cell by cell with a 3-point Gauss-Legendre rule per axis (exact
    for the products of multilinear functions), from the nodal hat functions of the
    (n+1)^d cells of the unit square / cube; boundary vertices are dropped."""
    h = 1.0 / (n + 1)
    gx, gw = np.polynomial.legendre.leggauss(3)
    qx, qw = 0.5 * (gx + 1.0), 0.5 * gw                     # on [0, 1]
    corners = np.array(np.meshgrid(*[[0, 1]] * d, indexing="ij")).reshape(d, -1).T   # (2^d, d)
    pts = np.array(np.meshgrid(*[qx] * d, indexing="ij")).reshape(d, -1).T
    wts = np.prod(np.array(np.meshgrid(*[qw] * d, indexing="ij")).reshape(d, -1).T, axis=1)
    # local basis values and reference gradients at the quadrature points
    val = np.ones((len(corners), len(pts)))
    grad = np.ones((len(corners), len(pts), d))
    for c, cor in enumerate(corners):
        for a in range(d):
            f = pts[:, a] if cor[a] else 1.0 - pts[:, a]
            df = 1.0 if cor[a] else -1.0
            val[c] *= f
            for b in range(d):
                grad[c, :, b] *= df if b == a else f
    K_loc = np.einsum("ipk,jpk,p->ij", grad, grad, wts) * h ** (d - 2)
    M_loc = np.einsum("ip,jp,p->ij", val, val, wts) * h ** d
    loc = K_loc + kappa2 * M_loc
    N = n ** d
    A = np.zeros((N, N))
    for cell in np.ndindex(*([n + 1] * d)):
        gidx = []
        for cor in corners:
            v = [cell[a] + cor[a] - 1 for a in range(d)]     # interior index of the corner vertex
            gidx.append(-1 if min(v) < 0 or max(v) >= n else sum(v[a] * n ** a for a in range(d)))
        for i, gi in enumerate(gidx):
            if gi < 0:
                continue
            for j, gj in enumerate(gidx):
                if gj >= 0:
                    A[gi, gj] += loc[i, j]
    return A if scale_hd else A / h ** d


def prolongation_1d(nc):
    """Coarse hat functions (width 2H, H = 2h) sampled at the fine interior vertices."""
    nf = 2 * nc + 1
    hf = 1.0 / (nf + 1)
    H = 2.0 * hf
    xf = (np.arange(nf) + 1.0) * hf
    Xc = (np.arange(nc) + 1.0) * H
    return np.maximum(0.0, 1.0 - np.abs(xf[:, None] - Xc[None, :]) / H)


def prolongation(nc, d):
    P1 = prolongation_1d(nc)
    if d == 2:
        return np.kron(P1, P1)
    return np.kron(np.kron(P1, P1), P1)


def colour_order(n, d, radius=1):
    """Sites in colour-major order (the parity-colour reading; radius-2 stencils: the
    nine classes (i mod 3, j mod 3) by code (i mod 3) + 3 (j mod 3)), lexicographic inside."""
    idx = np.arange(n ** d)
    if radius == 2:
        code = (idx % n) % 3 + 3 * ((idx // n) % 3)
        return np.concatenate([idx[code == c] for c in range(9)])
    if d == 2:
        seq = [(0, 0), (1, 1), (0, 1), (1, 0)]
    else:
        seq = [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0), (1, 1, 1)]
    coords = [idx % n, (idx // n) % n] + ([idx // (n * n)] if d == 3 else [])
    perm = []
    for c in seq:
        mask = np.ones(n ** d, bool)
        for a in range(d):
            mask &= (coords[a] % 2) == c[a]
        perm.extend(idx[mask].tolist())
    return np.array(perm)


def B_dense(N, obs_site, obs_w):
    m = obs_site.shape[0]
    B = np.zeros((N, m))
    for k in range(m):
        for s, w in zip(obs_site[k], obs_w[k]):
            if s >= 0:
                B[s, k] += w
    return B


class Hierarchy:
    """Dense operators of every level, index 0 = coarsest."""

    def __init__(self, n, d, n_levels, kappa2, B=None, Gamma=None, scale_hd=1, disc=0, gamma=1):
        self.d = d
        self.radius = 2 if disc == 2 else 1
        self.gamma = gamma
        self.A = [None] * n_levels
        self.B = [None] * n_levels
        self.P = [None] * n_levels     # P[l]: level l-1 -> l
        self.n = [None] * n_levels
        if disc == 2:
            A = ssl_operator(n, kappa2, scale_hd)
        elif disc == 1:
            A = q1_operator(n, d, kappa2, scale_hd)
        else:
            A = fd_operator(n, d, kappa2, scale_hd)
        self.A[-1] = A
        self.B[-1] = B if B is not None else np.zeros((n ** d, 0))
        self.n[-1] = n
        nn = n
        for l in range(n_levels - 1, 0, -1):
            nc = (nn - 1) // 2
            P = prolongation(nc, d)
            self.P[l] = P
            self.A[l - 1] = P.T @ self.A[l] @ P
            self.B[l - 1] = P.T @ self.B[l]
            self.n[l - 1] = nc
            nn = nc
        m = self.B[-1].shape[1]
        self.Gamma = Gamma if Gamma is not None else np.zeros((0, 0))
        self.Gi = np.linalg.inv(self.Gamma) if m else np.zeros((0, 0))
        self.m = m

    def Atilde(self, l):
        return self.A[l] + self.B[l] @ self.Gi @ self.B[l].T

    def splitting(self, l, direction):
        """M~ of Eq. M_lowrank_gibbs (omega = 1) in natural site order."""
        A = self.A[l]
        perm = colour_order(self.n[l], self.d, self.radius)
        Ap = A[np.ix_(perm, perm)]
        Mp = np.tril(Ap) if direction == 0 else np.triu(Ap)
        M = np.zeros_like(A)
        M[np.ix_(perm, perm)] = Mp
        return M + self.B[l] @ self.Gi @ self.B[l].T

    def smoother_matrix(self, l, direction):
        M = self.splitting(l, direction)
        return np.eye(M.shape[0]) - np.linalg.solve(M, self.Atilde(l))

    def iteration_matrix(self, l=None):
        """X_l of the noise-free (1,1)-cycle with exact coarsest solve: the coarse
        correction of level l applies the coarse cycle gamma_l times from zero,
        psi = (I - X_{l-1}^gamma_l) A~_{l-1}^-1 P^T r, with gamma_L = 1 on the finest
        level and gamma_l = gamma below (Alg. 1)."""
        if l is None:
            l = len(self.A) - 1
        At = self.Atilde(l)
        N = At.shape[0]
        if l == 0:
            return np.zeros((N, N))
        P = self.P[l]
        Ac = self.Atilde(l - 1)
        Xc = self.iteration_matrix(l - 1)
        reps = 1 if l == len(self.A) - 1 else self.gamma
        Xg = np.linalg.matrix_power(Xc, reps)
        cgc = np.eye(N) - P @ (np.eye(Ac.shape[0]) - Xg) @ np.linalg.solve(Ac, P.T @ At)
        return self.smoother_matrix(l, 1) @ cgc @ self.smoother_matrix(l, 0)


def a_norm(X, A):
    w, V = np.linalg.eigh(A)
    Ah = (V * np.sqrt(w)) @ V.T
    Aih = (V / np.sqrt(w)) @ V.T
    return np.linalg.norm(Ah @ X @ Aih, 2)
