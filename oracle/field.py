"""Random field, control sources and target state (oracle, test infrastructure only).

Grid: n nodes per side on [0,1]^2, x_i = i h, h = 1/(n-1); arrays are (n, n)
indexed [iy, ix] (x fastest).

Random field (Sec. 2, prior N(mbar, C), C = A^-alpha with A = -gamma Lap + delta I,
homogeneous Neumann, alpha = 2; the elliptic example of Sec. 4.2 uses this
Matern class).  Reading of the discretisation: the field lives on the n x n
nodes; Lap is the reflecting-end second difference with spacing h_m = 1/n,
whose eigenvectors are exactly the DCT-II vectors
    v_k(j) = s_k cos(pi k (j + 1/2) / n),   s_0 = sqrt(1/n), s_k = sqrt(2/n),
with eigenvalues -mu_k, mu_k = 4 n^2 sin^2(pi k / (2n)).  The eigenpairs of A
are (lambda_k1k2 = delta + gamma (mu_k1 + mu_k2), v_k1 (x) v_k2), and the
Karhunen-Loeve expansion (Sec. 3.3, KLE = PCA basis of m) of a draw is
    m = mbar + n * sum_{k1,k2} lambda^-1 xi_{k1 k2} v_k1(ix) v_k2(iy),
the factor n making the modes orthonormal in L^2(Omega) (mass 1/n^2 per node).
"""
from __future__ import annotations

import numpy as np

from .philox import field_normals


def dct2_basis(n: int) -> np.ndarray:
    """V[k, j] = s_k cos(pi k (j + 1/2) / n): rows are the orthonormal DCT-II vectors."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    s = np.where(k == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    return s * np.cos(np.pi * k * (j + 0.5) / n)


def neumann_laplacian_1d(n: int) -> np.ndarray:
    """Reflecting-end second difference [1, -2, 1] / h_m^2 with h_m = 1/n (dense, for tests)."""
    L = np.zeros((n, n))
    for j in range(n):
        if j > 0:
            L[j, j - 1] += 1.0
            L[j, j] -= 1.0
        if j < n - 1:
            L[j, j + 1] += 1.0
            L[j, j] -= 1.0
    return L * n * n


def kl_eigenvalues(n: int, gamma: float, delta: float) -> np.ndarray:
    """lam[k2, k1] = delta + gamma (mu_k1 + mu_k2): eigenvalues of A = -gamma Lap + delta I."""
    k = np.arange(n)
    mu = 4.0 * n * n * np.sin(np.pi * k / (2.0 * n)) ** 2
    return delta + gamma * (mu[None, :] + mu[:, None])


def synthesize(xi: np.ndarray, n: int, gamma: float = 0.1, delta: float = 1.0,
               m_mean: float = 0.0) -> np.ndarray:
    """KL synthesis m[s, iy, ix] from normals xi[s, k2, k1] (mode (k1, k2) = (x, y) frequency)."""
    lam = kl_eigenvalues(n, gamma, delta)
    V = dct2_basis(n)
    coef = xi / lam
    # m[iy, ix] = n * sum_{k2,k1} V[k2, iy] coef[k2, k1] V[k1, ix], as two matrix products
    return m_mean + n * (V.T @ coef @ V)


def sample_fields(seed: int, first: int, count: int, n: int, gamma: float = 0.1,
                  delta: float = 1.0, m_mean: float = 0.0) -> np.ndarray:
    """m[s, iy, ix] for global sample indices first .. first+count-1; the normal for
    mode (k1, k2) of sample s is field_normals(...)[s, k2 n + k1]."""
    xi = field_normals(seed, first, count, n * n).reshape(count, n, n)   # [s, k2, k1]
    return synthesize(xi, n, gamma, delta, m_mean)


def control_sources(n: int, L: int, width: float) -> np.ndarray:
    """G[node, j]: the Gaussian sources f_j of Sec. 4.2 on an L x L lattice,
    f_j(x) = exp(-|x - x_j|^2 / (2 sigma^2)) / (sigma sqrt(2 pi)) (the paper's
    normaliser, kept as printed), centres x_j = ((jx+1/2)/L, (jy+1/2)/L),
    control index j = jy L + jx.  Rows are nodes in [iy, ix] order."""
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")          # X[iy, ix] = x_ix
    G = np.empty((n * n, L * L))
    for jy in range(L):
        for jx in range(L):
            cx, cy = (jx + 0.5) / L, (jy + 0.5) / L
            g = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * width ** 2))
            G[:, jy * L + jx] = (g / (width * np.sqrt(2.0 * np.pi))).ravel()
    return G


def target_state(n: int) -> np.ndarray:
    """u_target(x, y) = sin(pi x) sin(pi y) at the nodes, [iy, ix]."""
    x = np.arange(n) / (n - 1)
    return np.sin(np.pi * x)[:, None] * np.sin(np.pi * x)[None, :]
