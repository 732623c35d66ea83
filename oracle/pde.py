"""Semilinear elliptic state equation, QoI and adjoint gradient (oracle, test infrastructure only).

State equation (Sec. 4.2):  -div(e^m grad u) + r u^3 = sum_j z_j f_j on (0,1)^2,
u = 0 on the boundary.  Discretised by the 5-point finite-volume stencil on
the vertex grid x_i = i h, h = 1/(n-1), unknowns at the interior nodes:

  (A_h u)_P = [ k_E (u_P - u_E) + k_W (u_P - u_W) + k_N (u_P - u_N) + k_S (u_P - u_S) ] / h^2,

with face coefficient k between nodes a, b equal to exp((m_a + m_b)/2).
Residual R(u) = A_h u + r u^3 - f (Sec. 2, R(u, m, z) = 0 with f = G z), its
u-Jacobian J = A_h + diag(3 r u^2) is symmetric positive definite.

Newton: u0 = 0, full steps, backtracking (halving, at most 10) only when the
residual norm grows; stop once ||R||_2 <= rtol ||f||_2 and take one more step.
Every linear solve is a banded Cholesky factorisation of J (a direct solve,
as the paper uses direct solvers, Sec. 4), reused for the adjoint.

QoI (Sec. 4.2, tracking type, with a factor 1/2):  Q(u) = 1/2 h^2 sum_interior (u - u_t)^2.
Adjoint (Sec. 2.3): J lam = dQ/du = h^2 (u - u_t); since dR/dz = -G,
grad_z Q = G^T lam.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import cho_solve_banded, cholesky_banded


@dataclass
class Problem:
    n: int
    r: float = 1.0
    gamma: float = 0.1
    delta: float = 1.0
    m_mean: float = 0.0
    L: int = 5
    width: float = 0.05
    newton_rtol: float = 1e-10
    newton_maxit: int = 30

    @property
    def h(self) -> float:
        return 1.0 / (self.n - 1)

    @property
    def d_z(self) -> int:
        return self.L * self.L


def face_coefficients(m: np.ndarray):
    """kx[iy, ix] on the face between (ix, iy) and (ix+1, iy), shape (n, n-1);
    ky[iy, ix] on the face between (ix, iy) and (ix, iy+1), shape (n-1, n)."""
    kx = np.exp(0.5 * (m[:, :-1] + m[:, 1:]))
    ky = np.exp(0.5 * (m[:-1, :] + m[1:, :]))
    return kx, ky


def apply_A(kx, ky, u: np.ndarray, h: float) -> np.ndarray:
    """(A_h u) at the interior nodes, returned as a full (n, n) array with zero boundary;
    u is a full (n, n) array whose boundary values are taken as given (zero for the PDE)."""
    out = np.zeros_like(u)
    c = u[1:-1, 1:-1]
    out[1:-1, 1:-1] = (kx[1:-1, 1:] * (c - u[1:-1, 2:]) + kx[1:-1, :-1] * (c - u[1:-1, :-2])
                       + ky[1:, 1:-1] * (c - u[2:, 1:-1]) + ky[:-1, 1:-1] * (c - u[:-2, 1:-1])) / h ** 2
    return out


def residual(kx, ky, u, f, r, h):
    """R(u) = A_h u + r u^3 - f at the interior nodes (boundary entries zero)."""
    R = apply_A(kx, ky, u, h)
    R[1:-1, 1:-1] += r * u[1:-1, 1:-1] ** 3 - f[1:-1, 1:-1]
    return R


def jacobian_banded(kx, ky, u, r, h):
    """Upper banded storage (scipy convention, bandwidth n-2) of J = A_h + diag(3 r u^2)
    over the interior unknowns ordered p = (iy-1)(n-2) + (ix-1)."""
    n = u.shape[0]
    ni = n - 2
    d = ni * ni
    ab = np.zeros((ni + 1, d))
    diag = (kx[1:-1, 1:] + kx[1:-1, :-1] + ky[1:, 1:-1] + ky[:-1, 1:-1]) / h ** 2 + 3.0 * r * u[1:-1, 1:-1] ** 2
    ab[ni, :] = diag.ravel()
    # east neighbour: entry (p, p+1) for ix < n-2; stored at row ni-1, column p+1
    east = (-kx[1:-1, 1:-1] / h ** 2)                     # faces between interior ix and ix+1, (ni, ni-1)
    e = np.zeros((ni, ni))
    e[:, 1:] = east
    ab[ni - 1, :] = e.ravel()
    # north neighbour: entry (p, p+ni); stored at row 0, column p+ni
    north = -ky[1:-1, 1:-1] / h ** 2                      # faces between interior iy and iy+1, (ni-1, ni)
    nb = np.zeros((ni, ni))
    nb[1:, :] = north
    ab[0, :] = nb.ravel()
    return ab


def jacobian_dense(kx, ky, u, r, h):
    """J assembled column by column from the matrix-free operator (for pins only)."""
    n = u.shape[0]
    ni = n - 2
    d = ni * ni
    J = np.empty((d, d))
    e = np.zeros((n, n))
    for p in range(d):
        iy, ix = divmod(p, ni)
        e[1 + iy, 1 + ix] = 1.0
        col = apply_A(kx, ky, e, h)
        col[1:-1, 1:-1] += 3.0 * r * u[1:-1, 1:-1] ** 2 * e[1:-1, 1:-1]
        J[:, p] = col[1:-1, 1:-1].ravel()
        e[1 + iy, 1 + ix] = 0.0
    return J


class NotConverged(RuntimeError):
    pass


def newton_solve(kx, ky, f, r, h, rtol=1e-10, maxit=30, history=None):
    """Solve A_h u + r u^3 = f (Dirichlet zero).  Returns (u, cholesky factor of J(u))."""
    n = f.shape[0]
    u = np.zeros((n, n))
    fnorm = np.linalg.norm(f[1:-1, 1:-1])
    R = residual(kx, ky, u, f, r, h)
    rn = np.linalg.norm(R)
    extra_done = False
    for it in range(maxit + 1):
        if history is not None:
            history.append(rn)
        if rn <= rtol * fnorm:
            if extra_done or fnorm == 0.0:
                break
            extra_done = True
        elif it == maxit:
            raise NotConverged(f"Newton: ||R|| = {rn:.3e} after {maxit} steps")
        c = cholesky_banded(jacobian_banded(kx, ky, u, r, h), lower=False)
        du = cho_solve_banded((c, False), -R[1:-1, 1:-1].ravel()).reshape(n - 2, n - 2)
        step = 1.0
        for _ in range(11):
            un = u.copy()
            un[1:-1, 1:-1] += step * du
            Rn = residual(kx, ky, un, f, r, h)
            rnn = np.linalg.norm(Rn)
            if rnn <= rn or step < 2.0 ** -9:
                break
            step *= 0.5
        u, R, rn = un, Rn, rnn
        if extra_done:
            if history is not None:
                history.append(rn)
            break
    c = cholesky_banded(jacobian_banded(kx, ky, u, r, h), lower=False)
    return u, c


def qoi(u, u_t, h):
    """Q = 1/2 h^2 sum over interior nodes of (u - u_t)^2."""
    d = u[1:-1, 1:-1] - u_t[1:-1, 1:-1]
    return 0.5 * h * h * float(np.sum(d * d))


def qoi_du(u, u_t, h):
    """dQ/du at the interior nodes, (n-2, n-2)."""
    return h * h * (u[1:-1, 1:-1] - u_t[1:-1, 1:-1])


def adjoint_solve(chol, rhs_int):
    """Solve J lam = rhs with the Cholesky factor of J (J symmetric, so J^T = J)."""
    ni = rhs_int.shape[0]
    return cho_solve_banded((chol, False), rhs_int.ravel()).reshape(ni, ni)


def interior_rows(G, n):
    """Rows of G (nodes in [iy, ix] order) that belong to interior nodes."""
    return G.reshape(n, n, -1)[1:-1, 1:-1, :].reshape((n - 2) ** 2, -1)


@dataclass
class SampleResult:
    u: np.ndarray       # (n, n)
    q: float
    lam: np.ndarray     # (n-2, n-2)
    grad: np.ndarray    # (d_z,)


def solve_sample(m, z, G, u_t, prob: Problem, with_adjoint=True):
    """State solve, QoI and adjoint gradient for one field m and control z."""
    n, h = prob.n, prob.h
    kx, ky = face_coefficients(m)
    f = (G @ z).reshape(n, n)
    u, chol = newton_solve(kx, ky, f, prob.r, h, prob.newton_rtol, prob.newton_maxit)
    q = qoi(u, u_t, h)
    if not with_adjoint:
        return SampleResult(u, q, None, None)
    lam = adjoint_solve(chol, qoi_du(u, u_t, h))
    grad = interior_rows(G, n).T @ lam.ravel()
    return SampleResult(u, q, lam, grad)


def solve_batch(ms, z, G, u_t, prob: Problem, with_adjoint=True, z_per_sample=False):
    """Loop over samples (z shared unless z_per_sample)."""
    out = []
    for i in range(ms.shape[0]):
        zi = z[i] if z_per_sample else z
        out.append(solve_sample(ms[i], zi, G, u_t, prob, with_adjoint))
    return out


def state_jacobian_columns(chol, G_int, n):
    """du/dz = J^{-1} G (the linearised solves of Sec. 3.4, forward route), (d, d_z)."""
    return cho_solve_banded((chol, False), G_int)


def projected_jacobian(chol, G_int, Phi, h, route="forward"):
    """Y = Phi^T M J^{-1} G (M = h^2 I), the reduced control Jacobian of Sec. 3.4, (r_u, d_z).
    Forward route: the d_z solves J X = G, then Phi^T M X.  Adjoint route: the r_u solves
    J Lam = M Phi (J symmetric), then Lam^T G."""
    if route == "forward":
        return h * h * (Phi.T @ cho_solve_banded((chol, False), G_int))
    lam = cho_solve_banded((chol, False), h * h * Phi)
    return lam.T @ G_int
