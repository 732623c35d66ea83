"""Pins of the oracle's state solve, QoI and adjoint gradient (CPU only).

* Banded Jacobian against the matrix-free operator probed column by column.
* Discrete manufactured solution: f := A_h u* + r u*^3 gives back u*.
* Continuum manufactured solution u* = sin(pi x) sin(pi y) with a smooth m: the
  error falls by ~4 per grid refinement (second order).
* Newton converges quadratically; with r = 0 the state is linear in z.
* Adjoint gradient (Sec. 2.3) against central finite differences of Q in z.
"""
import numpy as np
import pytest

from oracle import field, pde
from synthetic_inputs import controls


def _smooth_m(n):
    x = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return 0.3 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y), X, Y


def test_banded_matches_matrix_free():
    n, r = 9, 1.0
    m = field.sample_fields(1, 0, 1, n)[0]
    kx, ky = pde.face_coefficients(m)
    u = np.zeros((n, n))
    u[1:-1, 1:-1] = np.random.default_rng(0).standard_normal((n - 2, n - 2))
    h = 1.0 / (n - 1)
    Jd = pde.jacobian_dense(kx, ky, u, r, h)
    np.testing.assert_allclose(Jd, Jd.T, rtol=0, atol=1e-12 * np.abs(Jd).max())
    ab = pde.jacobian_banded(kx, ky, u, r, h)
    ni = n - 2
    Jb = np.zeros_like(Jd)
    for j in range(ni * ni):
        for i in range(max(0, j - ni), j + 1):
            Jb[i, j] = ab[ni + i - j, j]
            Jb[j, i] = ab[ni + i - j, j]
    np.testing.assert_allclose(Jb, Jd, rtol=0, atol=1e-13 * np.abs(Jd).max())
    # banded Cholesky solve equals the dense solve
    from scipy.linalg import cho_solve_banded, cholesky_banded
    b = np.random.default_rng(1).standard_normal(ni * ni)
    x1 = cho_solve_banded((cholesky_banded(ab), False), b)
    x2 = np.linalg.solve(Jd, b)
    np.testing.assert_allclose(x1, x2, rtol=1e-13, atol=1e-13 * np.abs(x2).max())


def test_discrete_manufactured_solution():
    n, r = 17, 1.0
    h = 1.0 / (n - 1)
    m = field.sample_fields(1, 3, 1, n)[0]
    kx, ky = pde.face_coefficients(m)
    us = np.zeros((n, n))
    us[1:-1, 1:-1] = np.random.default_rng(2).uniform(-1, 1, (n - 2, n - 2))
    f = pde.apply_A(kx, ky, us, h)
    f[1:-1, 1:-1] += r * us[1:-1, 1:-1] ** 3
    u, _ = pde.newton_solve(kx, ky, f, r, h)
    assert np.linalg.norm(u - us) <= 1e-11 * np.linalg.norm(us)


def test_continuum_manufactured_solution_second_order():
    r = 1.0
    errs = []
    for n in (17, 33, 65, 129):
        h = 1.0 / (n - 1)
        m, X, Y = _smooth_m(n)
        us = np.sin(np.pi * X) * np.sin(np.pi * Y)
        mx = 0.6 * np.pi * np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
        my = -0.3 * np.pi * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        f = -np.exp(m) * (mx * ux + my * uy - 2 * np.pi ** 2 * us) + r * us ** 3
        kx, ky = pde.face_coefficients(m)
        u, _ = pde.newton_solve(kx, ky, f, r, h)
        errs.append(np.abs(u - us).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.8) & (ratios < 4.2)), ratios


def test_newton_quadratic_and_zero_rhs():
    n = 33
    prob = pde.Problem(n=n, L=5)
    G = field.control_sources(n, prob.L, prob.width)
    m = field.sample_fields(1, 0, 1, n)[0]
    kx, ky = pde.face_coefficients(m)
    z = 4.0 * controls(5, 1, prob.d_z)[0]       # a strongly nonlinear case
    f = (G @ z).reshape(n, n)
    hist = []
    pde.newton_solve(kx, ky, f, prob.r, prob.h, history=hist)
    hist = np.array(hist) / hist[0]
    # quadratic: once in the asymptotic range, e_{k+1} <= C e_k^2
    k = [i for i in range(1, len(hist) - 1) if 1e-12 < hist[i] < 1e-2]
    assert k, hist
    for i in k:
        assert hist[i + 1] <= 10.0 * hist[i] ** 2 + 1e-13, hist
    u0, _ = pde.newton_solve(kx, ky, np.zeros((n, n)), prob.r, prob.h)
    assert np.all(u0 == 0.0)


def test_linear_superposition_r0():
    n = 17
    prob = pde.Problem(n=n, r=0.0, L=3)
    G = field.control_sources(n, 3, prob.width)
    m = field.sample_fields(1, 0, 1, n)[0]
    kx, ky = pde.face_coefficients(m)
    z = controls(5, 2, 9)
    us = [pde.newton_solve(kx, ky, (G @ zz).reshape(n, n), 0.0, prob.h)[0] for zz in (z[0], z[1], z[0] + z[1])]
    np.testing.assert_allclose(us[2], us[0] + us[1], rtol=0, atol=1e-12 * np.abs(us[2]).max())


@pytest.mark.parametrize("seed_index", [0, 1])
def test_adjoint_gradient_finite_difference(seed_index):
    n = 17
    prob = pde.Problem(n=n, L=3)
    G = field.control_sources(n, prob.L, prob.width)
    ut = field.target_state(n)
    m = field.sample_fields(1, seed_index, 1, n)[0]
    z = controls(5, 1, prob.d_z)[0]
    res = pde.solve_sample(m, z, G, ut, prob)
    step = 1e-5
    fd = np.empty(prob.d_z)
    for k in range(prob.d_z):
        zp, zm = z.copy(), z.copy()
        zp[k] += step
        zm[k] -= step
        qp = pde.solve_sample(m, zp, G, ut, prob, with_adjoint=False).q
        qm = pde.solve_sample(m, zm, G, ut, prob, with_adjoint=False).q
        fd[k] = (qp - qm) / (2 * step)
    assert np.linalg.norm(res.grad - fd) <= 1e-6 * np.linalg.norm(fd)
    # a random direction too
    d = np.random.default_rng(4).standard_normal(prob.d_z)
    qp = pde.solve_sample(m, z + step * d, G, ut, prob, with_adjoint=False).q
    qm = pde.solve_sample(m, z - step * d, G, ut, prob, with_adjoint=False).q
    np.testing.assert_allclose(res.grad @ d, (qp - qm) / (2 * step), rtol=1e-6)


def test_qoi_definition():
    n = 9
    h = 1.0 / (n - 1)
    ut = field.target_state(n)
    u = np.zeros((n, n))
    # Q(0) = 1/2 h^2 sum sin^2 = 1/2 * (discrete) 1/4 for the trapezoid rule on this grid
    q = pde.qoi(u, ut, h)
    np.testing.assert_allclose(q, 0.5 * 0.25, rtol=1e-14)
