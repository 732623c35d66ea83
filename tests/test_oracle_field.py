"""Pins of the oracle's random-field pieces (CPU only).

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* Box-Muller normals: moments and a Kolmogorov-Smirnov test.
* KL basis (Sec. 2, C = (-gamma Lap + delta I)^-2 with Neumann ends): the DCT-II
  vectors and closed-form eigenvalues against a dense eigendecomposition of the
  assembled operator on tiny grids, including eigenspace projectors inside
  degenerate clusters.
* Synthesised fields: empirical covariance against n^2 A^-2 (L^2-normalised KL).
* Control sources: closed-form value at a lattice centre and the lattice order.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import field, philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(np.array(r[0:4], dtype=np.uint64), np.array(r[4:6], dtype=np.uint64))
        assert [int(v) for v in out] == r[6:10]


def test_uniform52_range_and_exactness():
    a = np.array([0, 0xFFFFFFFF, 0x12345678], dtype=np.uint64)
    b = np.array([0, 0xFFFFFFFF, 0x9ABCDEF0], dtype=np.uint64)
    u = philox.uniform52(a, b)
    assert u[0] == 0.5 * 2.0 ** -52
    assert u[1] == 1.0 - 0.5 * 2.0 ** -52
    assert np.all((u > 0) & (u < 1))


def test_normals_distribution():
    xi = philox.field_normals(seed=11, first_sample=0, n_samples=40, n_modes=5001).ravel()
    assert abs(xi.mean()) < 4.0 / np.sqrt(xi.size)
    assert abs(xi.var() - 1.0) < 4.0 * np.sqrt(2.0 / xi.size)
    assert stats.kstest(xi, "norm").pvalue > 1e-3
    # odd mode count: last block's second normal is dropped, the rest are unchanged
    a = philox.field_normals(3, 5, 2, 7)
    b = philox.field_normals(3, 5, 2, 8)
    np.testing.assert_array_equal(a, b[:, :7])
    # counters are per sample: a subset reproduces the same rows
    c = philox.field_normals(3, 6, 1, 8)
    np.testing.assert_array_equal(c[0], b[1])


def _dense_A(n, gamma, delta):
    L1 = field.neumann_laplacian_1d(n)
    I = np.eye(n)
    lap = np.kron(I, L1) + np.kron(L1, I)     # flat index iy*n + ix: kron(I, L1) acts on ix
    return delta * np.eye(n * n) - gamma * lap


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_kl_eigenpairs_against_dense(n):
    gamma, delta = 0.1, 1.0
    A = _dense_A(n, gamma, delta)
    lam = field.kl_eigenvalues(n, gamma, delta)
    V = field.dct2_basis(n)
    np.testing.assert_allclose(V @ V.T, np.eye(n), atol=1e-13)
    # every closed-form pair is an eigenpair of the assembled operator
    scale = np.abs(A).max()
    for k2 in range(n):
        for k1 in range(n):
            v = np.outer(V[k2], V[k1]).ravel()
            np.testing.assert_allclose(A @ v, lam[k2, k1] * v, atol=1e-12 * scale)
    # the spectra agree, and so do the eigenspaces (cluster projectors)
    ev, U = np.linalg.eigh(A)
    np.testing.assert_allclose(np.sort(lam.ravel()), ev, rtol=1e-12, atol=1e-12 * scale)
    flat = lam.ravel()
    B = np.stack([np.outer(V[q // n], V[q % n]).ravel() for q in range(n * n)], axis=1)
    for val in np.unique(np.round(ev, 8)):
        sel_dense = np.abs(ev - val) < 1e-8 * max(1.0, val)
        sel_cf = np.abs(flat - val) < 1e-8 * max(1.0, val)
        assert sel_dense.sum() == sel_cf.sum()
        P1 = U[:, sel_dense] @ U[:, sel_dense].T
        P2 = B[:, sel_cf] @ B[:, sel_cf].T
        np.testing.assert_allclose(P1, P2, atol=1e-10)


def test_synthesis_unit_mode_convention():
    n = 6
    xi = np.zeros((1, n, n))
    k1, k2 = 2, 1                      # x frequency 2, y frequency 1
    xi[0, k2, k1] = 1.0
    m = field.synthesize(xi, n, 0.1, 1.0, 0.0)[0]
    lam = 1.0 + 0.1 * 4 * n * n * (np.sin(np.pi * k1 / (2 * n)) ** 2 + np.sin(np.pi * k2 / (2 * n)) ** 2)
    j = np.arange(n)
    vx = np.sqrt(2.0 / n) * np.cos(np.pi * k1 * (j + 0.5) / n)
    vy = np.sqrt(2.0 / n) * np.cos(np.pi * k2 * (j + 0.5) / n)
    np.testing.assert_allclose(m, n / lam * np.outer(vy, vx), atol=1e-14)


def test_field_covariance_statistics():
    n, N = 6, 20000
    m = field.sample_fields(seed=21, first=0, count=N, n=n).reshape(N, -1)
    A = _dense_A(n, 0.1, 1.0)
    Ainv = np.linalg.inv(A)
    C_exact = n * n * Ainv @ Ainv
    C_emp = np.cov(m.T, bias=True)
    # entrywise standard error of a sample covariance: sqrt((C_ii C_jj + C_ij^2)/N)
    d = np.sqrt(np.diag(C_exact))
    se = np.sqrt((np.outer(d, d) ** 2 + C_exact ** 2) / N)
    assert np.max(np.abs(C_emp - C_exact) / se) < 5.0
    # mean pointwise variance equals sum lambda^-2
    lam = field.kl_eigenvalues(n, 0.1, 1.0)
    np.testing.assert_allclose(np.trace(C_exact) / (n * n), np.sum(lam ** -2.0), rtol=1e-12)


def test_control_sources():
    n, L, w = 21, 5, 0.05
    G = field.control_sources(n, L, w)
    assert G.shape == (n * n, L * L)
    # control (jx=2, jy=2) is centred at (0.5, 0.5) = node (10, 10)
    j = 2 * L + 2
    np.testing.assert_allclose(G[10 * n + 10, j], 1.0 / (w * np.sqrt(2 * np.pi)), rtol=1e-15)
    # control (jx=1, jy=3): centre (0.3, 0.7); x varies fastest in the control index
    x, y = 0.25, 0.7
    jj = 3 * L + 1
    ix, iy = 5, 14
    val = np.exp(-((x - 0.3) ** 2 + (y - 0.7) ** 2) / (2 * w * w)) / (w * np.sqrt(2 * np.pi))
    np.testing.assert_allclose(G[iy * n + ix, jj], val, rtol=1e-13)
    ut = field.target_state(n)
    np.testing.assert_allclose(ut[10, 10], 1.0, rtol=1e-15)
    np.testing.assert_allclose(ut[5, 14], np.sin(np.pi * 0.7) * np.sin(np.pi * 0.25), rtol=1e-14)
