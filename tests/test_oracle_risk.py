"""Pins of the oracle's risk measures (Sec. 2.1-2.3), CPU only.

* Smoothed plus function: values and first/second derivatives continuous at 0
  and eps (C^2, as Sec. 2.1 states) and s <= x^+ <= s + eps/2.
* Stratified Gaussian QoIs: mean -> mu, variance -> sigma^2 and
  CVaR_0.95 -> mu + sigma phi(Phi^-1(0.95)) / 0.05 (closed form of the normal).
* Brute-force Rockafellar-Uryasev minimum on tiny N against the smoothed t*.
* t* is the minimiser of the smoothed objective: no point of a dense grid of t does
  better, also with ties, a constant sample and N (1 - beta) < 1 (CVaR = max Q).
* Risk gradients against finite differences through per-sample linear QoIs.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import risk


def test_splus_c2_and_bounds():
    eps = 1e-4
    for x0 in (0.0, eps):
        for f in (risk.splus, risk.splus_d1, risk.splus_d2):
            lo = f(x0 - 1e-13, eps)
            hi = f(x0 + 1e-13, eps)
            scale = {risk.splus: eps, risk.splus_d1: 1.0, risk.splus_d2: 1.0 / eps}[f]
            assert abs(lo - hi) <= 1e-7 * scale
    x = np.linspace(-3 * eps, 3 * eps, 10001)
    s = risk.splus(x, eps)
    xp = np.maximum(x, 0)
    assert np.all(s <= xp + 1e-18) and np.all(xp <= s + eps / 2 + 1e-18)
    # derivatives are the derivatives: finite differences inside each piece
    xs = np.array([-0.5 * eps, 0.3 * eps, 0.7 * eps, 2 * eps])
    d = 1e-9 * eps
    np.testing.assert_allclose((risk.splus(xs + d, eps) - risk.splus(xs - d, eps)) / (2 * d),
                               risk.splus_d1(xs, eps), atol=1e-6)
    np.testing.assert_allclose((risk.splus_d1(xs + d, eps) - risk.splus_d1(xs - d, eps)) / (2 * d),
                               risk.splus_d2(xs, eps), atol=1e-6 / eps)
    assert risk.splus(0.0, eps) == 0.0 and risk.splus(eps, eps) == 0.5 * eps


def test_gaussian_closed_forms():
    N = 10000
    mu, sigma = 2.0, 0.5
    Q = mu + sigma * stats.norm.ppf((np.arange(1, N + 1) - 0.5) / N)
    G = np.zeros((N, 1))
    rho, _ = risk.mean_var(Q, G, kappa=1.0)
    np.testing.assert_allclose(Q.mean(), mu, atol=1e-12)
    np.testing.assert_allclose(rho, mu + sigma ** 2, rtol=1e-3)
    beta = 0.95
    exact = mu + sigma * stats.norm.pdf(stats.norm.ppf(beta)) / (1 - beta)
    np.testing.assert_allclose(exact, mu + 2.0627128 * sigma, rtol=1e-7)
    val, _, dt, t = risk.cvar(Q, G, beta=beta, eps=1e-4)
    np.testing.assert_allclose(val, exact, rtol=1e-3)
    np.testing.assert_allclose(t, mu + sigma * stats.norm.ppf(beta), rtol=1e-3)
    assert abs(dt) < 1e-9


@pytest.mark.parametrize("N", [5, 8, 12])
def test_cvar_bruteforce_tiny(N):
    rng = np.random.default_rng(N)
    Q = rng.standard_normal(N)
    beta = 0.75
    bf = risk.cvar_bruteforce(Q, beta)
    eps = 1e-9
    val, _, _, t = risk.cvar(Q, np.zeros((N, 1)), beta=beta, eps=eps)
    # smoothing lowers the value by at most eps/2 per sample weight
    assert bf - 0.5 * eps / (1 - beta) - 1e-14 <= val <= bf + 1e-14
    # definition of CVaR for equally weighted atoms at a level with N(1-beta) integer
    if float(N * (1 - beta)).is_integer():
        k = int(round(N * (1 - beta)))
        np.testing.assert_allclose(bf, np.sort(Q)[-k:].mean(), rtol=1e-14)


def test_risk_gradients_finite_difference():
    # Q_i(z) = a_i + b_i . z + 1/2 c_i |z|^2: exact per-sample gradients are known
    rng = np.random.default_rng(7)
    N, d = 40, 3
    a, b, c = rng.standard_normal(N), rng.standard_normal((N, d)), rng.uniform(0.5, 1.5, N)
    z0 = rng.standard_normal(d)

    def per_sample(z):
        return a + b @ z + 0.5 * c * (z @ z), b + c[:, None] * z[None, :]

    def f_mv(z):
        return risk.mean_var(per_sample(z)[0], per_sample(z)[1], kappa=1.0)

    def f_cv(z):
        v, g, _, _ = risk.cvar(per_sample(z)[0], per_sample(z)[1], beta=0.9, eps=1e-2)
        return v, g

    for f in (f_mv, f_cv):
        _, g = f(z0)
        step = 1e-6
        fd = np.array([(f(z0 + step * e)[0] - f(z0 - step * e)[0]) / (2 * step) for e in np.eye(d)])
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)
    # d rho / dt at a fixed t, and the t-derivative of the value
    Q = per_sample(z0)[0]
    t = np.median(Q)
    dt = risk.cvar_dt(Q, t, 0.9, 1e-2)
    fd_t = (risk.cvar_value(Q, t + 1e-7, 0.9, 1e-2) - risk.cvar_value(Q, t - 1e-7, 0.9, 1e-2)) / 2e-7
    np.testing.assert_allclose(dt, fd_t, rtol=1e-6)


@pytest.mark.parametrize("case", ["random", "ties", "constant", "single_tail"])
def test_tstar_is_the_minimiser(case):
    rng = np.random.default_rng(11)
    beta, eps = 0.9, 1e-3
    Q = {"random": rng.standard_normal(37),
         "ties": np.repeat(rng.standard_normal(5), 7),
         "constant": np.full(9, 0.3),
         "single_tail": rng.standard_normal(6)}[case]   # N (1 - beta) = 0.6 < 1
    t = risk.cvar_tstar(Q, beta, eps)
    v = risk.cvar_value(Q, t, beta, eps)
    grid = np.linspace(Q.min() - 2 * eps, Q.max() + 2 * eps, 20001)
    vals = grid + risk.splus(Q[None, :] - grid[:, None], eps).sum(axis=1) / (Q.size * (1 - beta))
    assert v <= vals.min() + 1e-12
    bf = risk.cvar_bruteforce(Q, beta)
    assert bf - 0.5 * eps / (1 - beta) - 1e-12 <= v <= bf + 1e-12
    if case == "single_tail":
        assert bf == Q.max()
