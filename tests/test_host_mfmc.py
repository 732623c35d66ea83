"""Multifidelity Monte Carlo estimator (paper_2305_20053_gb300/mfmc.py), CPU only.

* A low fidelity that is an affine function of the high one, Q_lo = a Q_hi + b (and the same
  for each gradient component), makes the control variate exact: the estimate equals the mean
  of the high fidelity over all n_lo samples.
* An independent low fidelity gets weight ~0: the estimate is the high-fidelity mean.
* Over many repetitions with jointly Gaussian fidelities of correlation rho, the estimator is
  unbiased and its variance relative to the plain n_hi-sample mean is 1 - (1 - n_hi/n_lo) rho^2
  (the control-variate result for optimal weights), within sampling error.
"""
import numpy as np
import pytest

from paper_2305_20053_gb300 import mfmc


def test_affine_low_fidelity_is_exact():
    rng = np.random.default_rng(0)
    n_hi, n_lo, d = 20, 500, 3
    q = rng.standard_normal(n_lo) * 2 + 5
    g = rng.standard_normal((n_lo, d))
    est = mfmc.combine(q[:n_hi], 0.7 * q - 3.0, g[:n_hi], -2.0 * g + 1.5)
    assert est.mean == pytest.approx(q.mean(), rel=1e-13)
    np.testing.assert_allclose(est.grad, g.mean(axis=0), rtol=1e-12, atol=1e-14)
    assert est.alpha == pytest.approx(1 / 0.7, rel=1e-12) and est.rho == pytest.approx(1.0, rel=1e-12)
    assert est.variance_ratio == pytest.approx(n_hi / n_lo, rel=1e-12)


def test_independent_low_fidelity_gets_no_weight():
    rng = np.random.default_rng(1)
    n_hi, n_lo = 4000, 8000
    q = rng.standard_normal(n_lo)
    lo = rng.standard_normal(n_lo)
    est = mfmc.combine(q[:n_hi], lo)
    assert abs(est.alpha) < 0.05 and abs(est.mean - q[:n_hi].mean()) < 0.01 and est.variance_ratio > 0.99


def test_unbiased_with_the_predicted_variance_reduction():
    rng = np.random.default_rng(2)
    n_hi, n_lo, rho, reps = 16, 256, 0.9, 4000
    means, plain = [], []
    for _ in range(reps):
        x = rng.standard_normal(n_lo)
        hi = 3.0 + x
        lo = 0.5 * (rho * x + np.sqrt(1 - rho * rho) * rng.standard_normal(n_lo)) + 1.0
        e = mfmc.combine(hi[:n_hi], lo)
        means.append(e.mean)
        plain.append(e.hi_mean)
    means, plain = np.array(means), np.array(plain)
    assert abs(means.mean() - 3.0) < 4 * means.std() / np.sqrt(reps)
    predicted = 1 - (1 - n_hi / n_lo) * rho * rho
    # estimated weights add a small-sample excess of order 1 / n_hi
    assert means.var() / plain.var() == pytest.approx(predicted, rel=0.15)
