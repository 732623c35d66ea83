"""Multifidelity Monte Carlo with the MR-DINO surrogate as the control variate (the extension the
paper's conclusions name, after Ng & Willcox): the mean of the QoI and its z-gradient from a
few high-fidelity samples (plain PDE path) and many low-fidelity ones (the network), unbiased
for the high-fidelity mean whatever the surrogate's error.

With the first n_hi of the n_lo low-fidelity samples shared with the high-fidelity ones,

    E_MF = mean(Q_hi[:n_hi]) + alpha (mean(Q_lo[:n_lo]) - mean(Q_lo[:n_hi])),

alpha = cov(Q_hi, Q_lo) / var(Q_lo) over the shared samples (the variance-minimising weight of
a control variate).  Each gradient component takes the same form with its own weight.  The
estimator's variance relative to the plain n_hi-sample mean is about
1 - (1 - n_hi / n_lo) rho^2, rho the correlation of the two fidelities.
Host arithmetic over per-sample outputs; the samples themselves come from the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class MfmcEstimate:
    mean: float            # multifidelity estimate of E[Q]
    grad: np.ndarray       # multifidelity estimate of grad_z E[Q]
    alpha: float           # control-variate weight of the QoI
    rho: float             # correlation of Q_hi and Q_lo over the shared samples
    variance_ratio: float  # predicted variance of `mean` over that of the n_hi-sample mean
    hi_mean: float         # the plain n_hi-sample mean, for comparison


def _cv_weight(hi, lo):
    """alpha = cov(hi, lo) / var(lo) per column (0 where var(lo) = 0)."""
    hc, lc = hi - hi.mean(axis=0), lo - lo.mean(axis=0)
    var = np.sum(lc * lc, axis=0)
    cov = np.sum(hc * lc, axis=0)
    return np.where(var > 0, cov / np.where(var > 0, var, 1.0), 0.0)


def combine(q_hi, q_lo, g_hi=None, g_lo=None):
    """The estimator from per-sample values: q_hi [n_hi] (and g_hi [n_hi][d_Z]) of the high
    fidelity, q_lo [n_lo] (g_lo [n_lo][d_Z]) of the low fidelity, whose first n_hi samples are
    the high-fidelity ones."""
    q_hi, q_lo = np.asarray(q_hi, np.float64), np.asarray(q_lo, np.float64)
    n_hi, n_lo = q_hi.size, q_lo.size
    if n_lo < n_hi or n_hi < 2:
        raise ValueError("need 2 <= n_hi <= n_lo")
    shared = q_lo[:n_hi]
    alpha = float(_cv_weight(q_hi[:, None], shared[:, None])[0])
    mean = float(q_hi.mean() + alpha * (q_lo.mean() - shared.mean()))
    sh, sl = q_hi.std(), shared.std()
    rho = float(np.corrcoef(q_hi, shared)[0, 1]) if sh > 0 and sl > 0 else 0.0
    ratio = 1.0 - (1.0 - n_hi / n_lo) * rho * rho
    grad = None
    if g_hi is not None:
        g_hi, g_lo = np.asarray(g_hi, np.float64), np.asarray(g_lo, np.float64)
        a = _cv_weight(g_hi, g_lo[:n_hi])
        grad = g_hi.mean(axis=0) + a * (g_lo.mean(axis=0) - g_lo[:n_hi].mean(axis=0))
    return MfmcEstimate(mean=mean, grad=grad, alpha=alpha, rho=rho, variance_ratio=ratio, hi_mean=float(q_hi.mean()))


def estimate(problem, dino, m_dev, n_hi, n_lo, z_host):
    """E[Q] and grad_z E[Q] at z over the fields m_dev [n_lo][n][n]: the plain path (state and
    adjoint solves) on the first n_hi fields, the network on all n_lo."""
    import torch
    n, dz = problem.n, problem.d_z
    dev = m_dev.device
    zt = torch.tensor(np.asarray(z_host, np.float64), device=dev)
    u = torch.empty(n_hi, n, n, dtype=torch.float64, device=dev)
    q = torch.empty(n_hi, dtype=torch.float64, device=dev)
    st = torch.empty(n_hi, dtype=torch.int32, device=dev)
    g = torch.empty(n_hi, dz, dtype=torch.float64, device=dev)
    problem.ouu_pde_solve_batch(m_dev, n_hi, zt, 0, u, q, st)
    problem.ouu_adjoint_batch(m_dev, u, n_hi, None, g)
    ql = torch.empty(n_lo, dtype=torch.float64, device=dev)
    gl = torch.empty(n_lo, dz, dtype=torch.float64, device=dev)
    dino.ouu_dino_eval(m_dev, n_lo, z_host, None, None, ql, gl)
    return combine(q.cpu().numpy(), ql.cpu().numpy(), g.cpu().numpy(), gl.cpu().numpy())
