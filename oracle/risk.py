"""Risk measures over a sample average and their gradients (oracle, test infrastructure only).

Sec. 2.1-2.3.  Given per-sample QoIs Q_i and gradients g_i = grad_z Q_i:

Mean + variance (a moment-based measure, Sec. 2.1 "moments of Q"):
    rho = Qbar + kappa Var,  Var = (1/N) sum (Q_i - Qbar)^2          (plug-in 1/N)
    grad rho = (1/N) sum [1 + 2 kappa (Q_i - Qbar)] g_i

Smoothed CVaR (Sec. 2.1 Rockafellar-Uryasev form with the C^2 plus function,
and its SAA of Sec. 2.2):
    rho(z, t) = t + 1/(N (1-beta)) sum s_eps(Q_i - t)
    s_eps(x) = 0 (x <= 0),  x^3/eps^2 - x^4/(2 eps^3) (0 < x < eps),  x - eps/2 (x >= eps)
    d rho/dz = 1/(N (1-beta)) sum s'_eps(Q_i - t) g_i
    d rho/dt = 1 - 1/(N (1-beta)) sum s'_eps(Q_i - t)
With t_optimal the variable t is set to the minimiser t* of rho(z, .), found by
bisection on the monotone d rho/dt (rho is convex in t).
"""
from __future__ import annotations

import numpy as np


def splus(x, eps):
    x = np.asarray(x, dtype=np.float64)
    mid = x ** 3 / eps ** 2 - x ** 4 / (2.0 * eps ** 3)
    return np.where(x <= 0.0, 0.0, np.where(x < eps, mid, x - 0.5 * eps))


def splus_d1(x, eps):
    x = np.asarray(x, dtype=np.float64)
    mid = 3.0 * x ** 2 / eps ** 2 - 2.0 * x ** 3 / eps ** 3
    return np.where(x <= 0.0, 0.0, np.where(x < eps, mid, 1.0))


def splus_d2(x, eps):
    x = np.asarray(x, dtype=np.float64)
    mid = 6.0 * x / eps ** 2 - 6.0 * x ** 2 / eps ** 3
    return np.where(x <= 0.0, 0.0, np.where(x < eps, mid, 0.0))


def mean_var(Q, G, kappa=1.0):
    """(rho, grad) for mean + kappa * variance; Q (N,), G (N, d_z)."""
    Q = np.asarray(Q, dtype=np.float64)
    N = Q.size
    qbar = Q.mean()
    var = np.mean((Q - qbar) ** 2)
    w = (1.0 + 2.0 * kappa * (Q - qbar)) / N
    return qbar + kappa * var, w @ G


def cvar_value(Q, t, beta, eps):
    Q = np.asarray(Q, dtype=np.float64)
    return t + np.sum(splus(Q - t, eps)) / (Q.size * (1.0 - beta))


def cvar_dt(Q, t, beta, eps):
    Q = np.asarray(Q, dtype=np.float64)
    return 1.0 - np.sum(splus_d1(Q - t, eps)) / (Q.size * (1.0 - beta))


def cvar_tstar(Q, beta, eps, iters=200):
    """Minimiser of t -> rho(z, t): bisection of the non-decreasing d rho/dt on
    [min Q - eps, max Q] (d rho/dt = 1 - 1/(1-beta) < 0 at the left end, 1 at the right)."""
    Q = np.asarray(Q, dtype=np.float64)
    lo, hi = Q.min() - eps, Q.max()
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if cvar_dt(Q, mid, beta, eps) < 0.0:
            lo = mid
        else:
            hi = mid
    return lo if cvar_dt(Q, lo, beta, eps) >= 0.0 else hi


def cvar(Q, G, beta=0.95, eps=1e-4, t=0.0, t_optimal=True):
    """(rho, grad_z, grad_t, t_used) of the smoothed CVaR SAA."""
    Q = np.asarray(Q, dtype=np.float64)
    if t_optimal:
        t = cvar_tstar(Q, beta, eps)
    N = Q.size
    w = splus_d1(Q - t, eps) / (N * (1.0 - beta))
    return cvar_value(Q, t, beta, eps), w @ G, cvar_dt(Q, t, beta, eps), t


def cvar_bruteforce(Q, beta):
    """Non-smoothed CVaR by the Rockafellar-Uryasev minimisation: the piecewise-linear
    convex function of t attains its minimum at one of the sample values."""
    Q = np.asarray(Q, dtype=np.float64)
    N = Q.size
    vals = [t + np.sum(np.maximum(Q - t, 0.0)) / (N * (1.0 - beta)) for t in Q]
    return float(min(vals))
