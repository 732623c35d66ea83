"""The outer optimisation under uncertainty (Sec. 2.2, Sec. 4.1-4.2): minimise the SAA cost
J(z) = rho(z) + P(z) over box-bounded controls z, for the smoothed CVaR jointly in (z, t)
(the Rockafellar-Uryasev form of Sec. 2.1), by L-BFGS-B, every cost and gradient being one
ouu_risk_and_grad call (plain path or MR-DINO).  Host logic only: the optimiser is SciPy's
L-BFGS-B, the evaluations are the library's.

  relative_cost_error: the accuracy measure of Sec. 4.1,
      |J(z*_approx) - J(z*_ref)| / |J(z*_ref)|,
  with both costs evaluated by the same reference evaluator.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class OuuResult:
    z: np.ndarray          # optimal controls
    t: float               # optimal CVaR variable (0 for mean + variance)
    cost: float            # J at the optimum
    evaluations: int       # cost + gradient evaluations
    iterations: int
    converged: bool
    message: str
    history: list = field(default_factory=list)   # cost per evaluation


def minimize_risk(evaluate, d_z, joint_t, z0=None, t0=0.0, lo=-1.0, hi=1.0, penalty=0.0, maxiter=200,
                  gtol=1e-8, ftol=1e-12):
    """min over z in [lo, hi]^d_z (and t in R when joint_t) of rho(z[, t]) + penalty/2 ||z||^2.

    evaluate(z, t) -> (rho, grad_z rho, d rho / dt): one SAA evaluation (t ignored when not
    joint_t).  Returns an OuuResult."""
    from scipy.optimize import minimize
    z0 = np.zeros(d_z) if z0 is None else np.asarray(z0, dtype=np.float64)
    x0 = np.concatenate([z0, [t0]]) if joint_t else z0.copy()
    hist = []

    def fun(x):
        z = x[:d_z]
        t = float(x[d_z]) if joint_t else 0.0
        rho, gz, gt = evaluate(z, t)
        cost = float(rho) + 0.5 * penalty * float(z @ z)
        g = np.asarray(gz, dtype=np.float64) + penalty * z
        hist.append(cost)
        return cost, (np.concatenate([g, [float(gt)]]) if joint_t else g)

    bounds = [(lo, hi)] * d_z + ([(None, None)] if joint_t else [])
    r = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=bounds,
                 options={"maxiter": maxiter, "gtol": gtol, "ftol": ftol, "maxcor": 20})
    return OuuResult(z=r.x[:d_z].copy(), t=float(r.x[d_z]) if joint_t else 0.0, cost=float(r.fun),
                     evaluations=int(r.nfev), iterations=int(r.nit), converged=bool(r.success),
                     message=str(r.message), history=hist)


def library_evaluator(problem, backend, dino, m_dev, n_samples, risk):
    """evaluate(z, t) over the fields m_dev with the library: the risk descriptor `risk`
    (capi.RiskDesc) with its t replaced by the optimiser's t and t_optimal off for CVaR."""
    from paper_2305_20053_gb300 import capi
    joint = risk.kind == capi.RISK_CVAR_SMOOTH

    def evaluate(z, t):
        r = capi.risk_desc(risk.kind, kappa=risk.kappa, beta=risk.beta, eps=risk.eps, t=t if joint else 0.0,
                           t_optimal=0)
        v, g, gt, _, _ = problem.ouu_risk_and_grad(backend, dino, m_dev, n_samples, [r], z)
        return v[0], g[0], gt[0]

    return evaluate, joint


def solve(problem, backend, dino, m_dev, n_samples, risk, z0=None, lo=-1.0, hi=1.0, penalty=0.0, maxiter=200):
    """The OUU problem over the n_samples fields in m_dev by L-BFGS-B on the library's SAA
    evaluations; for CVaR, t starts at the minimiser t* for z0."""
    from paper_2305_20053_gb300 import capi
    evaluate, joint = library_evaluator(problem, backend, dino, m_dev, n_samples, risk)
    d_z = problem.d_z
    t0 = 0.0
    if joint:
        z_start = np.zeros(d_z) if z0 is None else np.asarray(z0, dtype=np.float64)
        r = capi.risk_desc(risk.kind, beta=risk.beta, eps=risk.eps, t_optimal=1)
        t0 = float(problem.ouu_risk_and_grad(backend, dino, m_dev, n_samples, [r], z_start)[3][0])
    return minimize_risk(evaluate, d_z, joint, z0=z0, t0=t0, lo=lo, hi=hi, penalty=penalty, maxiter=maxiter)


def reference_cost(problem, m_dev, n_samples, risk, z, penalty=0.0):
    """J(z) by the plain path over the reference fields (CVaR at its minimising t)."""
    from paper_2305_20053_gb300 import capi
    r = capi.risk_desc(risk.kind, kappa=risk.kappa, beta=risk.beta, eps=risk.eps, t_optimal=1)
    v = problem.ouu_risk_and_grad(capi.BACKEND_PDE, None, m_dev, n_samples, [r], z)[0][0]
    return float(v) + 0.5 * penalty * float(np.dot(z, z))


def relative_cost_error(cost_approx, cost_ref):
    """Sec. 4.1: |J(z*_approx) - J(z*_ref)| / |J(z*_ref)|."""
    return abs(cost_approx - cost_ref) / abs(cost_ref)
