"""Host logic of the outer OUU solve (paper_2305_20053_gb300/ouu.py), CPU only, with the oracle
standing in for the library's SAA evaluations.

* A separable quadratic QoI Q_i(z) = 1/2 sum_j a_ij (z_j - c_ij)^2 (mean, kappa = 0): the
  box-constrained minimiser is clip(sum_i a_ij c_ij / sum_i a_ij, lo, hi), written out.
* The smoothed CVaR of the PDE's tracking QoI (oracle, 9 x 9 grid, 4 controls, 8 fields),
  minimised jointly in (z, t) (Sec. 2.1 Rockafellar-Uryasev form): the KKT conditions hold
  at the result (projected gradient ~ 0, d rho / dt ~ 0), and it reaches the cost of the
  minimisation over z alone with t = t*(z) at every evaluation.
* The relative optimal cost error of Sec. 4.1.
"""
import numpy as np
import pytest

from oracle import field, pde, risk
from paper_2305_20053_gb300 import ouu
from synthetic_inputs import SEED_SAA


def test_box_constrained_quadratic():
    rng = np.random.default_rng(3)
    N, d = 6, 5
    a = rng.uniform(0.5, 2.0, (N, d))
    c = rng.uniform(-2.0, 2.0, (N, d))
    c[:, 1] += 3.0          # this coordinate's unconstrained minimiser lies above the box
    c[:, 3] -= 3.0          # and this one below

    def evaluate(z, t):
        Q = 0.5 * np.sum(a * (z - c) ** 2, axis=1)
        G = a * (z - c)
        v, g = risk.mean_var(Q, G, kappa=0.0)
        return v, g, 0.0

    res = ouu.minimize_risk(evaluate, d, joint_t=False, lo=-1.0, hi=1.0)
    want = np.clip(np.sum(a * c, axis=0) / np.sum(a, axis=0), -1.0, 1.0)
    np.testing.assert_allclose(res.z, want, atol=1e-7)
    assert res.z[1] == 1.0 and res.z[3] == -1.0 and res.converged


def _pde_evaluator(beta=0.9, eps=1e-2):
    n, L, N = 9, 2, 8
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)
    ms = field.sample_fields(SEED_SAA, 0, N, n)

    def qg(z):
        refs = pde.solve_batch(ms, z, G, ut, prob)
        return np.array([r.q for r in refs]), np.stack([r.grad for r in refs])

    def evaluate(z, t):
        Q, Gq = qg(z)
        v, g, dt, _ = risk.cvar(Q, Gq, beta, eps, t=t, t_optimal=False)
        return v, g, dt

    def evaluate_tstar(z, t):
        Q, Gq = qg(z)
        v, g, _, _ = risk.cvar(Q, Gq, beta, eps)
        return v, g, 0.0

    return evaluate, evaluate_tstar, L * L


def test_cvar_joint_in_z_and_t_meets_kkt():
    evaluate, evaluate_tstar, d = _pde_evaluator()
    z0 = np.full(d, 0.3)
    joint = ouu.minimize_risk(evaluate, d, joint_t=True, z0=z0, t0=0.1, lo=-1.0, hi=1.0)
    _, g, dt = evaluate(joint.z, joint.t)
    free = (joint.z > -1.0 + 1e-9) & (joint.z < 1.0 - 1e-9)
    assert np.all(np.abs(g[free]) <= 1e-6 * max(1.0, np.abs(g).max()))
    assert np.all(g[joint.z >= 1.0 - 1e-9] <= 1e-9) and np.all(g[joint.z <= -1.0 + 1e-9] >= -1e-9)
    assert abs(dt) <= 1e-6
    outer = ouu.minimize_risk(evaluate_tstar, d, joint_t=False, z0=z0, lo=-1.0, hi=1.0)
    assert joint.cost == pytest.approx(outer.cost, rel=1e-7)
    assert joint.cost < evaluate(z0, 0.1)[0]


def test_relative_cost_error():
    assert ouu.relative_cost_error(1.1, 1.0) == pytest.approx(0.1)
    assert ouu.relative_cost_error(-0.9, -1.0) == pytest.approx(0.1)
