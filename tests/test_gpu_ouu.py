"""The outer OUU solve (Sec. 2.2, Sec. 4.2: L-BFGS-B over box-bounded controls, for CVaR jointly
in (z, t)) driven by the library's plain path reaches the optimum that the same optimiser
driven by the FP64 oracle reaches: 17 x 17 grid, 9 controls in [-1, 1], 32 fields (the
oracle's draws on both sides), smoothed CVaR_0.9 (eps = 1e-3) and mean + variance.
Tolerances: optimal cost 1e-6 relative, optimal controls 1e-4 (max norm), and the relative
optimal cost error of Sec. 4.1 between the two below 1e-6."""
import numpy as np
import pytest

from oracle import field, pde, risk
from synthetic_inputs import SEED_SAA

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


@pytest.mark.parametrize("kind", ["cvar", "meanvar"])
def test_library_and_oracle_reach_the_same_optimum(kind):
    from paper_2305_20053_gb300 import capi, ouu
    n, L, N = 17, 3, 32
    ms = field.sample_fields(SEED_SAA, 0, N, n)
    m = torch.tensor(ms, device="cuda")
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    if kind == "cvar":
        rd = capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-3)
    else:
        rd = capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)
    z0 = np.full(L * L, 0.2)
    gpu = ouu.solve(P, capi.BACKEND_PDE, None, m, N, rd, z0=z0)

    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)

    def evaluate(z, t):
        refs = pde.solve_batch(ms, z, G, ut, prob)
        Q, Gq = np.array([r.q for r in refs]), np.stack([r.grad for r in refs])
        if kind == "cvar":
            v, g, dt, _ = risk.cvar(Q, Gq, 0.9, 1e-3, t=t, t_optimal=False)
            return v, g, dt
        v, g = risk.mean_var(Q, Gq, 1.0)
        return v, g, 0.0

    t0 = 0.0
    if kind == "cvar":
        refs = pde.solve_batch(ms, z0, G, ut, prob)
        t0 = risk.cvar_tstar(np.array([r.q for r in refs]), 0.9, 1e-3)
    orc = ouu.minimize_risk(evaluate, L * L, joint_t=(kind == "cvar"), z0=z0, t0=t0)
    assert gpu.cost == pytest.approx(orc.cost, rel=1e-6)
    assert np.max(np.abs(gpu.z - orc.z)) <= 1e-4
    assert ouu.relative_cost_error(ouu.reference_cost(P, m, N, rd, gpu.z), orc.cost) <= 1e-6
    assert gpu.cost < evaluate(z0, t0)[0]
    P.close()
