"""GPU parity of the plain (PDE) path against the FP64 oracle, through the C ABI.

Tolerances (relative, per result): fields m 1e-12 (absolute, values O(1));
states u 1e-9 (l2); QoIs 1e-9; adjoints 1e-9 (l2); per-sample gradients 1e-8;
risk values and risk gradients 1e-8.
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import field, pde, risk
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, SEED_TRAIN_Z, controls

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def problem(n, L, N, **kw):
    from paper_2305_20053_gb300 import capi
    return capi.Problem(n=n, lattice_L=L, max_samples=N, **kw)


def fields(P, seed, first, N):
    """The oracle's fields (host) and the same values on the device: both sides of a parity
    test start from the oracle's draws."""
    ms = field.sample_fields(seed, first, N, P.n)
    return ms, torch.tensor(ms, device="cuda")


@pytest.mark.parametrize("n,N,first", [(33, 8, 0), (129, 3, 4093), (5, 2, 0), (17, 5, 2 ** 32 + 7)])
def test_sample_fields_parity(n, N, first):
    P = problem(n, 2, N)
    m = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, first, N, m)
    ref = field.sample_fields(SEED_SAA, first, N, n)
    assert np.abs(m.cpu().numpy() - ref).max() <= 1e-12


def _oracle(ms, z, n, L, z_per_sample=False):
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)
    return pde.solve_batch(ms, z, G, ut, prob, with_adjoint=True, z_per_sample=z_per_sample)


@pytest.mark.parametrize("n,L,N,per_sample", [(33, 5, 64, False), (17, 3, 37, True), (5, 1, 1, False)])
def test_state_adjoint_parity(n, L, N, per_sample):
    P = problem(n, L, N)
    ms, m = fields(P, SEED_SAA, 0, N)
    if per_sample:
        z = controls(SEED_TRAIN_Z, N, L * L)
        zt = torch.tensor(z, device="cuda")
        stride = L * L
    else:
        z = controls(SEED_EVAL_Z, 1, L * L)[0]
        zt = torch.tensor(z, device="cuda")
        stride = 0
    u = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, N, zt, stride, u, q, st)
    lam = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    g = torch.empty(N, L * L, dtype=torch.float64, device="cuda")
    P.ouu_adjoint_batch(m, u, N, lam, g)
    refs = _oracle(ms, z, n, L, z_per_sample=per_sample)
    u, q, lam, g, st = (t.cpu().numpy() for t in (u, q, lam, g, st))
    assert np.all(st == 0)
    for i, r in enumerate(refs):
        assert rel(u[i], r.u) <= 1e-9, i
        assert abs(q[i] - r.q) <= 1e-9 * abs(r.q), i
        assert rel(lam[i][1:-1, 1:-1], r.lam) <= 1e-9, i
        assert np.all(lam[i][0] == 0) and np.all(lam[i][:, -1] == 0)
        assert rel(g[i], r.grad) <= 1e-8, i


RISKS_CFG1 = None


def _risks():
    from paper_2305_20053_gb300 import capi
    return [capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0),
            capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1),
            capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-2, t=0.1, t_optimal=0)]


def test_risk_and_grad_parity_33x33_64_samples():
    from paper_2305_20053_gb300 import capi
    n, L, N = 33, 5, 64
    P = problem(n, L, N)
    ms, m = fields(P, SEED_SAA, 0, N)
    zs = list(controls(SEED_EVAL_Z, 5, L * L)) + [np.zeros(L * L)]
    for z in zs:
        val, grad, gt, t, stats = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, _risks(), z)
        refs = _oracle(ms, z, n, L)
        Q = np.array([r.q for r in refs])
        Gq = np.stack([r.grad for r in refs])
        v0, g0 = risk.mean_var(Q, Gq, kappa=1.0)
        v1, g1, dt1, t1 = risk.cvar(Q, Gq, beta=0.95, eps=1e-4, t_optimal=True)
        v2, g2, dt2, _ = risk.cvar(Q, Gq, beta=0.9, eps=1e-2, t=0.1, t_optimal=False)
        assert abs(val[0] - v0) <= 1e-8 * abs(v0)
        assert rel(grad[0], g0) <= 1e-8
        assert abs(val[1] - v1) <= 1e-8 * abs(v1)
        assert abs(t[1] - t1) <= 1e-8 * abs(t1)
        assert rel(grad[1], g1) <= 1e-8
        assert abs(gt[1] - dt1) <= 1e-8
        assert abs(val[2] - v2) <= 1e-8 * abs(v2)
        assert rel(grad[2], g2) <= 1e-8 or np.linalg.norm(g2) == 0.0
        assert abs(gt[2] - dt2) <= 1e-8
        assert stats.n_not_converged == 0 and stats.newton_min >= 1 or not np.any(z)


def test_cvar_skips_zero_weight_adjoints():
    from paper_2305_20053_gb300 import capi
    n, L, N = 17, 3, 200
    P = problem(n, L, N)
    ms, m = fields(P, SEED_SAA, 0, N)
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1)]
    val, grad, gt, t, stats = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z)
    assert 0 < stats.adjoint_solves < N // 5
    refs = _oracle(ms, z, n, L)
    Q = np.array([r.q for r in refs])
    Gq = np.stack([r.grad for r in refs])
    v1, g1, _, _ = risk.cvar(Q, Gq, beta=0.95, eps=1e-4, t_optimal=True)
    assert abs(val[0] - v1) <= 1e-8 * abs(v1)
    assert rel(grad[0], g1) <= 1e-8


def test_full_size_risk_and_gradient_against_oracle():
    """The benchmark's launch configuration (129 x 129, N = 4096, d_Z = 100): the risk values,
    t* and z-gradients of the smoothed CVaR_0.95 and mean + variance against the oracle run on
    every one of the 4096 fields (spawned processes on the host cores), at 1e-8 relative."""
    from oracle_pool import qoi_and_gradients
    from paper_2305_20053_gb300 import capi
    n, L, N = 129, 10, 4096
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    Q, Gq = qoi_and_gradients(SEED_SAA, N, n, L, z)   # the pool starts before this process's GPU work
    P = problem(n, L, N)
    ms, m = fields(P, SEED_SAA, 0, N)
    del ms
    val, grad, gt, t, stats = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, _risks()[:2], z)
    v0, g0 = risk.mean_var(Q, Gq, kappa=1.0)
    v1, g1, dt1, t1 = risk.cvar(Q, Gq, beta=0.95, eps=1e-4, t_optimal=True)
    assert abs(val[0] - v0) <= 1e-8 * abs(v0) and rel(grad[0], g0) <= 1e-8
    assert abs(val[1] - v1) <= 1e-8 * abs(v1) and rel(grad[1], g1) <= 1e-8
    assert abs(t[1] - t1) <= 1e-8 * abs(t1) and abs(gt[1] - dt1) <= 1e-8
    P.close()


def test_full_size_129x129_4096_samples():
    """The benchmark's launch configuration: sampled per-sample QoIs against the oracle,
    the risk values against the oracle's risk formulas on the GPU QoIs, and the risk
    gradients against central differences of the GPU risk (properties at any size)."""
    from paper_2305_20053_gb300 import capi
    n, L, N = 129, 10, 4096
    P = problem(n, L, N)
    ms, m = fields(P, SEED_SAA, 0, N)
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    zt = torch.tensor(z, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, N, zt, 0, None, q, st)
    q = q.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    idx = [0, 1, 777, 2048, 4000, 4095]
    refs = _oracle(ms[idx], z, n, L)
    for k, r in zip(idx, refs):
        assert abs(q[k] - r.q) <= 1e-9 * abs(r.q), k
    risks = _risks()[:2]
    val, grad, gt, t, stats = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z)
    assert stats.n_not_converged == 0
    v0, _ = risk.mean_var(q, np.zeros((N, 1)), kappa=1.0)
    v1, _, _, t1 = risk.cvar(q, np.zeros((N, 1)), beta=0.95, eps=1e-4)
    assert abs(val[0] - v0) <= 1e-10 * abs(v0)
    assert abs(val[1] - v1) <= 1e-10 * abs(v1)
    d = np.random.default_rng(0).standard_normal(L * L)
    d /= np.linalg.norm(d)
    step = 1e-5
    vp = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z + step * d)[0]
    vm = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z - step * d)[0]
    fd = (vp - vm) / (2 * step)
    for r in range(2):
        assert abs(grad[r] @ d - fd[r]) <= 1e-5 * np.linalg.norm(grad[r]), (r, grad[r] @ d, fd[r])


def test_nonfinite_and_not_converged_are_reported():
    from paper_2305_20053_gb300 import capi
    n, L, N = 17, 3, 4
    P = problem(n, L, N)
    _, m = fields(P, SEED_SAA, 0, N)
    m[2, 5, 5] = float("nan")
    z = torch.tensor(controls(SEED_EVAL_Z, 1, L * L)[0], device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.OuuError) as e:
        P.ouu_pde_solve_batch(m, N, z, 0, None, q, st)
    assert e.value.status == 5
    assert st.cpu().numpy().tolist() == [0, 0, 2, 0]
    P2 = problem(n, L, N, newton_maxit=1)
    _, m2 = fields(P2, SEED_SAA, 0, N)
    with pytest.raises(capi.OuuError) as e:
        P2.ouu_pde_solve_batch(m2, N, z, 0, None, q, st)
    assert e.value.status == 4
    assert np.all(st.cpu().numpy() == 1)


def test_zero_control_gives_zero_state():
    n, L, N = 9, 2, 3
    P = problem(n, L, N)
    _, m = fields(P, SEED_SAA, 0, N)
    z = torch.zeros(L * L, dtype=torch.float64, device="cuda")
    u = torch.full((N, n, n), 7.0, dtype=torch.float64, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, N, z, 0, u, q, st)
    assert torch.all(u == 0).item()
    np.testing.assert_allclose(q.cpu().numpy(), 0.125, rtol=1e-14)
