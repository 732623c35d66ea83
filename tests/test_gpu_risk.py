"""GPU risk weights (Sec. 2.1-2.2) against the FP64 oracle on QoI sets chosen to reach every
branch of the t* search: a Gaussian sample, ties, windows of many samples within eps
of the quantile (more than one per lane; more than the shared window holds), samples
sharing the top 32 key bits (the 64-bit radix fallback), more samples than the
register-held keys cover, tiny N, and a fixed t.

Tolerances: t* within 1e-12 relative (the GPU stops its bracket a few ulps wide, the
oracle bisects to adjacent doubles); rho and d rho/dt within 1e-12 and 1e-9 absolute;
the weights applied to three seeded gradient columns, and the kernel's own weighted
gradient sums, within 1e-9 relative.
"""
import zlib

import numpy as np
import pytest

from oracle import risk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _qoi(case, rng):
    if case == "gauss4096":
        return 5.0 + 0.7 * rng.standard_normal(4096)
    if case == "uniform1000":
        return rng.uniform(2.0, 9.0, 1000)
    if case == "ties5000":
        return np.round(rng.uniform(4.0, 6.0, 5000), 2)
    if case == "window1500":
        return 5.0 + 1e-6 * rng.uniform(size=1500)
    if case == "window3000":
        return 5.0 + 1e-6 * rng.uniform(size=3000)
    if case == "prefix200":
        return np.concatenate([5.0 + 1e-9 * np.arange(200.0), rng.uniform(1.0, 4.0, 300)])
    if case == "large20000":
        return np.exp(rng.standard_normal(20000))
    if case == "n1":
        return np.array([3.25])
    if case == "n7":
        return rng.uniform(0.0, 1.0, 7)
    raise ValueError(case)


@pytest.mark.parametrize("case", ["gauss4096", "uniform1000", "ties5000", "window1500", "window3000", "prefix200",
                                  "large20000", "n1", "n7"])
def test_risk_weights_parity(case):
    from paper_2305_20053_gb300 import capi
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    Q = _qoi(case, rng)
    N = Q.size
    G = rng.standard_normal((N, 3))
    beta, eps, kappa = 0.95, 1e-4, 1.0
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=beta, eps=eps, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=kappa),
             capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-3, t=float(np.median(Q)), t_optimal=0)]
    q = torch.tensor(Q, device="cuda")
    w = torch.empty(len(risks), N, device="cuda", dtype=torch.float64)
    G32 = G.astype(np.float32)
    out, grad = capi.ouu_kernel_risk_weights(q, risks, w, gq=torch.tensor(G32, device="cuda"))
    W = w.cpu().numpy()
    G = G32.astype(np.float64)   # the gradients the kernel sums

    rho, g, dt, t = risk.cvar(Q, G, beta=beta, eps=eps, t_optimal=True)
    assert abs(out[0, 2] - t) <= 1e-12 * max(1.0, abs(t))
    assert abs(out[0, 0] - rho) <= 1e-12 * max(1.0, abs(rho))
    assert abs(out[0, 1] - dt) <= 1e-9
    np.testing.assert_allclose(W[0] @ G, g, rtol=1e-9, atol=1e-12 * np.abs(G).sum())
    np.testing.assert_allclose(grad[0], g, rtol=1e-9, atol=1e-12 * np.abs(G).sum())

    rho_mv, g_mv = risk.mean_var(Q, G, kappa=kappa)
    assert abs(out[1, 0] - rho_mv) <= 1e-12 * max(1.0, abs(rho_mv))
    np.testing.assert_allclose(W[1] @ G, g_mv, rtol=1e-9, atol=1e-12 * np.abs(G).sum())
    np.testing.assert_allclose(grad[1], g_mv, rtol=1e-9, atol=1e-12 * np.abs(G).sum())

    tf = float(np.median(Q))
    rho_f, g_f, dt_f, _ = risk.cvar(Q, G, beta=0.9, eps=1e-3, t=tf, t_optimal=False)
    assert out[2, 2] == tf
    assert abs(out[2, 0] - rho_f) <= 1e-12 * max(1.0, abs(rho_f))
    assert abs(out[2, 1] - dt_f) <= 1e-9
    np.testing.assert_allclose(W[2] @ G, g_f, rtol=1e-9, atol=1e-12 * np.abs(G).sum())
    np.testing.assert_allclose(grad[2], g_f, rtol=1e-9, atol=1e-12 * np.abs(G).sum())


def test_risk_weights_repeat_calls_agree():
    """No state is carried between calls: a second call gives the same values."""
    from paper_2305_20053_gb300 import capi
    Q = 5.0 + np.random.default_rng(3).standard_normal(4096)
    q = torch.tensor(Q, device="cuda")
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1)]
    w1 = torch.empty(1, Q.size, device="cuda", dtype=torch.float64)
    w2 = torch.empty_like(w1)
    o1 = capi.ouu_kernel_risk_weights(q, risks, w1)
    o2 = capi.ouu_kernel_risk_weights(q, risks, w2)
    assert np.array_equal(o1, o2)
    assert torch.equal(w1, w2)
