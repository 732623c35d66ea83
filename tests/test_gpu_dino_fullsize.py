"""MR-DINO evaluation at the widths of the 129 x 129 workload's network, against the oracle.

Network (Sec. 3.3): r_M = 200 KL coordinates and d_Z = 100 controls -> 400 -> 400 -> 400 -> r_U = 200,
GELU, seeded Glorot weights with small seeded biases, a positive per-mode output scale, an
M-orthonormal random POD basis and a random mean state.  The fields are drawn by the oracle
(oracle/field.py) and copied to the device, so both sides see the same inputs.  Oracle:
oracle/dino.py in FP64, and with bf16=True the same operands rounded to bfloat16 where the
CUDA path rounds them (projection inputs, every GEMM operand, the tangents).

* n = 33, N = 300 (three 128-sample tiles, the last ragged), every network mode (0: per-layer
  GEMM kernels, 1: one CTA per tile, 2: 4-CTA clusters): ouu_dino_eval (phi, forward-mode
  d_z phi in max_batch = 128 chunks, reduced Q, reverse-mode grad_z Q) and ouu_risk_and_grad
  (smoothed CVaR_0.95 at t*, mean + variance).
* n = 129, N = 4096, the default mode with the captured graph (the benchmark's launch
  configuration): ouu_risk_and_grad on two calls in a row (capture, replay) and the
  per-sample Q and grad_z Q of ouu_dino_eval.

Tolerances (relative l2 over all entries unless stated; as in the small-network tests):
  phi 2e-2 vs FP64, 5e-3 vs BF16-emulated;  d_z phi 3e-2 / 1e-2;
  Q per sample 2e-2 / 2e-3;  grad_z Q 3e-2 / 1e-2;
  risk values 1e-3 vs BF16-emulated; risk gradients 1e-2 (mean + variance), 2e-2 (CVaR,
  whose weights s'(Q_i - t*) switch within eps = 1e-4 of t*).
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field, risk
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RM, RU, W, L = 200, 200, 400, 10
DZ = L * L
BETA, EPS = 0.95, 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _network(n, max_eval, max_batch=128):
    """The seeded network and basis on both sides: (GPU handle, oracle MLP, Phi, ubar, u_t, h)."""
    from paper_2305_20053_gb300 import capi
    h = 1.0 / (n - 1)
    widths = [RM + DZ, W, W, W, RU]
    Ws, bs = glorot_uniform_mlp(widths, seed=191)
    bs = [0.1 * random_state_like(192 + l, b.shape) for l, b in enumerate(bs)]
    flat = capi.flatten_params(Ws, bs)
    Ws64, bs64 = capi.unflatten_params(flat, widths)     # the FP32-rounded weights both sides use
    scale = np.linspace(0.05, 0.01, RU).astype(np.float32)
    net = dino.MLP(Ws64, bs64, RM, out_scale=scale.astype(np.float64))
    d = (n - 2) ** 2
    Qm, _ = np.linalg.qr(random_state_like(197, (d, RU)))
    Phi = Qm / h                                         # h^2 Phi^T Phi = I
    ubar = 0.05 * random_state_like(198, (d,))
    phi_full = np.zeros((RU, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(RU, n - 2, n - 2)
    ub_full = np.zeros((n, n))
    ub_full[1:-1, 1:-1] = ubar.reshape(n - 2, n - 2)
    D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=max_batch, max_eval=max_eval)
    D.ouu_dino_set_params(flat)
    D.ouu_dino_set_output_scale(scale)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.tensor(ub_full, device="cuda"))
    ut = field.target_state(n)[1:-1, 1:-1].ravel()
    return D, net, Phi, ubar, ut, h


def _oracle(net, mf, z, Phi, ubar, ut, h, n, bf16, chunk=512):
    """Per-sample (Q, grad_z Q, phi, d_z phi) of the oracle surrogate, in chunks of samples."""
    Wkl, _ = dino.kl_projection_matrix(n, RM)
    xi = dino.project_fields(mf, Wkl, bf16=bf16)
    parts = [dino.eval_surrogate(net, xi[s:s + chunk], z, Phi, ubar, ut, h, decode=not bf16, bf16=bf16)
             for s in range(0, xi.shape[0], chunk)]
    return [np.concatenate([p[k] for p in parts]) for k in range(4)]


def _risks_oracle(Q, G):
    v0, g0 = risk.mean_var(Q, G, 1.0)
    v1, g1, _, t1 = risk.cvar(Q, G, BETA, EPS)
    return np.array([v1, v0]), np.stack([g1, g0]), t1


@pytest.fixture(scope="module")
def small():
    n, N = 33, 300
    D, net, Phi, ubar, ut, h = _network(n, N)
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    ref64 = _oracle(net, mf, z, Phi, ubar, ut, h, n, bf16=False)
    refbf = _oracle(net, mf, z, Phi, ubar, ut, h, n, bf16=True)
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    yield dict(D=D, n=n, N=N, m=m, z=z, ref64=ref64, refbf=refbf)
    D.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_eval_bench_widths_against_oracle(small, mode):
    D, N, m, z = small["D"], small["N"], small["m"], small["z"]
    D.ouu_dino_set_fused_network(mode)
    phi = torch.empty(N, RU, dtype=torch.float32, device="cuda")
    jphi = torch.empty(N, DZ, RU, dtype=torch.float32, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    gq = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
    D.ouu_dino_eval(m, N, z, phi, jphi, q, gq)
    phi, jphi, q, gq = (t.cpu().numpy() for t in (phi, jphi, q, gq))
    Q64, g64, p64, J64 = small["ref64"]
    Qbf, gbf, pbf, Jbf = small["refbf"]
    assert rel(phi, p64) <= 2e-2 and rel(phi, pbf) <= 5e-3, (rel(phi, p64), rel(phi, pbf))
    J = np.transpose(jphi, (0, 2, 1))
    assert rel(J, J64) <= 3e-2 and rel(J, Jbf) <= 1e-2, (rel(J, J64), rel(J, Jbf))
    assert np.max(np.abs(q - Q64) / np.abs(Q64)) <= 2e-2
    assert np.max(np.abs(q - Qbf) / np.abs(Qbf)) <= 2e-3
    assert rel(gq, g64) <= 3e-2 and rel(gq, gbf) <= 1e-2, (rel(gq, g64), rel(gq, gbf))
    # the last, ragged tile on its own
    assert rel(gq[256:], gbf[256:]) <= 1e-2 and np.max(np.abs(q[256:] - Qbf[256:]) / np.abs(Qbf[256:])) <= 2e-3


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_risk_bench_widths_against_oracle(small, mode):
    from paper_2305_20053_gb300 import capi
    D, N, m, z, n = small["D"], small["N"], small["m"], small["z"], small["n"]
    D.ouu_dino_set_fused_network(mode)
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=BETA, eps=EPS, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
    val, grad, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
    Qbf, gbf, _, _ = small["refbf"]
    rv, rg, _ = _risks_oracle(Qbf, gbf)
    np.testing.assert_allclose(val, rv, rtol=1e-3)
    assert rel(grad[0], rg[0]) <= 2e-2 and rel(grad[1], rg[1]) <= 1e-2, (rel(grad[0], rg[0]), rel(grad[1], rg[1]))
    P.close()


def test_risk_129x129_4096_samples_against_oracle():
    """The benchmark's launch configuration: 129 x 129 fields, N = 4096, default network mode,
    the evaluation captured into a graph on the first call and replayed on the second."""
    from paper_2305_20053_gb300 import capi
    n, N = 129, 4096
    D, net, Phi, ubar, ut, h = _network(n, N, max_batch=256)
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    Qbf, gbf, _, _ = _oracle(net, mf, z, Phi, ubar, ut, h, n, bf16=True)
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    del mf
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=BETA, eps=EPS, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
    rv, rg, _ = _risks_oracle(Qbf, gbf)
    for _ in range(2):
        val, grad, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
        np.testing.assert_allclose(val, rv, rtol=1e-3)
        assert rel(grad[0], rg[0]) <= 2e-2 and rel(grad[1], rg[1]) <= 1e-2, (rel(grad[0], rg[0]), rel(grad[1], rg[1]))
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    gq = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
    D.ouu_dino_eval(m, N, z, None, None, q, gq)
    q, gq = q.cpu().numpy(), gq.cpu().numpy()
    assert np.max(np.abs(q - Qbf) / np.abs(Qbf)) <= 2e-3
    assert rel(gq, gbf) <= 1e-2
    P.close()
    D.close()
