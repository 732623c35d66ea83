"""GPU parity of the MR-DINO kernels against the FP64 oracle on the same weights,
bases and fields (small network so that the oracle runs in seconds).

Tolerances (relative l2 unless stated):
  KL coordinates: 2e-2 vs FP64, 2e-4 vs the oracle with BF16 operands emulated
  phi: 2e-2 vs FP64, 5e-3 vs BF16-emulated; d_z phi: 3e-2 / 1e-2
  reduced Q: 2e-2 vs FP64, 2e-3 vs BF16-emulated (per sample); grad_z Q: 3e-2 / 1e-2
  loss gradient (one batch): 2e-2, cosine >= 0.999; states projection 1e-5;
  Jacobian data 1e-4; POD eigenvalues 1e-9, modes 1e-7, M-orthonormality 1e-12.
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field, pde
from synthetic_inputs import SEED_EVAL_Z, SEED_HELDOUT, SEED_SAA, SEED_TRAIN_FIELDS, SEED_TRAIN_Z, controls, \
    glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_GRID, L, RM, RU, W = 17, 3, 16, 12, 32
DZ = L * L


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _net(seed=11):
    from paper_2305_20053_gb300 import capi
    widths = [RM + DZ, W, W, W, RU]
    Ws, bs = glorot_uniform_mlp(widths, seed=seed)
    bs = [0.1 * random_state_like(seed + 50 + l, b.shape) for l, b in enumerate(bs)]
    flat = capi.flatten_params(Ws, bs)
    Ws64, bs64 = capi.unflatten_params(flat, widths)      # the FP32-rounded weights both sides use
    scale = np.linspace(1.0, 0.1, RU).astype(np.float32)  # a fixed output scale, as build_bases sets one
    return flat, dino.MLP(Ws64, bs64, RM, out_scale=scale.astype(np.float64)), widths, scale


@pytest.fixture(scope="module")
def setup():
    """Oracle states of 24 training pairs, oracle POD, and a network + problem on the GPU."""
    from paper_2305_20053_gb300 import capi
    n = N_GRID
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)
    ms = field.sample_fields(SEED_TRAIN_FIELDS, 0, 24, n)
    zs = controls(SEED_TRAIN_Z, 24, DZ)
    states = [pde.solve_sample(ms[i], zs[i], G, ut, prob, with_adjoint=False).u for i in range(24)]
    U = np.stack([s[1:-1, 1:-1].ravel() for s in states])
    Phi, ubar, ev = dino.pod(U, RU, prob.h)
    phi_full = np.zeros((RU, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(RU, n - 2, n - 2)
    ubar_full = np.zeros((n, n))
    ubar_full[1:-1, 1:-1] = ubar.reshape(n - 2, n - 2)
    flat, net, widths, scale = _net()
    D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=64)
    D.ouu_dino_set_params(flat)
    D.ouu_dino_set_output_scale(scale)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.tensor(ubar_full, device="cuda"))
    P = capi.Problem(n=n, lattice_L=L, max_samples=64)
    return dict(prob=prob, G=G, ut=ut, ms=ms, zs=zs, states=states, U=U, Phi=Phi, ubar=ubar, ev=ev, net=net,
                flat=flat, widths=widths, D=D, P=P)


def test_kl_projection(setup):
    D, n, N = setup["D"], N_GRID, 40
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)   # the oracle's draws on both sides
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    xi = torch.empty(N, RM, dtype=torch.float32, device="cuda")
    D.ouu_dino_project_fields(m, N, xi)
    Wkl, order = dino.kl_projection_matrix(n, RM)
    x64 = dino.project_fields(mf, Wkl)
    xbf = dino.project_fields(mf, Wkl, bf16=True)
    xi = xi.cpu().numpy()
    assert rel(xi, x64) <= 2e-2
    assert rel(xi, xbf) <= 2e-4
    # a KL draw projects onto its own normals
    from oracle import philox
    np.testing.assert_allclose(x64, philox.field_normals(SEED_SAA, 0, N, n * n)[:, order[:RM]], atol=1e-10)


def test_eval_parity(setup):
    D, n, N = setup["D"], N_GRID, 40
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)   # the oracle's draws on both sides
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    phi = torch.empty(N, RU, dtype=torch.float32, device="cuda")
    jphi = torch.empty(N, DZ, RU, dtype=torch.float32, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    gq = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
    D.ouu_dino_eval(m, N, z, phi, jphi, q, gq)
    Wkl, _ = dino.kl_projection_matrix(n, RM)
    ut_int = setup["ut"][1:-1, 1:-1].ravel()
    h = 1.0 / (n - 1)
    Q64, g64, p64, J64 = dino.eval_surrogate(setup["net"], dino.project_fields(mf, Wkl), z, setup["Phi"],
                                             setup["ubar"], ut_int, h, decode=True)
    Qbf, gbf, pbf, Jbf = dino.eval_surrogate(setup["net"], dino.project_fields(mf, Wkl, bf16=True), z, setup["Phi"],
                                             setup["ubar"], ut_int, h, decode=False, bf16=True)
    phi, jphi, q, gq = (t.cpu().numpy() for t in (phi, jphi, q, gq))
    assert rel(phi, p64) <= 2e-2 and rel(phi, pbf) <= 5e-3
    J = np.transpose(jphi, (0, 2, 1))
    assert rel(J, J64) <= 3e-2 and rel(J, Jbf) <= 1e-2
    assert np.max(np.abs(q - Q64) / np.abs(Q64)) <= 2e-2
    assert np.max(np.abs(q - Qbf) / np.abs(Qbf)) <= 2e-3
    assert rel(gq, g64) <= 3e-2 and rel(gq, gbf) <= 1e-2


def test_loss_gradient_parity(setup):
    D = setup["D"]
    B, n_data = 16, 20
    xi = random_state_like(101, (n_data, RM)).astype(np.float32)
    z = controls(102, n_data, DZ).astype(np.float32)
    y = (0.1 * random_state_like(103, (n_data, RU))).astype(np.float32)
    jy = (0.05 * random_state_like(104, (n_data, DZ, RU))).astype(np.float32)
    idx = np.array([3, 17, 0, 5, 9, 11, 2, 19, 4, 8, 13, 1, 6, 15, 7, 10], dtype=np.int32)
    T = lambda a: torch.tensor(a, device="cuda")
    loss, g = D.ouu_dino_loss_grad(T(xi), T(z), T(y), T(jy), T(idx), B)
    net = setup["net"]
    Y = np.transpose(jy[idx], (0, 2, 1)).astype(np.float64)
    l64, dW, db = net.loss_and_grad(xi[idx].astype(np.float64), z[idx].astype(np.float64),
                                    y[idx].astype(np.float64), Y, w_j=1.0)
    from paper_2305_20053_gb300 import capi
    g64 = np.concatenate([np.concatenate([a.ravel(), b]) for a, b in zip(dW, db)])
    assert abs(loss - l64) <= 1e-2 * l64
    assert rel(g, g64) <= 2e-2
    assert g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)) >= 0.999
    # per block too (each weight matrix and bias)
    o = 0
    for W_, b_ in zip(dW, db):
        for part in (W_.ravel(), b_):
            k = part.size
            assert rel(g[o:o + k], part) <= 5e-2, o
            o += k


def test_adam_step_moves_by_lr(setup):
    """First Adam step from zero moments: every weight moves by lr * g / (|g| + eps), i.e. by
    about lr against the sign of its gradient (checked where the oracle gradient is large)."""
    from paper_2305_20053_gb300 import capi
    n = N_GRID
    flat, net, widths, scale = _net(seed=21)
    D2 = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=16)
    D2.ouu_dino_set_params(flat)
    D2.ouu_dino_set_output_scale(scale)
    B = 16
    xi = random_state_like(201, (B, RM)).astype(np.float32)
    z = controls(202, B, DZ).astype(np.float32)
    y = (0.1 * random_state_like(203, (B, RU))).astype(np.float32)
    jy = (0.05 * random_state_like(204, (B, DZ, RU))).astype(np.float32)
    idx = np.arange(B, dtype=np.int32)
    T = lambda a: torch.tensor(a, device="cuda")
    lr = 1e-3
    D2.ouu_dino_train_step(T(xi), T(z), T(y), T(jy), T(idx), B, lr)
    after = D2.ouu_dino_get_params()
    _, dW, db = net.loss_and_grad(xi.astype(np.float64), z.astype(np.float64), y.astype(np.float64),
                                  np.transpose(jy, (0, 2, 1)).astype(np.float64))
    g64 = np.concatenate([np.concatenate([a.ravel(), b]) for a, b in zip(dW, db)])
    step = after.astype(np.float64) - flat.astype(np.float64)
    big = np.abs(g64) > 0.05 * np.abs(g64).max()
    assert big.sum() > 50
    np.testing.assert_allclose(np.abs(step[big]), lr, rtol=1e-3)
    assert np.all(np.sign(step[big]) == -np.sign(g64[big]))
    D2.close()


def test_project_states_and_jacobian_data(setup):
    D, P, n = setup["D"], setup["P"], N_GRID
    N = 6
    ms = setup["ms"][:N]
    us = np.stack(setup["states"][:N])
    m_t = torch.tensor(ms, device="cuda")
    u_t = torch.tensor(us, device="cuda")
    y = torch.empty(N, RU, dtype=torch.float32, device="cuda")
    D.ouu_dino_project_states(u_t, N, y)
    h = 1.0 / (n - 1)
    y64 = h * h * (setup["U"][:N] - setup["ubar"]) @ setup["Phi"]
    assert rel(y.cpu().numpy(), y64) <= 1e-5
    jy = torch.empty(N, DZ, RU, dtype=torch.float32, device="cuda")
    D.ouu_dino_jacobian_data(P, m_t, u_t, N, jy)
    G_int = pde.interior_rows(setup["G"], n)
    ref = []
    for i in range(N):
        kx, ky = pde.face_coefficients(ms[i])
        f = (setup["G"] @ setup["zs"][i]).reshape(n, n)
        u, chol = pde.newton_solve(kx, ky, f, 1.0, h)
        dudz = pde.state_jacobian_columns(chol, G_int, n)
        ref.append((h * h * setup["Phi"].T @ dudz).T)       # [dz][ru]
    assert rel(jy.cpu().numpy(), np.stack(ref)) <= 1e-4


def test_pod_build_parity(setup):
    from paper_2305_20053_gb300 import capi
    n = N_GRID
    D3 = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=16)
    u = torch.tensor(np.stack(setup["states"]), device="cuda")
    ev = D3.ouu_dino_build_bases(u, 24)
    phi = torch.empty(RU, n, n, dtype=torch.float64, device="cuda")
    ubar = torch.empty(n, n, dtype=torch.float64, device="cuda")
    D3.ouu_dino_get_bases(phi, ubar)
    phi = phi.cpu().numpy()
    h = 1.0 / (n - 1)
    np.testing.assert_allclose(ubar.cpu().numpy()[1:-1, 1:-1].ravel(), setup["ubar"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(ev[:RU], setup["ev"][:RU], rtol=1e-9)
    P = phi[:, 1:-1, 1:-1].reshape(RU, -1).T
    np.testing.assert_allclose(h * h * P.T @ P, np.eye(RU), atol=1e-12)
    np.testing.assert_allclose(D3.ouu_dino_get_output_scale(), np.sqrt(setup["ev"][:RU] / 24), rtol=1e-6)
    gaps = np.abs(np.diff(setup["ev"][:RU + 1])) / setup["ev"][0]
    for k in range(RU):
        if min(gaps[k], gaps[k - 1] if k else 1.0) > 1e-6:
            assert rel(P[:, k], setup["Phi"][:, k]) <= 1e-7, k
    assert np.all(phi[:, 0, :] == 0) and np.all(phi[:, :, -1] == 0)
    D3.close()


def test_dino_risk_path(setup):
    from paper_2305_20053_gb300 import capi
    from oracle import risk
    D, P, n, N = setup["D"], setup["P"], N_GRID, 40
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)   # the oracle's draws on both sides
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    risks = [capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0),
             capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1)]
    val, grad, gt, t, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
    Wkl, _ = dino.kl_projection_matrix(n, RM)
    xbf = dino.project_fields(mf, Wkl, bf16=True)
    ut_int = setup["ut"][1:-1, 1:-1].ravel()
    Q, gQ, _, _ = dino.eval_surrogate(setup["net"], xbf, z, setup["Phi"], setup["ubar"], ut_int, 1.0 / (n - 1),
                                      decode=False, bf16=True)
    v0, g0 = risk.mean_var(Q, gQ, 1.0)
    v1, g1, _, _ = risk.cvar(Q, gQ, 0.9, 1e-4)
    assert abs(val[0] - v0) <= 1e-3 * abs(v0) and rel(grad[0], g0) <= 1e-2
    assert abs(val[1] - v1) <= 1e-3 * abs(v1) and rel(grad[1], g1) <= 2e-2


def test_graph_replay_matches_eager(setup):
    """The captured graph of the DINO risk evaluation gives the eager results, also after z changes.
    The per-block partial sums of the weighted gradient are added atomically in FP64, whose
    order varies from run to run: gradients agree to 1e-12 relative, risk values exactly
    (their partial sums are combined in a fixed order)."""
    from paper_2305_20053_gb300 import capi
    D, P, n, N = setup["D"], setup["P"], N_GRID, 40
    m = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 0, N, m)
    risks = [capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0),
             capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1)]
    zs = controls(SEED_EVAL_Z + 7, 3, DZ)
    D.ouu_dino_set_graphs(0)
    eager = [P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)[:2] for z in zs]
    D.ouu_dino_set_graphs(1)
    graphed = [P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)[:2] for z in zs]   # capture, replay, replay
    for (v0, g0), (v1, g1) in zip(eager, graphed):
        np.testing.assert_array_equal(v0, v1)
        np.testing.assert_allclose(g1, g0, rtol=1e-12, atol=1e-15 * np.abs(g0).max())


@pytest.mark.parametrize("mode", [1, 2])
def test_fused_network_matches_layer_kernels(setup, mode):
    """The one-kernel evaluation networks (mode 1: one CTA per tile; mode 2: 4-CTA clusters, here
    with two of the four column quarters past the width) give the per-layer GEMM path's results
    (the same BF16 roundings and K order; only FP32 sums of the QoI and the FP64 risk reductions
    may differ)."""
    from paper_2305_20053_gb300 import capi
    D, P, n, N = setup["D"], setup["P"], N_GRID, 40
    m = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 0, N, m)
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    out = {}
    for fused in (mode, 0):
        D.ouu_dino_set_fused_network(fused)
        q = torch.empty(N, dtype=torch.float64, device="cuda")
        gq = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
        phi = torch.empty(N, RU, dtype=torch.float32, device="cuda")
        D.ouu_dino_eval(m, N, z, phi, None, q, gq)
        risks = [capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0),
                 capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1)]
        v, g, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
        out[fused] = (q.cpu().numpy(), gq.cpu().numpy(), phi.cpu().numpy(), v, g)
    D.ouu_dino_set_fused_network(0)
    (q1, g1, p1, v1, r1), (q0, g0, p0, v0, r0) = out[mode], out[0]
    np.testing.assert_allclose(p1, p0, rtol=1e-5, atol=1e-6 * np.abs(p0).max())
    np.testing.assert_allclose(q1, q0, rtol=1e-5)
    assert rel(g1, g0) <= 1e-5
    np.testing.assert_allclose(v1, v0, rtol=1e-5)
    assert rel(r1, r0) <= 1e-5


def test_cluster_network_bench_shape():
    """The one-kernel networks (modes 1 and 2) at the widths of the 129 x 129 workload's network
    (r_M 200, width 400, r_U 200, d_Z 100), random weights and an M-orthonormal random basis,
    over three 128-sample tiles (the last ragged), against the per-layer path on IDENTICAL
    projection coordinates (the network alone, so that the projection's atomically added
    partial sums cannot differ between the runs): phi and grad_z Q to 1e-6 (the same
    arithmetic), Q to 1e-6 (its FP32 row sums run in another order)."""
    from paper_2305_20053_gb300 import capi
    n, L, RMb, RUb, Wb, N = 33, 10, 200, 200, 400, 300
    dz, h = L * L, 1.0 / (n - 1)
    Ws, bs = glorot_uniform_mlp([RMb + dz, Wb, Wb, Wb, RUb], seed=91)
    bs = [0.1 * random_state_like(92 + l, b.shape) for l, b in enumerate(bs)]
    D = capi.Dino(n=n, lattice_L=L, r_m=RMb, r_u=RUb, width=Wb, max_batch=16, max_eval=N)
    D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
    D.ouu_dino_set_output_scale(np.linspace(0.05, 0.01, RUb).astype(np.float32))
    Q, _ = np.linalg.qr(random_state_like(97, ((n - 2) ** 2, RUb)))
    phi = np.zeros((RUb, n, n))
    phi[:, 1:-1, 1:-1] = (Q / h).T.reshape(RUb, n - 2, n - 2)
    ub = np.zeros((n, n))
    ub[1:-1, 1:-1] = 0.05 * random_state_like(98, (n - 2, n - 2))
    D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.tensor(ub, device="cuda"))
    xi = torch.tensor(random_state_like(99, (N, RMb)).astype(np.float32), device="cuda")
    z = controls(SEED_EVAL_Z, 1, dz)[0]
    out = {}
    for mode in (0, 1, 2):
        q = torch.empty(N, dtype=torch.float64, device="cuda")
        gq = torch.empty(N, dz, dtype=torch.float64, device="cuda")
        ph = torch.empty(N, RUb, dtype=torch.float32, device="cuda")
        D.ouu_kernel_dino_network(xi, N, z, mode, q, ph, gq)
        out[mode] = (q.cpu().numpy(), gq.cpu().numpy(), ph.cpu().numpy())
    q0, g0, p0 = out[0]
    assert np.all(np.isfinite(q0)) and np.all(np.isfinite(g0)) and np.abs(g0).max() > 0
    for mode in (1, 2):
        qm, gm, pm = out[mode]
        np.testing.assert_allclose(pm, p0, rtol=1e-6, atol=1e-7 * np.abs(p0).max())
        np.testing.assert_allclose(qm, q0, rtol=1e-6)
        assert rel(gm, g0) <= 1e-6, (mode, rel(gm, g0))


def test_auto_backend_falls_back_to_the_plain_path(setup):
    """BACKEND_AUTO runs the plain path until the network passes its held-out check against it
    for this problem (ouu_dino_validate), the network after that, and the plain path again for
    another problem or once the network changes.  The untrained network here fails a 1 % / 5 %
    check; an unbounded check passes it.  Risk values: 1e-9 relative against the plain path on
    the same inputs, 1e-6 against the network's own evaluation."""
    from paper_2305_20053_gb300 import capi
    D, P, n, N = setup["D"], setup["P"], N_GRID, 40
    m = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_HELDOUT, 0, N, m)
    risks = [capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0),
             capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1)]
    zs = controls(SEED_EVAL_Z + 11, 2, DZ)
    z = zs[0]
    pde_v = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z)[0]
    dino_v = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)[0]

    def auto(prob):
        v = prob.ouu_risk_and_grad(capi.BACKEND_AUTO, D, m, N, risks, z)[0]
        return v, prob.ouu_last_backend()

    v, b = auto(P)                          # never checked: the plain path
    assert b == capi.BACKEND_PDE
    np.testing.assert_allclose(v, pde_v, rtol=1e-9)
    er, eg, ok = D.ouu_dino_validate(P, m, N, risks, zs, risk_tol=0.01, grad_tol=0.05)
    assert not ok and np.isfinite(er) and np.isfinite(eg) and (er > 0.01 or eg > 0.05)
    assert auto(P)[1] == capi.BACKEND_PDE
    er2, eg2, ok = D.ouu_dino_validate(P, m, N, risks, zs, risk_tol=1e30, grad_tol=1e30)
    assert ok and er2 == pytest.approx(er, rel=1e-3) and eg2 == pytest.approx(eg, rel=1e-3)
    v, b = auto(P)
    assert b == capi.BACKEND_DINO
    np.testing.assert_allclose(v, dino_v, rtol=1e-6)
    P2 = capi.Problem(n=n, lattice_L=L, max_samples=N)   # the check named P, not P2
    assert auto(P2)[1] == capi.BACKEND_PDE
    D.ouu_dino_set_params(D.ouu_dino_get_params())       # a changed network is checked again
    assert auto(P)[1] == capi.BACKEND_PDE
    P2.close()
