"""The 257 x 257 configuration (100 controls, MR-DINO SAA over N = 16384 samples) against the
FP64 oracle: field synthesis, the plain state/adjoint path on a few samples, the MR-DINO
evaluation of a small network, and the KL projection at the full size (N = 16384, 8.7 GB of
FP64 fields) on sampled rows.

Tolerances as in the 129 x 129 tests: fields 1e-12, u and Q 1e-9, per-sample gradients
1e-8; MR-DINO against the BF16-emulated oracle phi 5e-3, Q 2e-3, grad_z Q 1e-2; projection
1e-5 + 5e-7 sqrt(n^2) of the row scale.
"""
import math

import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field, pde
from oracle.dino import round_bf16
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_GRID, L = 257, 10
DZ = L * L


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def test_fields_257():
    from paper_2305_20053_gb300 import capi
    P = capi.Problem(n=N_GRID, lattice_L=L, max_samples=3)
    m = torch.empty(3, N_GRID, N_GRID, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 16381, 3, m)
    assert np.abs(m.cpu().numpy() - field.sample_fields(SEED_SAA, 16381, 3, N_GRID)).max() <= 1e-12


def test_state_adjoint_257():
    from paper_2305_20053_gb300 import capi
    N = 2
    P = capi.Problem(n=N_GRID, lattice_L=L, max_samples=N)
    ms = field.sample_fields(SEED_SAA, 0, N, N_GRID)   # the oracle's draws on both sides
    m = torch.tensor(ms, device="cuda")
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    u = torch.empty_like(m)
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, N, torch.tensor(z, device="cuda"), 0, u, q, st)
    lam = torch.empty_like(m)
    g = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
    P.ouu_adjoint_batch(m, u, N, lam, g)
    prob = pde.Problem(n=N_GRID, L=L)
    G = field.control_sources(N_GRID, L, prob.width)
    refs = pde.solve_batch(ms, z, G, field.target_state(N_GRID), prob, with_adjoint=True)
    u, q, g, st = (t.cpu().numpy() for t in (u, q, g, st))
    assert np.all(st == 0)
    for i, r in enumerate(refs):
        assert rel(u[i], r.u) <= 1e-9
        assert abs(q[i] - r.q) <= 1e-9 * abs(r.q)
        assert rel(g[i], r.grad) <= 1e-8


def test_dino_eval_257():
    """A small network (r = 24, width 48) on an M-orthonormal random basis: the evaluation
    path at 257 x 257 (projection over n^2 = 66049, reduced QoI, reverse-mode gradient)."""
    from paper_2305_20053_gb300 import capi
    RM = RU = 24
    W, N = 48, 64
    n, h = N_GRID, 1.0 / (N_GRID - 1)
    widths = [RM + DZ, W, W, W, RU]
    Ws, bs = glorot_uniform_mlp(widths, seed=31)
    bs = [0.1 * random_state_like(80 + l, b.shape) for l, b in enumerate(bs)]
    flat = capi.flatten_params(Ws, bs)
    Ws64, bs64 = capi.unflatten_params(flat, widths)
    scale = np.linspace(0.05, 0.01, RU).astype(np.float32)
    net = dino.MLP(Ws64, bs64, RM, out_scale=scale.astype(np.float64))
    d = (n - 2) ** 2
    Qm, _ = np.linalg.qr(random_state_like(90, (d, RU)))
    Phi = Qm / h                                   # h^2 Phi^T Phi = I
    ubar = 0.05 * random_state_like(91, (d,))
    phi_full = np.zeros((RU, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(RU, n - 2, n - 2)
    ub_full = np.zeros((n, n))
    ub_full[1:-1, 1:-1] = ubar.reshape(n - 2, n - 2)
    D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=N)
    D.ouu_dino_set_params(flat)
    D.ouu_dino_set_output_scale(scale)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.tensor(ub_full, device="cuda"))
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    mf = field.sample_fields(SEED_SAA, 0, N, n).reshape(N, -1)   # the oracle's draws on both sides
    m = torch.tensor(mf.reshape(N, n, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, DZ)[0]
    phi = torch.empty(N, RU, dtype=torch.float32, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    gq = torch.empty(N, DZ, dtype=torch.float64, device="cuda")
    D.ouu_dino_eval(m, N, z, phi, None, q, gq)
    Wkl, _ = dino.kl_projection_matrix(n, RM)
    xi = dino.project_fields(mf, Wkl, bf16=True)
    ut = field.target_state(n)[1:-1, 1:-1].ravel()
    Qbf, gbf, pbf, _ = dino.eval_surrogate(net, xi, z, Phi, ubar, ut, h, decode=False, bf16=True)
    phi, q, gq = (t.cpu().numpy() for t in (phi, q, gq))
    assert rel(phi, pbf) <= 5e-3
    assert np.max(np.abs(q - Qbf) / np.abs(Qbf)) <= 2e-3
    assert rel(gq, gbf) <= 1e-2


def test_projection_full_size_257():
    """N = 16384 fields of 257 x 257 (8.7 GB): the fused projection checked on 64 sampled rows."""
    from paper_2305_20053_gb300 import capi
    N, nn, rm = 16384, N_GRID * N_GRID, 200
    ldw = (nn + 63) // 64 * 64
    g = torch.Generator(device="cuda").manual_seed(5)
    m = torch.randn(N, nn, device="cuda", dtype=torch.float64, generator=g)
    W = (torch.randn(rm, ldw, device="cuda", generator=g) / math.sqrt(nn)).to(torch.bfloat16)
    W[:, nn:] = 0
    b = torch.zeros(rm, device="cuda")
    xi = torch.empty(N, rm, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_kl_project(m, N, nn, W, rm, b, xi, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    rows = np.random.default_rng(6).choice(N, 64, replace=False)
    rows_t = torch.tensor(rows, device="cuda")
    ms = m[rows_t].cpu().numpy()
    Wh = W[:, :nn].float().cpu().numpy().astype(np.float64)
    ref = round_bf16(ms) @ Wh.T
    got = xi[rows_t].cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= (1e-5 + 5e-7 * math.sqrt(nn)) * scale)
