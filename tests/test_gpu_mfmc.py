"""Multifidelity Monte Carlo through the library (paper_2305_20053_gb300/mfmc.py estimate): the
plain path on the first 24 of 200 fields, the network on all 200 (17 x 17 grid, 9 controls,
a small seeded network on an M-orthonormal basis), against the same estimator applied to the
oracle's per-sample values (FP64 PDE solves and adjoints; the oracle surrogate with the BF16
roundings of the CUDA path) on the same fields.  Tolerances: the estimate of E[Q] 1e-3
relative, its z-gradient 1e-2 (the network's values agree with the oracle's to 2e-3 / 1e-2)."""
import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field, pde
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def test_mfmc_estimate_against_oracle_values():
    from paper_2305_20053_gb300 import capi, mfmc
    n, L, n_hi, n_lo, RM, RU, W = 17, 3, 24, 200, 16, 12, 32
    dz, h = L * L, 1.0 / (n - 1)
    widths = [RM + dz, W, W, W, RU]
    Ws, bs = glorot_uniform_mlp(widths, seed=611)
    bs = [0.1 * random_state_like(612 + l, b.shape) for l, b in enumerate(bs)]
    flat = capi.flatten_params(Ws, bs)
    Ws64, bs64 = capi.unflatten_params(flat, widths)
    net = dino.MLP(Ws64, bs64, RM)
    Phi = np.linalg.qr(random_state_like(617, ((n - 2) ** 2, RU)))[0] / h
    phi_full = np.zeros((RU, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(RU, n - 2, n - 2)
    D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=n_lo)
    D.ouu_dino_set_params(flat)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.zeros(n, n, dtype=torch.float64, device="cuda"))
    P = capi.Problem(n=n, lattice_L=L, max_samples=n_lo)
    ms = field.sample_fields(SEED_SAA, 0, n_lo, n)
    z = controls(SEED_EVAL_Z, 1, dz)[0]
    got = mfmc.estimate(P, D, torch.tensor(ms, device="cuda"), n_hi, n_lo, z)
    prob = pde.Problem(n=n, L=L)
    refs = pde.solve_batch(ms[:n_hi], z, field.control_sources(n, L, prob.width), field.target_state(n), prob)
    q_hi, g_hi = np.array([r.q for r in refs]), np.stack([r.grad for r in refs])
    Wkl, _ = dino.kl_projection_matrix(n, RM)
    ut = field.target_state(n)[1:-1, 1:-1].ravel()
    q_lo, g_lo, _, _ = dino.eval_surrogate(net, dino.project_fields(ms.reshape(n_lo, -1), Wkl, bf16=True), z, Phi,
                                           np.zeros((n - 2) ** 2), ut, h, decode=False, bf16=True)
    want = mfmc.combine(q_hi, q_lo, g_hi, g_lo)
    assert got.mean == pytest.approx(want.mean, rel=1e-3)
    assert rel(got.grad, want.grad) <= 1e-2
    assert got.hi_mean == pytest.approx(want.hi_mean, rel=1e-9)
    P.close()
    D.close()
