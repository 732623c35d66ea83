"""POD decode of Sec. 3.3 on the tensor cores: u_w = Phi phi + ubar and the decoded QoI
Q(u_w) = 1/2 h^2 sum over the interior of (u_w - u_t)^2, against the oracle
(oracle/dino.py decode_states, decoded_qoi) on the same coefficients, basis and mean state.

* ouu_dino_decode at 33 x 33 (1089 columns: a ragged last column tile) with N = 300
  (three 128-row tiles, the last ragged), r_u = 12 and 200;
* at 129 x 129, N = 4096, r_u = 200 (the benchmark's sizes);
* ouu_dino_eval with u_dev: its decoded states equal ouu_dino_decode of its phi_dev, and the
  decoded QoI equals the reduced QoI 1/2 ||phi + c||^2 + const that ouu_dino_eval returns.

Tolerances, from the arithmetic: phi and Phi are each split into two BF16 parts and three of
the four cross products are kept, so every product carries a relative error below 3 x 2^-18
(about 1.1e-5) and the FP32 sums over r_u terms add about 1e-7 sqrt(r_u).  States: 5e-5
relative l2 per sample; boundary nodes exactly 0.  Decoded QoI: 2e-4 relative (its FP32 sums
of squares run over n^2 nodes in tiles of 256); decoded vs reduced QoI: 2e-4.
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _basis(n, ru, seed):
    h = 1.0 / (n - 1)
    d = (n - 2) ** 2
    Phi = np.linalg.qr(random_state_like(seed, (d, ru)))[0] / h     # h^2 Phi^T Phi = I
    ubar = 0.3 * random_state_like(seed + 1, (d,))
    phi_full = np.zeros((ru, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(ru, n - 2, n - 2)
    ub_full = np.zeros((n, n))
    ub_full[1:-1, 1:-1] = ubar.reshape(n - 2, n - 2)
    return Phi, ubar, phi_full, ub_full


def _dino(n, L, ru, N, seed, rm=16, width=32):
    from paper_2305_20053_gb300 import capi
    D = capi.Dino(n=n, lattice_L=L, r_m=rm, r_u=ru, width=width, max_batch=64, max_eval=N)
    Ws, bs = glorot_uniform_mlp([rm + L * L, width, width, width, ru], seed=seed)
    D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
    Phi, ubar, phi_full, ub_full = _basis(n, ru, seed + 10)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.tensor(ub_full, device="cuda"))
    return D, Phi, ubar


def _check(D, Phi, ubar, n, N, seed):
    h = 1.0 / (n - 1)
    ru = Phi.shape[1]
    coef = (0.5 * random_state_like(seed, (N, ru))).astype(np.float32)
    u = torch.full((N, n, n), float("nan"), dtype=torch.float32, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    D.ouu_dino_decode(torch.tensor(coef, device="cuda"), N, u, q)
    u, q = u.cpu().numpy(), q.cpu().numpy()
    ref = dino.decode_states(coef.astype(np.float64), Phi, ubar)
    ut = field.target_state(n)[1:-1, 1:-1].ravel()
    qref = dino.decoded_qoi(ref, ut, h)
    inner = u[:, 1:-1, 1:-1].reshape(N, -1)
    worst = max(rel(inner[i], ref[i]) for i in range(N))
    assert worst <= 5e-5, worst
    assert np.all(u[:, 0, :] == 0) and np.all(u[:, -1, :] == 0) and np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    np.testing.assert_allclose(q, qref, rtol=2e-4)


@pytest.mark.parametrize("ru", [12, 200])
def test_decode_33x33_ragged(ru):
    n, N = 33, 300
    D, Phi, ubar = _dino(n, 3, ru, N, seed=400 + ru)
    for rep in range(2):   # the second call reuses the handle's operand buffers
        _check(D, Phi, ubar, n, N, seed=410 + rep)
    D.close()


def test_decode_129x129_4096():
    n, N = 129, 4096
    D, Phi, ubar = _dino(n, 10, 200, N, seed=420, rm=200, width=64)
    _check(D, Phi, ubar, n, N, seed=421)
    D.close()


def test_eval_decoded_states_and_reduced_qoi():
    n, N, L = 33, 200, 3
    D, Phi, ubar = _dino(n, L, 12, N, seed=430)
    D.ouu_dino_set_output_scale(np.linspace(0.3, 0.05, 12).astype(np.float32))
    m = torch.tensor(field.sample_fields(SEED_SAA, 0, N, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    phi = torch.empty(N, 12, dtype=torch.float32, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    u = torch.empty(N, n, n, dtype=torch.float32, device="cuda")
    D.ouu_dino_eval(m, N, z, phi, None, q, None, u)
    u2 = torch.empty_like(u)
    qd = torch.empty(N, dtype=torch.float64, device="cuda")
    D.ouu_dino_decode(phi, N, u2, qd)
    np.testing.assert_array_equal(u.cpu().numpy(), u2.cpu().numpy())
    np.testing.assert_allclose(qd.cpu().numpy(), q.cpu().numpy(), rtol=2e-4)
    D.close()
