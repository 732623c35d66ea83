"""Projected control Jacobians of Sec. 3.4 (the DINO training targets) by both routes on the GPU:
forward (d_Z linearised solves per sample) and adjoint (r_u solves of J lam = M Phi_r, J
symmetric), each against the oracle's Phi^T M J^-1 G (oracle/pde.py projected_jacobian) at the
oracle's states.  17 x 17 grid, 25 controls and 12 POD modes, so the default picks the adjoint
route; 6 samples (the oracle's field draws and states on both sides).  Tolerance 1e-4 relative
l2 (FP32 MG-PCG at cg_rtol 1e-6, FP32 projections), as for the forward-route data elsewhere."""
import numpy as np
import pytest

from gpu_util import rel
from oracle import field, pde
from synthetic_inputs import SEED_TRAIN_FIELDS, SEED_TRAIN_Z, controls, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def test_forward_and_adjoint_routes_against_oracle():
    from paper_2305_20053_gb300 import capi
    n, L, RU, N = 17, 5, 12, 6
    dz, h = L * L, 1.0 / (n - 1)
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    G_int = pde.interior_rows(G, n)
    ms = field.sample_fields(SEED_TRAIN_FIELDS, 0, N, n)
    zs = controls(SEED_TRAIN_Z, N, dz)
    Phi = np.linalg.qr(random_state_like(501, ((n - 2) ** 2, RU)))[0] / h
    us, ref = [], []
    for i in range(N):
        kx, ky = pde.face_coefficients(ms[i])
        u, chol = pde.newton_solve(kx, ky, (G @ zs[i]).reshape(n, n), prob.r, h)
        us.append(u)
        ref.append(pde.projected_jacobian(chol, G_int, Phi, h, "forward").T)   # [dz][ru]
    ref = np.stack(ref)
    D = capi.Dino(n=n, lattice_L=L, r_m=8, r_u=RU, width=16, max_batch=8, max_eval=8)
    phi_full = np.zeros((RU, n, n))
    phi_full[:, 1:-1, 1:-1] = Phi.T.reshape(RU, n - 2, n - 2)
    D.ouu_dino_set_bases(torch.tensor(phi_full, device="cuda"), torch.zeros(n, n, dtype=torch.float64, device="cuda"))
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    m_t, u_t = torch.tensor(ms, device="cuda"), torch.tensor(np.stack(us), device="cuda")
    out = {}
    for route in (1, 2, 0):
        D.ouu_dino_set_jacobian_route(route)
        jy = torch.full((N, dz, RU), float("nan"), dtype=torch.float32, device="cuda")
        D.ouu_dino_jacobian_data(P, m_t, u_t, N, jy)
        out[route] = jy.cpu().numpy()
        assert rel(out[route], ref) <= 1e-4, (route, rel(out[route], ref))
    np.testing.assert_array_equal(out[0], out[2])   # the default took the adjoint route (25 > 12)
    with pytest.raises(capi.OuuError):
        D.ouu_dino_set_jacobian_route(3)
    P.close()
    D.close()
