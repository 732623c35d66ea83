"""What the trained reduced-basis network gains (Sec. 3-4), measured against the plain PDE
SAA path on the GPU, on a small problem (33 x 33 grid, 5 x 5 controls, N = 512 samples):

* the trained MR-DINO gives the risks (smoothed CVaR_0.9, mean + variance) and their
  z-gradients far more accurately than the same network untrained;
* derivative-informed training (the Jacobian term of the Sec. 3.4 loss) gives more accurate
  risk gradients than the same network trained on the state misfit alone (MR-NO, w_J = 0),
  the paper's central claim;
* one MR-DINO evaluation of the risk and its gradient is at least 10x faster than the plain
  path (Newton + adjoint solves), even at this size.

Errors are relative, averaged over three seeded controls.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_GRID, L, R, WIDTH, N_TRAIN, EPOCHS, N_SAA = 33, 5, 48, 128, 2048, 60, 512


@pytest.fixture(scope="module")
def trained():
    from paper_2305_20053_gb300 import build, capi
    from paper_2305_20053_gb300 import train as T
    from synthetic_inputs import SEED_SAA
    build.build()
    capi.load()
    P = capi.Problem(n=N_GRID, lattice_L=L, max_samples=N_TRAIN)
    nets = {}
    data = None
    for name, wj in (("untrained", 1.0), ("dino", 1.0), ("no", 0.0)):
        D = capi.Dino(n=N_GRID, lattice_L=L, r_m=R, r_u=R, width=WIDTH, max_batch=256, max_eval=N_SAA,
                      jac_weight=wj)
        T.init_params(D)
        if data is None:
            data = T.generate_training_data(P, D, N_TRAIN)
            phi = torch.empty(R, N_GRID, N_GRID, dtype=torch.float64, device="cuda")
            ub = torch.empty(N_GRID, N_GRID, dtype=torch.float64, device="cuda")
            D.ouu_dino_get_bases(phi, ub)
            scale = D.ouu_dino_get_output_scale()
        else:   # the same POD basis and output scale for every network
            D.ouu_dino_set_bases(phi, ub)
            D.ouu_dino_set_output_scale(np.asarray(scale, dtype=np.float32))
        if name != "untrained":
            T.train(D, data, epochs=EPOCHS, batch=256, lr_final=1e-5)
        nets[name] = D
    m = torch.empty(N_SAA, N_GRID, N_GRID, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 0, N_SAA, m)
    return P, nets, m


def _errors(P, D, m, zs, risks):
    from paper_2305_20053_gb300 import capi
    er, eg = [], []
    for z in zs:
        v0, g0, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N_SAA, risks, z)
        v1, g1, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N_SAA, risks, z)
        er.append(np.abs(v1 - v0) / np.abs(v0))
        eg.append(np.linalg.norm(g1 - g0, axis=1) / np.linalg.norm(g0, axis=1))
    return np.mean(er, axis=0), np.mean(eg, axis=0)


def test_training_and_derivative_information_gain(trained):
    from paper_2305_20053_gb300 import capi
    from synthetic_inputs import SEED_EVAL_Z, controls
    P, nets, m = trained
    zs = controls(SEED_EVAL_Z, 3, L * L)
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
    err = {k: _errors(P, D, m, zs, risks) for k, D in nets.items()}
    (r_u, g_u), (r_d, g_d), (r_n, g_n) = err["untrained"], err["dino"], err["no"]
    # training: gradients at least 5x more accurate than the untrained network, risks accurate
    assert np.all(g_d * 5 <= g_u), (g_d, g_u)
    assert np.all(r_d <= 0.05), r_d
    # derivative-informed training beats the state-only loss on the risk gradients
    assert np.all(g_d < g_n), (g_d, g_n)


def test_surrogate_speed_gain(trained):
    from paper_2305_20053_gb300 import capi
    from synthetic_inputs import SEED_EVAL_Z, controls
    P, nets, m = trained
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1)]

    def rate(backend, D, reps):
        for _ in range(2):
            P.ouu_risk_and_grad(backend, D, m, N_SAA, risks, z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            P.ouu_risk_and_grad(backend, D, m, N_SAA, risks, z)
        torch.cuda.synchronize()
        return reps / (time.perf_counter() - t0)

    pde = rate(capi.BACKEND_PDE, None, 3)
    dino = rate(capi.BACKEND_DINO, nets["dino"], 20)
    assert dino >= 10 * pde, (dino, pde)
