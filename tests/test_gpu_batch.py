"""Uneven batches (many OUU problems in one graph: the plain problems' solves in one
persistent launch per solve kind, MR-DINO problems on concurrent branches) against the
same problems evaluated one call at a time, and against the FP64 oracle (the items' fields
are the oracle's draws): plain items' risks and gradients to 1e-8 relative; MR-DINO items
against the oracle surrogate with the CUDA path's BF16 roundings, values 1e-3 and gradients
2e-2 (CVaR) / 1e-2 (mean + variance).

Plain items: risk values and t within 1e-12 relative (the per-sample solves are the same
arithmetic; only the FP64 sum of the slot accumulators runs in another order), gradients
within 1e-10 relative.  MR-DINO items: within 1e-6 (the projection's FP32 split sums are
added atomically).  Two runs with different controls; the tile autotuner must have timed
the networks' GEMM shapes; per-item and total times are positive.
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import dino, field, pde, risk
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PLAIN = [(33, 5, 64), (17, 3, 37), (65, 4, 100), (9, 2, 5), (33, 3, 20), (17, 2, 1)]
DINO = [(17, 3, 48), (33, 5, 30)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _risks(k):
    from paper_2305_20053_gb300 import capi
    rs = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1),
          capi.risk_desc(capi.RISK_MEAN_VAR, kappa=0.5 + k)]
    return rs[: 1 + k % 2] if k % 3 else rs


def _oracle_risks(Q, G, risks):
    """(values, gradients) of the item's risk descriptors by the oracle's formulas."""
    vals, grads = [], []
    for rd in risks:
        if rd.kind == 0:
            v, g = risk.mean_var(Q, G, rd.kappa)
        else:
            v, g, _, _ = risk.cvar(Q, G, rd.beta, rd.eps)
        vals.append(v)
        grads.append(g)
    return np.array(vals), np.stack(grads)


def _network(n, L, seed):
    """A small network with an M-orthonormal random basis (the evaluation path only); also
    returns the oracle's copy (FP32-rounded weights, same scale and basis)."""
    from paper_2305_20053_gb300 import capi
    RM = RU = 12
    W = 32
    dz, h = L * L, 1.0 / (n - 1)
    widths = [RM + dz, W, W, W, RU]
    Ws, bs = glorot_uniform_mlp(widths, seed=seed)
    bs = [0.1 * random_state_like(seed + 10 + l, b.shape) for l, b in enumerate(bs)]
    D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=64)
    flat = capi.flatten_params(Ws, bs)
    D.ouu_dino_set_params(flat)
    scale = np.linspace(0.05, 0.01, RU).astype(np.float32)
    D.ouu_dino_set_output_scale(scale)
    d = (n - 2) ** 2
    Q, _ = np.linalg.qr(random_state_like(seed + 20, (d, RU)))
    phi = np.zeros((RU, n, n))
    phi[:, 1:-1, 1:-1] = (Q / h).T.reshape(RU, n - 2, n - 2)
    ub = np.zeros((n, n))
    ub[1:-1, 1:-1] = 0.05 * random_state_like(seed + 21, (n - 2, n - 2))
    D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.tensor(ub, device="cuda"))
    Ws64, bs64 = capi.unflatten_params(flat, widths)
    net = dino.MLP(Ws64, bs64, RM, out_scale=scale.astype(np.float64))
    return D, (net, Q / h, ub[1:-1, 1:-1].ravel(), RM)


def test_uneven_batch_matches_single_calls():
    from paper_2305_20053_gb300 import capi
    items = []
    for k, (n, L, N) in enumerate(PLAIN):
        P = capi.Problem(n=n, lattice_L=L, max_samples=N)
        ms = field.sample_fields(SEED_SAA, 100 * k, N, n)
        items.append(dict(problem=P, backend=capi.BACKEND_PDE, dino=None, m=torch.tensor(ms, device="cuda"), ms=ms,
                          n=N, L=L, risks=_risks(k)))
    for j, (n, L, N) in enumerate(DINO):
        P = capi.Problem(n=n, lattice_L=L, max_samples=N)
        ms = field.sample_fields(SEED_SAA, 1000 + j, N, n)
        D, orc = _network(n, L, 40 + j)
        items.append(dict(problem=P, backend=capi.BACKEND_DINO, dino=D, orc=orc, m=torch.tensor(ms, device="cuda"),
                          ms=ms, n=N, L=L, risks=_risks(j + 1)))
    before = capi.load().ouu_kernel_gemm_tuned_shapes()
    B = capi.Batch(items, autotune=True)
    assert capi.load().ouu_kernel_gemm_tuned_shapes() > before
    for rep in range(2):
        zs = [controls(SEED_EVAL_Z + rep, 1 + k, it["problem"].d_z)[k] for k, it in enumerate(items)]
        res, item_ms, total_ms = B.run(zs)
        assert total_ms > 0 and np.all(item_ms > 0)
        for k, it in enumerate(items):
            v0, g0, gt0, t0, _ = it["problem"].ouu_risk_and_grad(it["backend"], it["dino"], it["m"], it["n"],
                                                                 it["risks"], zs[k])
            v1, g1, gt1, t1 = res[k]
            tol_v, tol_g = (1e-12, 1e-10) if it["backend"] == capi.BACKEND_PDE else (1e-6, 1e-6)
            np.testing.assert_allclose(v1, v0, rtol=tol_v)
            np.testing.assert_allclose(t1, t0, rtol=tol_v, atol=1e-300)
            for r in range(len(it["risks"])):
                assert rel(g1[r], g0[r]) <= tol_g, (k, r, rel(g1[r], g0[r]))
            if rep == 0:   # and the oracle on the item's own fields
                n, L, N = it["ms"].shape[1], it["L"], it["n"]
                if it["backend"] == capi.BACKEND_PDE:
                    prob = pde.Problem(n=n, L=L)
                    refs = pde.solve_batch(it["ms"], zs[k], field.control_sources(n, L, prob.width),
                                           field.target_state(n), prob)
                    vo, go = _oracle_risks(np.array([x.q for x in refs]), np.stack([x.grad for x in refs]),
                                           it["risks"])
                    np.testing.assert_allclose(v1, vo, rtol=1e-8)
                    for r in range(len(it["risks"])):
                        assert rel(g1[r], go[r]) <= 1e-8, (k, r)
                else:
                    net, Phi, ubar, RM = it["orc"]
                    Wkl, _ = dino.kl_projection_matrix(n, RM)
                    xi = dino.project_fields(it["ms"].reshape(N, -1), Wkl, bf16=True)
                    ut = field.target_state(n)[1:-1, 1:-1].ravel()
                    Qo, Go, _, _ = dino.eval_surrogate(net, xi, zs[k], Phi, ubar, ut, 1.0 / (n - 1), decode=False,
                                                       bf16=True)
                    vo, go = _oracle_risks(Qo, Go, it["risks"])
                    np.testing.assert_allclose(v1, vo, rtol=1e-3)
                    for r, rd in enumerate(it["risks"]):
                        assert rel(g1[r], go[r]) <= (2e-2 if rd.kind == 1 else 1e-2), (k, r, rel(g1[r], go[r]))
    B.close()


def test_batch_rejects_shared_problem():
    from paper_2305_20053_gb300 import capi
    P = capi.Problem(n=9, lattice_L=2, max_samples=4)
    m = torch.zeros(4, 9, 9, dtype=torch.float64, device="cuda")
    it = dict(problem=P, backend=capi.BACKEND_PDE, dino=None, m=m, n=4, risks=_risks(0))
    with pytest.raises(capi.OuuError):
        capi.Batch([it, dict(it)])
