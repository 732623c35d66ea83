"""A sample set spread over ranks, emulated on one GPU: two problem handles hold the two
blocks of the set (as two ranks would), their phases run one after the other, the QoIs are
concatenated (the all-gather) and the gradient parts added (the all-reduce).  No kernel waits
on another rank's.

* plain path, 33 x 33, N = 48 in blocks of 30 and 18: equal to ouu_risk_and_grad over the
  whole set to 1e-12 relative (same per-sample solves; only the order of the final sums
  differs), and to the FP64 oracle to 1e-8 (risk values and gradients);
* MR-DINO, 33 x 33, N = 300 in blocks of 128 and 172: equal to ouu_risk_and_grad over the
  whole set to 1e-6 (values) and 1e-4 (gradients): the projection splits its FP32 sums over K
  differently for other sample counts (a deterministic difference of about 1e-7 in the
  coordinates), and the weighted gradient sums cancel strongly;
* one rank through paper_2305_20053_gb300.shard (no process group): ouu_risk_and_grad's results;
* phase 2 without a pending phase 1, and a block outside the set, are refused.
"""
import numpy as np
import pytest

from gpu_util import rel
from oracle import field, pde, risk
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def _risks():
    from paper_2305_20053_gb300 import capi
    return [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.9, eps=1e-4, t_optimal=1),
            capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]


def _emulate(blocks, backend, dinos, m, z, risks):
    """Phases of every block in turn on its own problem handle and network (dinos[k], as each
    rank holds its own); returns the merged (risk, grad, grad_t, t)."""
    from paper_2305_20053_gb300 import capi
    n, L = m.shape[1], int(round(np.sqrt(len(z))))
    handles, qs, first = [], [], 0
    for k, cnt in enumerate(blocks):
        P = capi.Problem(n=n, lattice_L=L, max_samples=cnt)
        q = torch.empty(cnt, dtype=torch.float64, device="cuda")
        P.ouu_shard_qoi(backend, dinos[k], m[first:first + cnt], cnt, z, q)
        handles.append((P, first, dinos[k]))
        qs.append(q)
        first += cnt
    q_all = torch.cat(qs)
    outs = [P.ouu_shard_risk_partial(d, q_all, first, f, risks) for P, f, d in handles]
    for P, _, _ in handles:
        P.close()
    for o in outs[1:]:   # values, d rho / dt and t are computed from all QoIs on every rank
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[3], outs[0][3])
    return outs[0][0], sum(o[1] for o in outs), outs[0][2], outs[0][3]


def test_plain_path_two_blocks():
    from paper_2305_20053_gb300 import capi
    n, L, N = 33, 5, 48
    ms = field.sample_fields(SEED_SAA, 0, N, n)
    m = torch.tensor(ms, device="cuda")
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    risks = _risks()
    rho, g, gt, t = _emulate([30, 18], capi.BACKEND_PDE, [None, None], m, z, risks)
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    v0, g0, gt0, t0, _ = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, N, risks, z)
    np.testing.assert_allclose(rho, v0, rtol=1e-12)
    assert rel(g[0], g0[0]) <= 1e-12 and rel(g[1], g0[1]) <= 1e-12
    np.testing.assert_array_equal(t, t0)
    np.testing.assert_allclose(gt, gt0, rtol=1e-12, atol=1e-14)
    # and the oracle over the whole set
    prob = pde.Problem(n=n, L=L)
    refs = pde.solve_batch(ms, z, field.control_sources(n, L, prob.width), field.target_state(n), prob)
    Q = np.array([x.q for x in refs])
    Gq = np.stack([x.grad for x in refs])
    v1, g1, _, t1 = risk.cvar(Q, Gq, 0.9, 1e-4)
    vm, gm = risk.mean_var(Q, Gq, 1.0)
    np.testing.assert_allclose(rho, [v1, vm], rtol=1e-8)
    assert rel(g[0], g1) <= 1e-8 and rel(g[1], gm) <= 1e-8
    # one rank through the exchange plan (no process group): the same as ouu_risk_and_grad
    from paper_2305_20053_gb300 import shard
    plan = shard.ShardedSAA(N, "cuda")
    assert plan.world == 1 and plan.n_total == N and plan.first == 0
    r1, g1s, _, t1s = shard.risk_and_grad(P, capi.BACKEND_PDE, None, m, risks, z, plan)
    np.testing.assert_allclose(r1, v0, rtol=1e-12)
    assert rel(g1s[0], g0[0]) <= 1e-12 and rel(g1s[1], g0[1]) <= 1e-12
    P.close()


def test_dino_two_blocks():
    from paper_2305_20053_gb300 import capi
    n, L, N, RM, RU, W = 33, 5, 300, 16, 12, 64
    dz, h = L * L, 1.0 / (n - 1)
    Ws, bs = glorot_uniform_mlp([RM + dz, W, W, W, RU], seed=301)
    bs = [0.1 * random_state_like(302 + l, b.shape) for l, b in enumerate(bs)]
    Qm, _ = np.linalg.qr(random_state_like(307, ((n - 2) ** 2, RU)))
    phi = np.zeros((RU, n, n))
    phi[:, 1:-1, 1:-1] = (Qm / h).T.reshape(RU, n - 2, n - 2)
    ub = np.zeros((n, n))
    ub[1:-1, 1:-1] = 0.05 * random_state_like(308, (n - 2, n - 2))
    nets = []
    for _ in range(3):   # one per emulated rank, and one for the whole set
        D = capi.Dino(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=64, max_eval=N)
        D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
        D.ouu_dino_set_output_scale(np.linspace(0.5, 0.1, RU).astype(np.float32))
        D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.tensor(ub, device="cuda"))
        nets.append(D)
    m = torch.tensor(field.sample_fields(SEED_SAA, 0, N, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, dz)[0]
    risks = _risks()
    rho, g, gt, t = _emulate([128, 172], capi.BACKEND_DINO, nets[:2], m, z, risks)
    D = nets[2]
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    v0, g0, _, t0, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
    np.testing.assert_allclose(rho, v0, rtol=1e-6)
    assert rel(g[0], g0[0]) <= 1e-4 and rel(g[1], g0[1]) <= 1e-4, (rel(g[0], g0[0]), rel(g[1], g0[1]))
    # a network that evaluated other samples between the phases is refused
    q = torch.empty(128, dtype=torch.float64, device="cuda")
    P1 = capi.Problem(n=n, lattice_L=L, max_samples=128)
    P1.ouu_shard_qoi(capi.BACKEND_DINO, D, m[:128], 128, z, q)
    P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, N, risks, z)
    with pytest.raises(capi.OuuError) as e:
        P1.ouu_shard_risk_partial(D, q, 128, 0, risks)
    assert e.value.status == 6
    P1.close()
    P.close()
    for D in nets:
        D.close()


def test_phase_order_and_block_checks():
    from paper_2305_20053_gb300 import capi
    n, L, N = 17, 3, 8
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    q_all = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.OuuError) as e:
        P.ouu_shard_risk_partial(None, q_all, 2 * N, 0, _risks())
    assert e.value.status == 6
    m = torch.tensor(field.sample_fields(SEED_SAA, 0, N, n), device="cuda")
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    P.ouu_shard_qoi(capi.BACKEND_PDE, None, m, N, z, q_all[:N])
    with pytest.raises(capi.OuuError) as e:
        P.ouu_shard_risk_partial(None, q_all, 2 * N, N + 1, _risks())
    assert e.value.status == 1
    P.ouu_shard_risk_partial(None, q_all, 2 * N, N, _risks())   # the pending phase 1 is still there
    with pytest.raises(capi.OuuError) as e:                    # and is consumed by it
        P.ouu_shard_risk_partial(None, q_all, 2 * N, N, _risks())
    assert e.value.status == 6
    P.close()
