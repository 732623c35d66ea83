"""One sample set spread over two ranks (gloo, CPU): the exchange plan of
paper_2305_20053_gb300.shard (an all-gather of the QoIs, then an FP64 all-reduce of the
per-rank weighted gradient sums) gives the risk, its z-gradient, d rho / dt and t* of the
whole set (Sec. 2.2 SAA, Sec. 2.3 gradient), with the oracle standing in for each rank's
device phases: equal to the single-process oracle to 1e-12 relative, for mean + variance and
the smoothed CVaR_0.95 at t*, with blocks of unequal size."""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("counts", [(7, 5), (6, 6)])
def test_two_rank_sample_set(tmp_path, counts):
    import torch.multiprocessing as mp

    import dist_worker
    from oracle import field, pde, risk
    from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls

    port = _free_port()
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=dist_worker.shard_worker, args=(r, 2, port, list(counts), outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = [np.load(o) for o in outs]
    N = sum(counts)
    assert [int(x["first"]) for x in res] == [0, counts[0]] and all(int(x["n_total"]) == N for x in res)
    # the whole set in one process
    n, L = 9, 2
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    refs = pde.solve_batch(field.sample_fields(SEED_SAA, 0, N, n), z, G, field.target_state(n), prob)
    Q = np.array([x.q for x in refs])
    Gq = np.stack([x.grad for x in refs])
    v1, g1, dt1, t1 = risk.cvar(Q, Gq, 0.95, 1e-4)
    v0, g0 = risk.mean_var(Q, Gq, 1.0)
    for x in res:
        np.testing.assert_allclose(x["rho"], [v1, v0], rtol=1e-12)
        np.testing.assert_allclose(x["g"][0], g1, rtol=1e-12, atol=1e-15 * np.abs(g1).max())
        np.testing.assert_allclose(x["g"][1], g0, rtol=1e-12, atol=1e-15 * np.abs(g0).max())
        assert float(x["t"][0]) == t1 and float(x["gt"][0]) == pytest.approx(dt1, abs=1e-12)
    # both ranks hold the same result
    np.testing.assert_array_equal(res[0]["g"], res[1]["g"])
