"""The multi-rank path of bench.py on CPU (gloo, world size 2): disjoint per-rank sample
ranges of one Philox stream (weak scaling, no collective on the data path), the job time as
the maximum over ranks, and the whole-job rate; each rank's risk equals the single-process
evaluation of its own range."""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo(tmp_path):
    import torch.multiprocessing as mp

    import dist_worker
    from oracle import field, pde, risk
    from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls

    port, n_per = _free_port(), 3
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=dist_worker.worker, args=(r, 2, port, n_per, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = [np.load(o) for o in outs]
    assert [int(x["first"]) for x in res] == [0, n_per] and all(int(x["count"]) == n_per for x in res)
    both = np.concatenate([x["ms"] for x in res])
    np.testing.assert_array_equal(both, field.sample_fields(SEED_SAA, 0, 2 * n_per, 9))
    assert all(float(x["mx"]) == 15.0 for x in res)
    assert all(abs(float(x["rate"]) - 2 * 4 / 0.015) < 1e-9 for x in res)
    # each rank's risk is the single-process evaluation of its own range
    prob = pde.Problem(n=9, L=2)
    G = field.control_sources(9, 2, prob.width)
    z = controls(SEED_EVAL_Z, 1, 4)[0]
    for x in res:
        refs = pde.solve_batch(x["ms"], z, G, field.target_state(9), prob)
        rho, g = risk.mean_var(np.array([r.q for r in refs]), np.stack([r.grad for r in refs]), 1.0)
        assert float(x["rho"]) == rho and np.array_equal(x["g"], g)
