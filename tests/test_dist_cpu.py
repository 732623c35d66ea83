"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2): the one sample set split
into contiguous blocks of the same Philox stream (together exactly the single-process set,
also when the size does not divide evenly), and the job time as the maximum over ranks.
The exchange of one evaluation over those blocks is tested in test_shard_cpu.py."""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_samples():
    import bench
    assert bench.split_samples(4096, 1) == [(0, 4096)]
    assert bench.split_samples(4096, 8) == [(512 * r, 512) for r in range(8)]
    assert bench.split_samples(7, 3) == [(0, 3), (3, 2), (5, 2)]


@pytest.mark.parametrize("n_total", [6, 7])
def test_two_rank_gloo(tmp_path, n_total):
    import torch.multiprocessing as mp

    import dist_worker
    from oracle import field
    from synthetic_inputs import SEED_SAA

    port = _free_port()
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=dist_worker.worker, args=(r, 2, port, n_total, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = [np.load(o) for o in outs]
    assert int(res[0]["first"]) == 0 and int(res[1]["first"]) == int(res[0]["count"])
    assert sum(int(x["count"]) for x in res) == n_total
    both = np.concatenate([x["ms"] for x in res])
    np.testing.assert_array_equal(both, field.sample_fields(SEED_SAA, 0, n_total, 9))
    assert all(float(x["mx"]) == 15.0 for x in res)
