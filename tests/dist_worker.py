"""Child process of the world-size-2 gloo test (test_dist_cpu.py): the multi-rank host logic
of bench.py on CPU, with the oracle standing in for the GPU evaluation."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def worker(rank, world, port, n_per_rank, out_path):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch

    import bench
    from oracle import field, pde, risk
    from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls

    r, w, _ = bench.dist_env()
    dist = bench.dist_init(w, backend="gloo")
    first, count = bench.rank_samples(r, n_per_rank)
    n, L = 9, 2
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    ms = field.sample_fields(SEED_SAA, first, count, n)
    refs = pde.solve_batch(ms, z, G, ut, prob)
    Q = np.array([x.q for x in refs])
    Gq = np.stack([x.grad for x in refs])
    rho, g = risk.mean_var(Q, Gq, 1.0)
    bench.barrier(dist)
    my_ms = 10.0 + 5.0 * r   # a per-rank step time: the job's time is the slowest rank's
    mx = bench.max_over_ranks(dist, my_ms, torch.device("cpu"))
    rate = bench.job_rate(w, 4, mx)
    np.savez(out_path, first=first, count=count, ms=ms, rho=rho, g=g, mx=mx, rate=rate)
    dist.destroy_process_group()
