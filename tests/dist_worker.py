"""Child process of the world-size-2 gloo test (test_dist_cpu.py): the multi-rank host logic
of bench.py on CPU, with the oracle standing in for the GPU evaluation."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def worker(rank, world, port, n_total, out_path):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch

    import bench
    from oracle import field
    from synthetic_inputs import SEED_SAA

    r, w, _ = bench.dist_env()
    dist = bench.dist_init(w, backend="gloo")
    first, count = bench.split_samples(n_total, w)[r]
    ms = field.sample_fields(SEED_SAA, first, count, 9)
    bench.barrier(dist)
    my_ms = 10.0 + 5.0 * r   # a per-rank step time: the job's time is the slowest rank's
    mx = bench.max_over_ranks(dist, my_ms, torch.device("cpu"))
    np.savez(out_path, first=first, count=count, ms=ms, mx=mx)
    dist.destroy_process_group()


def shard_worker(rank, world, port, counts, out_path):
    """One rank of a sample set spread over ranks (paper_2305_20053_gb300.shard), on CPU: the
    oracle stands in for the library's two phases; the exchange plan and its collectives
    (all-gather of the QoIs, FP64 all-reduce of the gradient parts) are the product's."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist

    from oracle import field, pde, risk
    from paper_2305_20053_gb300.shard import ShardedSAA
    from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, controls

    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, L = 9, 2
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    ut = field.target_state(n)
    z = controls(SEED_EVAL_Z, 1, L * L)[0]
    plan = ShardedSAA(counts[rank], "cpu")
    first, count = plan.first, plan.n_local
    refs = pde.solve_batch(field.sample_fields(SEED_SAA, first, count, n), z, G, ut, prob)
    Q = np.array([x.q for x in refs])
    Gq = np.stack([x.grad for x in refs])

    def qoi():
        return torch.tensor(Q)

    def partial(q_all, n_total, first_local):
        q_all = q_all.numpy()
        Gpad = np.zeros((n_total, Gq.shape[1]))    # only this rank's rows: w @ Gpad = its part
        Gpad[first_local:first_local + count] = Gq
        v1, g1, dt1, t1 = risk.cvar(q_all, Gpad, 0.95, 1e-4)
        v0, g0 = risk.mean_var(q_all, Gpad, 1.0)
        return np.array([v1, v0]), np.stack([g1, g0]), np.array([dt1, 0.0]), np.array([t1, 0.0])

    rho, g, gt, t = plan.evaluate(qoi, partial)
    np.savez(out_path, rho=rho, g=g, gt=gt, t=t, first=first, n_total=plan.n_total, counts=np.array(plan.counts))
    dist.destroy_process_group()
