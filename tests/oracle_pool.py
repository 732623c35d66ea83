"""The oracle's plain path (FP64 Newton with a banded Cholesky solve, adjoint gradient) over
many fields, in spawned single-threaded processes: the reference of the full-size parity
tests.  Each worker draws its own block of fields from the oracle's generator."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _solve_block(args):
    seed, first, count, n, L, z = args
    sys.path.insert(0, ROOT)
    import numpy as np

    from oracle import field, pde
    prob = pde.Problem(n=n, L=L)
    G = field.control_sources(n, L, prob.width)
    refs = pde.solve_batch(field.sample_fields(seed, first, count, n), z, G, field.target_state(n), prob,
                           with_adjoint=True)
    return np.array([r.q for r in refs]), np.stack([r.grad for r in refs])


def qoi_and_gradients(seed, N, n, L, z, workers=None):
    """(Q [N], grad_z Q [N][d_Z]) of fields 0 .. N-1 of `seed` at the shared control z."""
    import multiprocessing as mp

    import numpy as np
    workers = workers or max(1, os.cpu_count() or 1)
    block = -(-N // (4 * workers))
    jobs = [(seed, f, min(block, N - f), n, L, z) for f in range(0, N, block)]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})   # read by each child when it imports numpy
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_solve_block, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
