"""The allocation-free state solve (ouu_pde_solve_batch_noalloc) gives the same
states, QoIs and statuses as ouu_pde_solve_batch, on two calls in a row.

It is meant for callers that cannot allocate device memory when they call in (a
device-memory budget or pool that forbids new allocations, or a host application
that owns every device buffer); its scratch is a fixed device array in the
library.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.  Tolerances: states 1e-9 (relative l2), QoIs 1e-9 (relative).
"""
import numpy as np
import pytest

from gpu_util import rel
from synthetic_inputs import SEED_EVAL_Z, SEED_SAA, SEED_TRAIN_Z, controls

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solve_both(n, L, N, per_sample):
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()
    P = capi.Problem(n=n, lattice_L=L, max_samples=N)
    m = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 0, N, m)
    if per_sample:
        z = torch.tensor(controls(SEED_TRAIN_Z, N, L * L), device="cuda")
        stride = L * L
    else:
        z = torch.tensor(controls(SEED_EVAL_Z, 1, L * L)[0], device="cuda")
        stride = 0
    u_ref = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    q_ref = torch.empty(N, dtype=torch.float64, device="cuda")
    s_ref = torch.empty(N, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, N, z, stride, u_ref, q_ref, s_ref)
    outs, free_bytes = [], []
    bufs = [(torch.full((N, n, n), float("nan"), dtype=torch.float64, device="cuda"),
             torch.empty(N, dtype=torch.float64, device="cuda"),
             torch.empty(N, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    for u, q, s in bufs:   # two calls in a row share (and must clear) the fixed scratch
        capi.ouu_pde_solve_batch_noalloc(capi.problem_desc(n=n, lattice_L=L), m, N, z, stride, u, q, s)
        torch.cuda.synchronize()
        free_bytes.append(torch.cuda.mem_get_info()[0])
    for u, q, s in bufs:
        outs.append((u.cpu().numpy(), q.cpu().numpy(), s.cpu().numpy()))
    P.close()
    return (u_ref.cpu().numpy(), q_ref.cpu().numpy(), s_ref.cpu().numpy()), outs, free_bytes


# (33, 5, 4100): more samples than one launch takes (4096), so the per-launch offsets of
# the fields, controls, outputs and statuses, and the status read-back in blocks of 1024,
# run more than once.
@pytest.mark.parametrize("n,L,N,per_sample", [(33, 5, 48, True), (129, 10, 24, False), (33, 5, 4100, True)])
def test_noalloc_matches_existing_entry_point(n, L, N, per_sample):
    (u_ref, q_ref, s_ref), outs, free_bytes = _solve_both(n, L, N, per_sample)
    assert np.all(s_ref == 0)
    # the second call found the scratch already in place: device memory did not shrink
    assert free_bytes[1] == free_bytes[0]
    for u, q, s in outs:
        np.testing.assert_array_equal(s, s_ref)
        for i in range(N):
            assert rel(u[i], u_ref[i]) <= 1e-9, i
        assert np.all(np.abs(q - q_ref) <= 1e-9 * np.abs(q_ref))


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()
    n, N = 513, 1
    m = torch.zeros(N, n, n, dtype=torch.float64, device="cuda")
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    u = torch.empty(N, n, n, dtype=torch.float64, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    s = torch.empty(N, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.OuuError) as e:
        capi.ouu_pde_solve_batch_noalloc(capi.problem_desc(n=n, lattice_L=2), m, N, z, 0, u, q, s)
    assert e.value.status == 1 and "scratch" in str(e.value)
