"""Persistence of a surrogate.  Export (train.save_surrogate / load_surrogate, .npz): a fresh
handle gets the same parameters, output scale and POD basis (bit for bit) and gives the same
network outputs on the same projection coordinates (1e-12 relative: the same kernels on the
same state); a handle of another width refuses the archive.  Checkpoint (ouu_dino_save /
ouu_dino_load): the Adam state comes back too, so the next training step of the restored
network matches the original's; another network's file and a truncated file are refused."""
import numpy as np
import pytest

from synthetic_inputs import SEED_EVAL_Z, controls, glorot_uniform_mlp, random_state_like

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


def test_saved_surrogate_reloads_exactly(tmp_path):
    from paper_2305_20053_gb300 import capi, train
    n, L, RM, RU, W, N = 17, 3, 16, 12, 32, 40
    dz, h = L * L, 1.0 / (n - 1)
    Ws, bs = glorot_uniform_mlp([RM + dz, W, W, W, RU], seed=31)
    bs = [0.1 * random_state_like(32 + l, b.shape) for l, b in enumerate(bs)]
    kw = dict(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=16, max_eval=N)
    D = capi.Dino(**kw)
    D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
    D.ouu_dino_set_output_scale(np.linspace(0.05, 0.01, RU).astype(np.float32))
    Q, _ = np.linalg.qr(random_state_like(37, ((n - 2) ** 2, RU)))
    phi = np.zeros((RU, n, n))
    phi[:, 1:-1, 1:-1] = (Q / h).T.reshape(RU, n - 2, n - 2)
    ub = np.zeros((n, n))
    ub[1:-1, 1:-1] = 0.05 * random_state_like(38, (n - 2, n - 2))
    D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.tensor(ub, device="cuda"))

    path = str(tmp_path / "surrogate.npz")
    train.save_surrogate(D, path)
    D2 = capi.Dino(**kw)
    train.load_surrogate(D2, path)
    assert np.array_equal(D2.ouu_dino_get_params(), D.ouu_dino_get_params())
    assert np.array_equal(D2.ouu_dino_get_output_scale(), D.ouu_dino_get_output_scale())
    phi2 = torch.empty(RU, n, n, dtype=torch.float64, device="cuda")
    ub2 = torch.empty(n, n, dtype=torch.float64, device="cuda")
    D2.ouu_dino_get_bases(phi2, ub2)
    assert np.array_equal(phi2.cpu().numpy(), phi) and np.array_equal(ub2.cpu().numpy(), ub)

    xi = torch.tensor(random_state_like(39, (N, RM)).astype(np.float32), device="cuda")
    z = controls(SEED_EVAL_Z, 1, dz)[0]
    out = []
    for H in (D, D2):
        q = torch.empty(N, dtype=torch.float64, device="cuda")
        gq = torch.empty(N, dz, dtype=torch.float64, device="cuda")
        ph = torch.empty(N, RU, dtype=torch.float32, device="cuda")
        H.ouu_kernel_dino_network(xi, N, z, 2, q, ph, gq)
        out.append((q.cpu().numpy(), gq.cpu().numpy(), ph.cpu().numpy()))
    (q1, g1, p1), (q2, g2, p2) = out
    assert np.all(np.isfinite(q1)) and np.abs(g1).max() > 0
    np.testing.assert_allclose(q2, q1, rtol=1e-12)
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-12 * np.abs(g1).max())
    np.testing.assert_allclose(p2, p1, rtol=1e-12, atol=1e-12 * np.abs(p1).max())

    D3 = capi.Dino(**dict(kw, width=40))
    with pytest.raises(ValueError, match="width"):
        train.load_surrogate(D3, path)
    for H in (D, D2, D3):
        H.close()


def test_checkpoint_resumes_training(tmp_path):
    """A network restored from a checkpoint taken after one Adam step has the same parameters,
    output scale and bases, and its next step matches the original's to 1e-6 on parameters
    that the step moves by about 1e-3 (a restarted Adam would move them differently by O(lr))."""
    from paper_2305_20053_gb300 import capi
    n, L, RM, RU, W, B = 17, 3, 16, 12, 32, 16
    dz, h = L * L, 1.0 / (n - 1)
    kw = dict(n=n, lattice_L=L, r_m=RM, r_u=RU, width=W, max_batch=B, max_eval=B)
    Ws, bs = glorot_uniform_mlp([RM + dz, W, W, W, RU], seed=41)
    D = capi.Dino(**kw)
    D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
    D.ouu_dino_set_output_scale(np.linspace(0.05, 0.01, RU).astype(np.float32))
    Q, _ = np.linalg.qr(random_state_like(42, ((n - 2) ** 2, RU)))
    phi = np.zeros((RU, n, n))
    phi[:, 1:-1, 1:-1] = (Q / h).T.reshape(RU, n - 2, n - 2)
    ub = np.zeros((n, n))
    ub[1:-1, 1:-1] = 0.05 * random_state_like(43, (n - 2, n - 2))
    D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.tensor(ub, device="cuda"))
    T = lambda a: torch.tensor(a, device="cuda")
    xi = T(random_state_like(201, (B, RM)).astype(np.float32))
    z = T(controls(202, B, dz).astype(np.float32))
    y = T((0.1 * random_state_like(203, (B, RU))).astype(np.float32))
    jy = T((0.05 * random_state_like(204, (B, dz, RU))).astype(np.float32))
    idx = T(np.arange(B, dtype=np.int32))
    D.ouu_dino_train_step(xi, z, y, jy, idx, B, 1e-3)

    path = str(tmp_path / "net.ckpt")
    D.ouu_dino_save(path)
    D2 = capi.Dino(**kw)
    D2.ouu_dino_load(path)
    p1 = D.ouu_dino_get_params()
    assert np.array_equal(D2.ouu_dino_get_params(), p1)
    assert np.array_equal(D2.ouu_dino_get_output_scale(), D.ouu_dino_get_output_scale())
    phi2 = torch.empty(RU, n, n, dtype=torch.float64, device="cuda")
    ub2 = torch.empty(n, n, dtype=torch.float64, device="cuda")
    D2.ouu_dino_get_bases(phi2, ub2)
    assert np.array_equal(phi2.cpu().numpy(), phi) and np.array_equal(ub2.cpu().numpy(), ub)

    D.ouu_dino_train_step(xi, z, y, jy, idx, B, 1e-3)
    D2.ouu_dino_train_step(xi, z, y, jy, idx, B, 1e-3)
    a, b = D.ouu_dino_get_params(), D2.ouu_dino_get_params()
    assert np.abs(a - p1).max() > 1e-4
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-6)

    D3 = capi.Dino(**dict(kw, width=40))
    with pytest.raises(capi.OuuError, match="other sizes"):
        D3.ouu_dino_load(path)
    short = tmp_path / "short.ckpt"
    with open(path, "rb") as fh:
        short.write_bytes(fh.read()[:-4])
    with pytest.raises(capi.OuuError, match="truncated"):
        D2.ouu_dino_load(str(short))
    for H in (D, D2, D3):
        H.close()
