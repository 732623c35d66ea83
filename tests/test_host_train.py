"""Host logic of the surrogate construction loop, CPU only: the learning-rate schedule is
the oracle's Sec. 4.2 schedule (lr0, then a quarter of it from half of the epochs on), and
its optional geometric tail runs from lr1 at half of the epochs to lr_final at the last one;
the flat parameter vector has the documented layout."""
import numpy as np
import pytest

from oracle import dino
from paper_2305_20053_gb300 import train


@pytest.mark.parametrize("epochs", [1, 2, 7, 200, 600])
def test_schedule_is_the_papers(epochs):
    for ep in range(epochs):
        assert train.lr_at(ep, epochs) == dino.lr_schedule(ep, epochs)


def test_geometric_tail():
    epochs, lr1, lrf = 600, 2.5e-4, 1e-5
    r = np.array([train.lr_at(ep, epochs, lr1=lr1, lr_final=lrf) for ep in range(epochs)])
    half = epochs // 2
    assert np.all(r[:half] == 1e-3)
    assert r[half] == pytest.approx(lr1, rel=1e-12) and r[-1] == pytest.approx(lrf, rel=1e-12)
    ratios = r[half + 1:] / r[half:-1]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-10)
    assert ratios[0] < 1.0


def test_parameter_vector_layout():
    """The flat FP32 parameter vector is [W0, b0, W1, b1, ...] with W_l row-major [out][in]
    (the layout ouu_dino_set_params documents); unflatten_params inverts flatten_params."""
    from paper_2305_20053_gb300 import capi
    from synthetic_inputs import glorot_uniform_mlp
    widths = [7, 5, 6, 3]
    Ws, bs = glorot_uniform_mlp(widths, seed=9)
    bs = [np.arange(len(b), dtype=np.float64) + 0.5 for b in bs]
    flat = capi.flatten_params(Ws, bs)
    assert flat.dtype == np.float32 and flat.size == sum(i * o + o for i, o in zip(widths[:-1], widths[1:]))
    assert flat[1] == np.float32(Ws[0][0, 1]) and flat[7] == np.float32(Ws[0][1, 0])   # row-major
    assert flat[35] == np.float32(bs[0][0])                                              # b0 after W0 (5 x 7)
    Ws2, bs2 = capi.unflatten_params(flat, widths)
    for a, b in zip(Ws + bs, Ws2 + bs2):
        np.testing.assert_array_equal(np.float32(a), b)
