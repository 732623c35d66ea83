"""Numerics of the fused FP64-field KL projection (Sec. 3.3 input reduction) against
float64 products of the same BF16-rounded operands (the oracle's BF16 rounding:
FP64 -> FP32 -> BF16, both to nearest even).  Products of BF16 values are exact in
FP32, so only the FP32 summation order differs: tolerance, relative to the largest
entry of each row, 1e-5 + 5e-7 sqrt(n^2).

Cases: n^2 odd (sample-pair tensor map) and even (row tensor map); N even, odd (a
last unpaired sample read with plain loads), one sample (plain loads only), a base
8 bytes off a 16-byte boundary (plain loads), a ragged last 128-sample tile, a ragged
last 64-wide K block, r_m not a multiple of 16, r_m not a multiple of 4 (every partial sum by
scalar atomics, the bias added once per row whichever visit of a tile a CTA ends on), an
output 4 bytes off a 16-byte boundary, and the 129 x 129 width.
"""
import math

import numpy as np
import pytest

from oracle.dino import round_bf16

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()


@pytest.mark.parametrize("N,nn,rm", [(40, 289, 16), (131, 289, 200), (1, 289, 16), (3, 300, 24), (129, 1024, 52),
                                     (300, 289, 30), (257, 16641, 200)])
def test_kl_project_parity(N, nn, rm):
    from paper_2305_20053_gb300 import capi
    rng = np.random.default_rng(1000 + N + nn + rm)
    m = rng.standard_normal((N, nn)) * 1.3 + 0.2
    ldw = (nn + 63) // 64 * 64
    W = np.zeros((rm, ldw))
    W[:, :nn] = round_bf16(rng.standard_normal((rm, nn)) / math.sqrt(nn))
    bias = rng.standard_normal(rm).astype(np.float32)
    m_d = torch.tensor(m, device="cuda")
    W_d = torch.tensor(W, device="cuda").to(torch.bfloat16)
    b_d = torch.tensor(bias, device="cuda")
    xi = torch.full((N, rm), float("nan"), device="cuda", dtype=torch.float32)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_kl_project(m_d, N, nn, W_d, rm, b_d, xi, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = round_bf16(m) @ W[:, :nn].T + bias.astype(np.float64)
    got = xi.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= (1e-5 + 5e-7 * math.sqrt(nn)) * scale)


def test_kl_project_offset_base():
    """Fields starting 8 bytes off a 16-byte boundary (a slice at an odd sample) go by plain loads."""
    from paper_2305_20053_gb300 import capi
    N, nn, rm = 5, 289, 16
    rng = np.random.default_rng(77)
    full = torch.tensor(rng.standard_normal((N + 1, nn)), device="cuda")
    m_d = full[1:]                       # starts at 289 * 8 bytes: 8 mod 16
    assert m_d.data_ptr() % 16 == 8
    W = np.zeros((rm, 320))
    W[:, :nn] = round_bf16(rng.standard_normal((rm, nn)) / 17.0)
    W_d = torch.tensor(W, device="cuda").to(torch.bfloat16)
    b_d = torch.zeros(rm, device="cuda")
    xi = torch.empty(N, rm, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_kl_project(m_d, N, nn, W_d, rm, b_d, xi, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = round_bf16(m_d.cpu().numpy()) @ W[:, :nn].T
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(xi.cpu().numpy() - ref) <= (1e-5 + 5e-7 * math.sqrt(nn)) * scale)


def test_kl_project_unaligned_output():
    """xi starting 4 bytes past a 16-byte boundary: no vector atomics, no bulk reductions."""
    from paper_2305_20053_gb300 import capi
    N, nn, rm = 300, 289, 16
    rng = np.random.default_rng(78)
    m = rng.standard_normal((N, nn))
    W = np.zeros((rm, 320))
    W[:, :nn] = round_bf16(rng.standard_normal((rm, nn)) / 17.0)
    bias = rng.standard_normal(rm).astype(np.float32)
    m_d = torch.tensor(m, device="cuda")
    W_d = torch.tensor(W, device="cuda").to(torch.bfloat16)
    b_d = torch.tensor(bias, device="cuda")
    buf = torch.full((N * rm + 4,), float("nan"), device="cuda", dtype=torch.float32)
    xi = buf[1:1 + N * rm].view(N, rm)
    assert xi.data_ptr() % 16 == 4
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_kl_project(m_d, N, nn, W_d, rm, b_d, xi, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert torch.isnan(buf[0]).item() and torch.isnan(buf[1 + N * rm:]).all().item()
    ref = round_bf16(m) @ W[:, :nn].T + bias.astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(xi.cpu().numpy().astype(np.float64) - ref) <= (1e-5 + 5e-7 * math.sqrt(nn)) * scale)


def test_kl_project_several_launches_and_repeat():
    """More than 512 tiles (65,536 samples) run as several launches, each over its own slice
    with the tile counters left zero for the next: 65,536 + 301 samples (the second launch
    ragged, N odd: its last sample by plain loads), checked on rows around the boundary and
    spread over both launches; a second call on the same inputs gives the same rows (the
    counters were reset)."""
    from paper_2305_20053_gb300 import capi
    N, nn, rm = 65536 + 301, 289, 24
    rng = np.random.default_rng(4242)
    m_d = torch.randn(N, nn, device="cuda", dtype=torch.float64, generator=torch.Generator(device="cuda").manual_seed(5))
    W = np.zeros((rm, 320))
    W[:, :nn] = round_bf16(rng.standard_normal((rm, nn)) / 17.0)
    W_d = torch.tensor(W, device="cuda").to(torch.bfloat16)
    bias = rng.standard_normal(rm).astype(np.float32)
    b_d = torch.tensor(bias, device="cuda")
    rows = np.unique(np.concatenate([np.arange(65530, 65542), rng.integers(0, N, 40), [0, N - 2, N - 1]]))
    out = []
    for _ in range(2):
        xi = torch.full((N, rm), float("nan"), device="cuda", dtype=torch.float32)
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        capi.ouu_kernel_kl_project(m_d, N, nn, W_d, rm, b_d, xi, err)
        torch.cuda.synchronize()
        assert err.item() == 0
        assert not torch.isnan(xi).any().item()
        out.append(xi[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.float64))
    ref = round_bf16(m_d[torch.tensor(rows, device="cuda")].cpu().numpy()) @ W[:, :nn].T + bias.astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    for got in out:
        assert np.all(np.abs(got - ref) <= (1e-5 + 5e-7 * math.sqrt(nn)) * scale)
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=(1e-5 + 5e-7 * math.sqrt(nn)) * scale.max())
