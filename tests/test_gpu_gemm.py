"""Numerics of the tcgen05/TMA BF16 GEMM against a plain fp32 PyTorch matmul of the
same BF16 operands (products are exact in FP32; only the summation order differs).

Reference in float64 of the same BF16 operands.  Tolerances, relative to the
largest entry of each row: FP32 outputs 1e-5 + 5e-7 sqrt(K) (FP32 summation of
K exact products); BF16 outputs one BF16 ulp (2^-8) plus that.
"""
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2305_20053_gb300 import build, capi
    build.build()
    capi.load()
    torch.backends.cuda.matmul.allow_tf32 = False


def _bf(shape, ld=None, seed=0, scale=1.0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    rows, k = shape
    ld = ld or (k + 7) // 8 * 8
    buf = torch.zeros(rows, ld, device="cuda", dtype=torch.bfloat16)
    buf[:, :k] = (scale * torch.randn(rows, k, device="cuda", generator=g)).to(torch.bfloat16)
    return buf


def _ref(A, B, K):
    return (A[:, :K].double() @ B[:, :K].double().T).float()


def _tol(K):
    return 1e-5 + 5e-7 * math.sqrt(K)


def _gelu_d1(x):
    return 0.5 * (1 + torch.erf(x / math.sqrt(2))) + x * torch.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def _close(x, ref, tol):
    scale = ref.abs().amax(dim=1, keepdim=True).clamp_min(1e-30)
    err = ((x - ref).abs() / scale).max().item()
    assert err <= tol, err


@pytest.mark.parametrize("M,N,K,lda", [(300, 400, 304, 304), (4096, 200, 16641, 16704), (1, 16, 8, 8),
                                       (513, 100, 200, 200), (400, 304, 25856, 25856)])
def test_linear_bias_transposed(M, N, K, lda):
    from paper_2305_20053_gb300 import capi
    A = _bf((M, K), lda, seed=1)
    B = _bf((N, K), None, seed=2)
    bias = torch.randn(N, device="cuda")
    out = torch.full((M, N), 7.0, device="cuda")
    ob = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    ot = torch.empty(N, M + 3, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, B, M, N, K, mode=0, alpha=0.5, bias=bias, out_f32=out, out_bf16=ob,
                              out_t_bf16=ot, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = 0.5 * _ref(A, B, K) + bias
    _close(out, ref, _tol(K))
    _close(ob.float(), ref, 2 ** -8 + _tol(K))
    _close(ot[:, :M].float().T, ref, 2 ** -8 + _tol(K))
    # accumulate into the existing output
    capi.ouu_kernel_gemm_bf16(A, B, M, N, K, mode=0, alpha=1.0, out_f32=out, accumulate=1, err=err)
    torch.cuda.synchronize()
    _close(out, ref + _ref(A, B, K), 2 * _tol(K))


def test_gelu_layer():
    from paper_2305_20053_gb300 import capi
    M, N, K = 256, 400, 400
    A = _bf((M, K), seed=3)
    B = _bf((N, K), seed=4, scale=1.0 / 20)
    bias = 0.1 * torch.randn(N, device="cuda")
    a = torch.empty(M, N, device="cuda")
    h = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    ht = torch.empty(N, M, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, B, M, N, K, mode=1, bias=bias, out_f32=a, out_bf16=h, out_t_bf16=ht, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = _ref(A, B, K) + bias
    _close(a, ref, _tol(K))
    g = torch.nn.functional.gelu(ref)
    assert (h.float() - g).abs().max().item() <= 2 ** -8 * g.abs().max().item() + 1e-4
    assert torch.equal(ht.T, h)


def test_tangent_scaling_epilogue():
    from paper_2305_20053_gb300 import capi
    B_, dz, N, K = 12, 100, 400, 400
    M = B_ * dz
    A = _bf((M, K), seed=5)
    W = _bf((N, K), seed=6, scale=1.0 / 20)
    aux = torch.randn(B_, N, device="cuda")
    hd = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    ad = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    out = torch.empty(M, N, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, W, M, N, K, mode=2, aux=aux, aux_rdiv=dz, out_f32=out, out_bf16=hd,
                              out2_bf16=ad, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    acc = _ref(A, W, K)
    scale = _gelu_d1(aux).repeat_interleave(dz, dim=0)
    _close(out, acc * scale, 2 * _tol(K))
    _close(ad.float(), acc, 2 ** -8 + _tol(K))


def test_gelu_with_derivative_epilogue():
    """Mode 3 (forward layer of the evaluation): BF16 gelu(a) and FP32 gelu'(a), a = acc + bias."""
    from paper_2305_20053_gb300 import capi
    M, N, K = 300, 400, 200
    A = _bf((M, K), seed=13)
    B = _bf((N, K), seed=14, scale=1.0 / 14)
    bias = 0.1 * torch.randn(N, device="cuda")
    d = torch.empty(M, N, device="cuda")
    h = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, B, M, N, K, mode=3, bias=bias, out_f32=d, out_bf16=h, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    a = _ref(A, B, K) + bias
    # gelu' has slope <= 0.6 in a: the FP32 summation error of a carries over at most that factor
    _close(d, _gelu_d1(a), _tol(K))
    g = torch.nn.functional.gelu(a)
    assert (h.float() - g).abs().max().item() <= 2 ** -8 * g.abs().max().item() + 1e-4


def test_gelu_normal_cdf_error_bound():
    """The epilogues' GELU uses the normal CDF of Abramowitz & Stegun 26.2.17 (absolute error
    < 7.5e-8) with one fast exponential shared by phi and Phi: gelu'(a) = Phi(a) + a phi(a) on a
    dense sweep of a over [-8, 8] (exact pre-activations: acc = i / 4096 from BF16-exact
    operands, plus a bias per column) within 5e-7 of the exact FP64 value, and within 3e-7
    where |a| <= 3 (where the network's pre-activations lie): the formula's 7.5e-8, the fast
    exponential's relative error on phi and the FP32 roundings of Phi and of the output."""
    from paper_2305_20053_gb300 import capi
    M, N, K = 128, 256, 64
    A = torch.zeros(M, K, device="cuda", dtype=torch.bfloat16)
    A[:, 0] = torch.arange(M, device="cuda", dtype=torch.float32) / 128.0
    B = torch.zeros(N, K, device="cuda", dtype=torch.bfloat16)
    B[:, 0] = 1.0 / 32.0
    bias = torch.linspace(-8.0, 8.0 - 16.0 / N, N, device="cuda")
    d = torch.empty(M, N, device="cuda")
    h = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, B, M, N, K, mode=3, bias=bias, out_f32=d, out_bf16=h, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    acc = (torch.arange(M, dtype=torch.float32) / 4096.0)[:, None]
    a32 = acc + bias.cpu()[None, :]           # the FP32 sum the epilogue forms
    a = a32.double()
    exact = 0.5 * (1 + torch.erf(a / math.sqrt(2))) + a * torch.exp(-0.5 * a * a) / math.sqrt(2 * math.pi)
    e = (d.cpu().double() - exact).abs()
    assert e.max().item() <= 5e-7, e.max().item()
    assert e[a.abs() <= 3].max().item() <= 3e-7, e[a.abs() <= 3].max().item()


def test_scale_epilogue():
    """Mode 4 (reverse layer of the evaluation): y = acc * aux, per-row factors repeated aux_rdiv times."""
    from paper_2305_20053_gb300 import capi
    B_, rd, N, K = 40, 3, 200, 400
    M = B_ * rd
    A = _bf((M, K), seed=15)
    W = _bf((N, K), seed=16, scale=1.0 / 20)
    aux = torch.randn(B_, N, device="cuda")
    out = torch.empty(M, N, device="cuda")
    hb = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_bf16(A, W, M, N, K, mode=4, aux=aux, aux_rdiv=rd, out_f32=out, out_bf16=hb, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = _ref(A, W, K) * aux.repeat_interleave(rd, dim=0)
    _close(out, ref, 2 * _tol(K))
    _close(hb.float(), ref, 2 ** -8 + 2 * _tol(K))


def test_reduced_qoi_epilogue():
    """Mode 5 (output layer of the evaluation, Sec. 3.3 reduced QoI): phi = (acc + b) s,
    Q = qconst + 1/2 sum (phi + c)^2 per row (FP32 row sums), BF16 seed (phi + c) s."""
    from paper_2305_20053_gb300 import capi
    M, N, K = 300, 200, 400
    A = _bf((M, K), seed=21)
    B = _bf((N, K), seed=22, scale=1.0 / 20)
    g = torch.Generator(device="cuda").manual_seed(23)
    bias = 0.1 * torch.randn(N, device="cuda", generator=g)
    s = 0.5 + torch.rand(N, device="cuda", generator=g)
    c = 0.2 * torch.randn(N, device="cuda", generator=g)
    phi = torch.empty(M, N, device="cuda")
    seed = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    q = torch.empty(M, device="cuda", dtype=torch.float64)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.ouu_kernel_gemm_qoi_bf16(A, B, M, N, K, bias, s, c, 0.75, phi, seed, q, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref_phi = ((A[:, :K].double() @ B[:, :K].double().T) + bias.double()) * s.double()
    v = ref_phi + c.double()
    ref_q = 0.75 + 0.5 * (v * v).sum(dim=1)
    _close(phi, ref_phi.float(), 2 * _tol(K))
    assert ((q - ref_q).abs() / ref_q.abs()).max().item() <= 1e-5
    ref_seed = (v * s.double()).float()
    _close(seed.float(), ref_seed, 2 ** -8 + 2 * _tol(K))
