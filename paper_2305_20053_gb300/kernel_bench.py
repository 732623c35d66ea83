"""Kernel micro-benchmarks through the library's kernel-level entries (CUDA events, warm-up
first), for timing single kernels and for profiler captures of one kernel on a small case.

  python -m paper_2305_20053_gb300.kernel_bench kl_project [--n 129] [--samples 1024] [--rm 200]
  python -m paper_2305_20053_gb300.kernel_bench gemm [--m 4096] [--gemm-n 400] [--k 400] [--mode 1]
  python -m paper_2305_20053_gb300.kernel_bench risk [--samples 4096]
  python -m paper_2305_20053_gb300.kernel_bench pde_state [--n 129] [--samples 152]
  python -m paper_2305_20053_gb300.kernel_bench network [--samples 4096] [--mode 2]
  python -m paper_2305_20053_gb300.kernel_bench decode [--n 129] [--samples 4096]

Inputs are seeded random device tensors of the shapes of the 129 x 129 workload; the printed
line gives the average time per launch and the achieved GB/s or TFLOP/s.
"""
from __future__ import annotations

import argparse
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_20053_gb300 import capi  # noqa: E402


def _time(fn, warmup, iters):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1000.0 / iters


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("kernel", choices=["kl_project", "gemm", "risk", "pde_state", "network", "decode"])
    ap.add_argument("--n", type=int, default=129)
    ap.add_argument("--samples", type=int, default=1024)
    ap.add_argument("--rm", type=int, default=200)
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--gemm-n", type=int, default=400)
    ap.add_argument("--k", type=int, default=400)
    ap.add_argument("--mode", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=20)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    capi.load()
    g = torch.Generator(device="cuda").manual_seed(0)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    if a.kernel == "kl_project":
        N, nn, rm = a.samples, a.n * a.n, a.rm
        ldw = (nn + 63) // 64 * 64
        m = torch.randn(N, nn, device="cuda", dtype=torch.float64, generator=g)
        W = (torch.randn(rm, ldw, device="cuda", generator=g) / a.n).to(torch.bfloat16)
        b = torch.zeros(rm, device="cuda")
        xi = torch.empty(N, rm, device="cuda")
        us = _time(lambda: capi.ouu_kernel_kl_project(m, N, nn, W, rm, b, xi, err), a.warmup, a.iters)
        gbs = (N * nn * 8 + rm * ldw * 2 + N * rm * 4) / us / 1e3
        print(f"kl_project N={N} n^2={nn} r_m={rm}: {us:.1f} us/launch, {gbs:.0f} GB/s algorithmic, err {err.item()}")
    elif a.kernel == "gemm":
        M, N, K = a.m, a.gemm_n, a.k
        ld = (K + 7) // 8 * 8
        A = torch.randn(M, ld, device="cuda", generator=g).to(torch.bfloat16)
        B = (torch.randn(N, ld, device="cuda", generator=g) / math.sqrt(K)).to(torch.bfloat16)
        bias = torch.zeros(N, device="cuda")
        out = torch.empty(M, N, device="cuda")
        ob = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
        aux = torch.randn(M, N, device="cuda", generator=g)
        kw = dict(mode=a.mode, err=err)
        if a.mode in (2, 4):
            kw.update(aux=aux, out_bf16=ob)
        else:
            kw.update(bias=bias, out_f32=out, out_bf16=ob if a.mode in (1, 3) else None)
        us = _time(lambda: capi.ouu_kernel_gemm_bf16(A, B, M, N, K, **kw), a.warmup, a.iters)
        print(f"gemm M={M} N={N} K={K} mode={a.mode}: {us:.1f} us/launch, {2 * M * N * K / us / 1e6:.1f} TFLOP/s, "
              f"err {err.item()}")
    elif a.kernel == "pde_state":
        # the persistent state-solve kernel (Newton, MG-PCG) over N seeded fields at one control
        N, L = a.samples, 10
        P = capi.Problem(n=a.n, lattice_L=L, max_samples=N)
        m = torch.empty(N, a.n, a.n, dtype=torch.float64, device="cuda")
        P.ouu_sample_fields(1, 0, N, m)
        z = torch.rand(L * L, device="cuda", dtype=torch.float64, generator=g) * 2 - 1
        q = torch.empty(N, device="cuda", dtype=torch.float64)
        st = torch.empty(N, device="cuda", dtype=torch.int32)
        us = _time(lambda: P.ouu_pde_solve_batch(m, N, z, 0, None, q, st), a.warmup, a.iters)
        print(f"pde_state n={a.n} N={N}: {us:.1f} us per call ({us / N:.1f} us per sample)")
    elif a.kernel in ("network", "decode"):
        import numpy as np
        from synthetic_inputs import glorot_uniform_mlp, random_state_like
        n, L, N, R, W = a.n, 10, a.samples, 200, 400
        dz, h = L * L, 1.0 / (a.n - 1)
        D = capi.Dino(n=n, lattice_L=L, r_m=R, r_u=R, width=W, max_batch=256, max_eval=N)
        Ws, bs = glorot_uniform_mlp([R + dz, W, W, W, R], seed=91)
        D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
        Q, _ = np.linalg.qr(random_state_like(97, ((n - 2) ** 2, R)))
        phi = np.zeros((R, n, n))
        phi[:, 1:-1, 1:-1] = (Q / h).T.reshape(R, n - 2, n - 2)
        D.ouu_dino_set_bases(torch.tensor(phi, device="cuda"), torch.zeros(n, n, dtype=torch.float64, device="cuda"))
        if a.kernel == "network":
            xi = torch.randn(N, R, device="cuda", generator=g)
            z = np.zeros(dz)
            qo = torch.empty(N, device="cuda", dtype=torch.float64)
            gq = torch.empty(N, dz, device="cuda", dtype=torch.float64)
            us = _time(lambda: D.ouu_kernel_dino_network(xi, N, z, a.mode, qo, None, gq), a.warmup, a.iters)
            fl = 2 * N * ((R + dz) * W + 2 * W * W + W * R) + 2 * N * (R * W + 2 * W * W + W * dz)
            print(f"network mode {a.mode} N={N}: {us:.1f} us per call (with its entry's copies and "
                  f"synchronisation), {fl / us / 1e6:.1f} TFLOP/s")
        else:
            coef = torch.randn(N, R, device="cuda", generator=g)
            u = torch.empty(N, n, n, device="cuda")
            qd = torch.empty(N, device="cuda", dtype=torch.float64)
            us = _time(lambda: D.ouu_dino_decode(coef, N, u, qd), a.warmup, a.iters)
            by = N * n * n * 4 + N * 3 * R * 2 + n * n * 3 * R * 2
            print(f"decode n={n} N={N}: {us:.1f} us per call (with its operand build and synchronisation), "
                  f"{by / us / 1e3:.0f} GB/s algorithmic")
        D.close()
    else:
        N = a.samples
        q = 5.0 + torch.randn(N, device="cuda", dtype=torch.float64, generator=g)
        risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1),
                 capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
        w = torch.empty(len(risks), N, device="cuda", dtype=torch.float64)
        us = _time(lambda: capi.ouu_kernel_risk_weights(q, risks, w), a.warmup, a.iters)
        print(f"risk weights N={N}: {us:.1f} us per call (includes the entry's own allocation and synchronisation)")


if __name__ == "__main__":
    main()
