"""Thin ctypes binding of libouu.so (the C ABI declared in include/ouu.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their data pointers are passed
through); host results come back as numpy arrays.  If the library has not been
built, loading raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libouu.so")

OUU_OK = 0
OUU_ERR_INVALID_ARG = 1
OUU_ERR_CUDA = 2
OUU_ERR_OOM = 3
OUU_ERR_NOT_CONVERGED = 4
OUU_ERR_NONFINITE = 5
OUU_ERR_STATE = 6
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "NONFINITE", 6: "STATE"}
RISK_MEAN_VAR = 0
RISK_CVAR_SMOOTH = 1
BACKEND_PDE = 0
BACKEND_DINO = 1
BACKEND_AUTO = 2


class OuuError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("reaction_r", ctypes.c_double), ("gamma", ctypes.c_double),
                ("delta", ctypes.c_double), ("m_mean", ctypes.c_double), ("lattice_L", ctypes.c_int),
                ("bump_width", ctypes.c_double), ("newton_rtol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
                ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int), ("max_samples", ctypes.c_int)]


class RiskDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("kappa", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps", ctypes.c_double), ("t", ctypes.c_double), ("t_optimal", ctypes.c_int)]


class DinoDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("lattice_L", ctypes.c_int), ("r_m", ctypes.c_int), ("r_u", ctypes.c_int),
                ("width", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_eval", ctypes.c_int),
                ("gamma", ctypes.c_double), ("delta", ctypes.c_double), ("m_mean", ctypes.c_double),
                ("jac_weight", ctypes.c_double)]


class EvalStats(ctypes.Structure):
    _fields_ = [("newton_min", ctypes.c_int), ("newton_max", ctypes.c_int), ("newton_mean", ctypes.c_double),
                ("cg_total", ctypes.c_int), ("adjoint_solves", ctypes.c_int), ("n_not_converged", ctypes.c_int),
                ("ms_state", ctypes.c_float), ("ms_weights", ctypes.c_float), ("ms_adjoint", ctypes.c_float),
                ("ms_reduce", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_project", ctypes.c_float), ("ms_network", ctypes.c_float)]


class BatchItem(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_void_p), ("backend", ctypes.c_int), ("dino", ctypes.c_void_p),
                ("m_dev", ctypes.c_void_p), ("n_samples", ctypes.c_int), ("risks", ctypes.POINTER(RiskDesc)),
                ("n_risks", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/ouu.h
SIGNATURES = {
    "ouu_default_problem_desc": (None, [ctypes.POINTER(ProblemDesc)]),
    "ouu_create_problem": (_i, [ctypes.POINTER(ProblemDesc), _vp, ctypes.POINTER(_vp)]),
    "ouu_destroy_problem": (_i, [_vp]),
    "ouu_sample_fields": (_i, [_vp, _u64, _i64, _i, _vp]),
    "ouu_pde_solve_batch": (_i, [_vp, _vp, _i, _vp, _i64, _vp, _vp, _vp]),
    "ouu_adjoint_batch": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "ouu_risk_and_grad": (_i, [_vp, _i, _vp, _vp, _i, ctypes.POINTER(RiskDesc), _i, _dp, _dp, _dp, _dp, _dp,
                               ctypes.POINTER(EvalStats)]),
    "ouu_pde_solve_batch_noalloc": (_i, [ctypes.POINTER(ProblemDesc), _vp, _i, _vp, _i64, _vp, _vp, _vp, _vp]),
    "ouu_shard_qoi": (_i, [_vp, _i, _vp, _vp, _i, _dp, _vp]),
    "ouu_shard_risk_partial": (_i, [_vp, _vp, _vp, _i, _i64, ctypes.POINTER(RiskDesc), _i, _dp, _dp, _dp, _dp]),
    "ouu_last_backend": (_i, [_vp]),
    "ouu_dino_save": (_i, [_vp, ctypes.c_char_p]),
    "ouu_dino_load": (_i, [_vp, ctypes.c_char_p]),
    "ouu_dino_validate": (_i, [_vp, _vp, _vp, _i, ctypes.POINTER(RiskDesc), _i, _dp, _i, ctypes.c_double,
                               ctypes.c_double, _dp, _dp, ctypes.POINTER(ctypes.c_int)]),
    "ouu_default_dino_desc": (None, [ctypes.POINTER(DinoDesc)]),
    "ouu_dino_create": (_i, [ctypes.POINTER(DinoDesc), _vp, ctypes.POINTER(_vp)]),
    "ouu_dino_destroy": (_i, [_vp]),
    "ouu_dino_num_params": (ctypes.c_size_t, [_vp]),
    "ouu_dino_set_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "ouu_dino_get_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "ouu_dino_set_bases": (_i, [_vp, _vp, _vp]),
    "ouu_dino_build_bases": (_i, [_vp, _vp, _i, _dp]),
    "ouu_dino_get_bases": (_i, [_vp, _vp, _vp]),
    "ouu_dino_set_output_scale": (_i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "ouu_dino_get_output_scale": (_i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "ouu_dino_project_fields": (_i, [_vp, _vp, _i, _vp]),
    "ouu_dino_project_states": (_i, [_vp, _vp, _i, _vp]),
    "ouu_dino_jacobian_data": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "ouu_dino_set_jacobian_route": (_i, [_vp, _i]),
    "ouu_dino_train_step": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, ctypes.c_float, _dp]),
    "ouu_dino_loss_grad": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, ctypes.POINTER(ctypes.c_float), _dp]),
    "ouu_dino_eval": (_i, [_vp, _vp, _i, _dp, _vp, _vp, _vp, _vp, _vp]),
    "ouu_dino_decode": (_i, [_vp, _vp, _i, _vp, _vp]),
    "ouu_dino_set_graphs": (_i, [_vp, _i]),
    "ouu_dino_set_fused_network": (_i, [_vp, _i]),
    "ouu_kernel_gemm_bf16": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _i, ctypes.c_float, _vp, _vp, _i, _i, _vp, _i, _i,
                                  _vp, _i, _vp, _i, _vp, _i, _vp, _vp]),
    "ouu_kernel_kl_project": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _vp, _vp, _vp]),
    "ouu_kernel_risk_weights": (_i, [_vp, _i, ctypes.POINTER(RiskDesc), _i, _vp, _dp, _vp, _i, _i, _dp, _vp]),
    "ouu_kernel_gemm_qoi_bf16": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _vp, _vp, _vp, ctypes.c_double, _vp, _i, _vp, _i,
                                      _vp, _vp, _vp]),
    "ouu_batch_create": (_i, [ctypes.POINTER(BatchItem), _i, _i, ctypes.POINTER(_vp)]),
    "ouu_batch_destroy": (None, [_vp]),
    "ouu_batch_run": (_i, [_vp, ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                           ctypes.POINTER(_dp), _dp, _dp]),
    "ouu_kernel_gemm_tuned_shapes": (_i, []),
    "ouu_kernel_dino_network": (_i, [_vp, _vp, _i, _dp, _i, _vp, _vp, _vp]),
    "ouu_last_error": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
    "ouu_problem_slots": (_i, [_vp]),
}

_lib = None


def load():
    """Load libouu.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not found: build it with __graft_entry__.build() "
                          "or `python -m paper_2305_20053_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    load().ouu_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status):
    if status != OUU_OK:
        raise OuuError(status, last_error())


def dev_ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def need(t, count, name):
    """Raises when the buffer t (tensor or array; None passes) holds fewer than count elements, so
    that a short buffer is an error here instead of an out-of-bounds access in the library."""
    size = None if t is None else (t.numel() if hasattr(t, "numel") else np.asarray(t).size)
    if size is not None and size < count:
        raise ValueError(f"{name}: {size} elements, the call needs {count}")


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


def problem_desc(**kw) -> ProblemDesc:
    d = ProblemDesc()
    load().ouu_default_problem_desc(ctypes.byref(d))
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def risk_desc(kind, kappa=1.0, beta=0.95, eps=1e-4, t=0.0, t_optimal=1) -> RiskDesc:
    return RiskDesc(kind, kappa, beta, eps, t, t_optimal)


class Problem:
    """Owns an ouu_problem_t.  Methods are one-to-one with the C calls."""

    def __init__(self, stream=None, **desc):
        import torch
        self.desc = problem_desc(**desc)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(load().ouu_create_problem(ctypes.byref(self.desc), _stream_handle(self.stream), ctypes.byref(h)))
        self.handle = h
        self.n = self.desc.n
        self.d_z = self.desc.lattice_L ** 2

    def close(self):
        if getattr(self, "handle", None):
            load().ouu_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def slots(self) -> int:
        return load().ouu_problem_slots(self.handle)

    def ouu_last_backend(self) -> int:
        """BACKEND_PDE or BACKEND_DINO: what the last successful ouu_risk_and_grad ran (-1: none yet)."""
        return load().ouu_last_backend(self.handle)

    def ouu_sample_fields(self, seed, first_index, n_samples, m_dev):
        import torch
        need(m_dev, n_samples * self.n * self.n, "m_dev")
        check(load().ouu_sample_fields(self.handle, seed, first_index, n_samples, dev_ptr(m_dev, torch.float64)))

    def ouu_pde_solve_batch(self, m_dev, n_samples, z_dev, z_stride, u_dev, q_dev, status_dev):
        import torch
        nn = self.n * self.n
        for t, count, name in ((m_dev, n_samples * nn, "m_dev"), (u_dev, n_samples * nn, "u_dev"),
                               (z_dev, z_stride * (n_samples - 1) + self.d_z if n_samples > 0 else 0, "z_dev"),
                               (q_dev, n_samples, "q_dev"), (status_dev, n_samples, "status_dev")):
            need(t, count, name)
        check(load().ouu_pde_solve_batch(self.handle, dev_ptr(m_dev, torch.float64), n_samples,
                                         dev_ptr(z_dev, torch.float64), z_stride, dev_ptr(u_dev, torch.float64),
                                         dev_ptr(q_dev, torch.float64), dev_ptr(status_dev, torch.int32)))

    def ouu_adjoint_batch(self, m_dev, u_dev, n_samples, lambda_dev, gradq_dev):
        import torch
        nn = self.n * self.n
        for t, count, name in ((m_dev, n_samples * nn, "m_dev"), (u_dev, n_samples * nn, "u_dev"),
                               (lambda_dev, n_samples * nn, "lambda_dev"),
                               (gradq_dev, n_samples * self.d_z, "gradq_dev")):
            need(t, count, name)
        check(load().ouu_adjoint_batch(self.handle, dev_ptr(m_dev, torch.float64), dev_ptr(u_dev, torch.float64),
                                       n_samples, dev_ptr(lambda_dev, torch.float64),
                                       dev_ptr(gradq_dev, torch.float64)))

    def ouu_risk_and_grad(self, backend, dino, m_dev, n_samples, risks, z_host):
        """Returns (risk[n_risks], grad_z[n_risks, d_Z], grad_t[n_risks], t[n_risks], stats).
        The ctypes argument blocks are kept between calls with the same risk descriptors
        (marshalling only; the returned arrays are fresh copies)."""
        import torch
        need(m_dev, n_samples * self.n * self.n, "m_dev")
        key = tuple(bytes(r) for r in risks)
        c = getattr(self, "_rg_cache", None)
        if c is None or c["key"] != key:
            nr = len(risks)
            bufs = dict(z=np.zeros(self.d_z), risk=np.zeros(nr), grad=np.zeros((nr, self.d_z)), gt=np.zeros(nr),
                        t=np.zeros(nr))
            c = dict(key=key, nr=nr, arr=(RiskDesc * nr)(*risks), st=EvalStats(), **bufs,
                     ptr={k: v.ctypes.data_as(_dp) for k, v in bufs.items()})
            c["st_ref"] = ctypes.byref(c["st"])
            self._rg_cache = c
        c["z"][:] = z_host
        p = c["ptr"]
        check(load().ouu_risk_and_grad(self.handle, backend, dino.handle if dino is not None else None,
                                       dev_ptr(m_dev, torch.float64), n_samples, c["arr"], c["nr"], p["z"], p["risk"],
                                       p["grad"], p["gt"], p["t"], c["st_ref"]))
        return (c["risk"].copy(), c["grad"].copy(), c["gt"].copy(), c["t"].copy(),
                EvalStats.from_buffer_copy(c["st"]))


    def ouu_shard_qoi(self, backend, dino, m_dev, n_local, z_host, q_local_dev):
        """Phase 1 of a sample set spread over ranks: this rank's QoIs into q_local_dev [n_local]."""
        import torch
        need(m_dev, n_local * self.n * self.n, "m_dev")
        need(q_local_dev, n_local, "q_local_dev")
        z = np.ascontiguousarray(z_host, dtype=np.float64)
        need(z, self.d_z, "z_host")
        check(load().ouu_shard_qoi(self.handle, backend, dino.handle if dino is not None else None,
                                   dev_ptr(m_dev, torch.float64), n_local, z.ctypes.data_as(_dp),
                                   dev_ptr(q_local_dev, torch.float64)))

    def ouu_shard_risk_partial(self, dino, q_all_dev, n_total, first_local, risks):
        """Phase 2: (risk[n_risks], grad_part[n_risks, d_Z], grad_t[n_risks], t[n_risks]) from the
        gathered QoIs q_all_dev [n_total]; summing grad_part over ranks gives the gradient."""
        import torch
        need(q_all_dev, n_total, "q_all_dev")
        nr = len(risks)
        arr = (RiskDesc * nr)(*risks)
        risk, grad, gt, t = np.zeros(nr), np.zeros((nr, self.d_z)), np.zeros(nr), np.zeros(nr)
        check(load().ouu_shard_risk_partial(self.handle, dino.handle if dino is not None else None,
                                            dev_ptr(q_all_dev, torch.float64), n_total, first_local, arr, nr,
                                            risk.ctypes.data_as(_dp), grad.ctypes.data_as(_dp),
                                            gt.ctypes.data_as(_dp), t.ctypes.data_as(_dp)))
        return risk, grad, gt, t


def ouu_pde_solve_batch_noalloc(desc, m_dev, n_samples, z_dev, z_stride, u_dev, q_dev, status_dev, stream=None):
    """Allocation-free batched state solve (no problem handle; fixed device scratch)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    check(load().ouu_pde_solve_batch_noalloc(ctypes.byref(desc), dev_ptr(m_dev, torch.float64), n_samples,
                                             dev_ptr(z_dev, torch.float64), z_stride, dev_ptr(u_dev, torch.float64),
                                             dev_ptr(q_dev, torch.float64), dev_ptr(status_dev, torch.int32),
                                             _stream_handle(stream)))


def ouu_kernel_gemm_bf16(A, B, M, N, K, mode=0, alpha=1.0, bias=None, aux=None, aux_rdiv=1, out_f32=None,
                         accumulate=0, out_bf16=None, out_t_bf16=None, out2_bf16=None, err=None, stream=None):
    """D = A B^T on the tensor cores with a fused epilogue (kernel-level test entry)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    ld = lambda t: 0 if t is None else t.stride(0)
    check(load().ouu_kernel_gemm_bf16(dev_ptr(A, torch.bfloat16), A.stride(0), dev_ptr(B, torch.bfloat16),
                                      B.stride(0), M, N, K, mode, alpha, dev_ptr(bias, torch.float32),
                                      dev_ptr(aux, torch.float32), ld(aux), aux_rdiv, dev_ptr(out_f32, torch.float32),
                                      ld(out_f32), accumulate, dev_ptr(out_bf16, torch.bfloat16), ld(out_bf16),
                                      dev_ptr(out_t_bf16, torch.bfloat16), ld(out_t_bf16),
                                      dev_ptr(out2_bf16, torch.bfloat16), ld(out2_bf16), dev_ptr(err, torch.int32),
                                      _stream_handle(stream)))


def ouu_kernel_risk_weights(q, risks, w, gq=None, stream=None):
    """Per-sample risk weights and (rho, d rho/dt, t) per risk; with per-sample gradients gq
    (FP32 [N][d]) also the risk gradients (kernel-level test entry).  Returns out [n, 3] or
    (out, grad [n, d])."""
    import numpy as np
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    n = len(risks)
    arr = (RiskDesc * n)(*risks)
    out = np.zeros(3 * n)
    dz = gq.shape[1] if gq is not None else 0
    grad = np.zeros(n * max(dz, 1))
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(load().ouu_kernel_risk_weights(dev_ptr(q, torch.float64), q.numel(), arr, n, dev_ptr(w, torch.float64),
                                         P(out), dev_ptr(gq, torch.float32), dz, dz, P(grad) if gq is not None else None,
                                         _stream_handle(stream)))
    if gq is None:
        return out.reshape(n, 3)
    return out.reshape(n, 3), grad.reshape(n, dz)


def ouu_kernel_gemm_qoi_bf16(A, B, M, N, K, bias, col_scale, col_add, qconst, out_f32, out_bf16, out_q, err,
                             stream=None):
    """Output layer with the reduced-QoI epilogue (kernel-level test entry)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    check(load().ouu_kernel_gemm_qoi_bf16(dev_ptr(A, torch.bfloat16), A.stride(0), dev_ptr(B, torch.bfloat16),
                                          B.stride(0), M, N, K, dev_ptr(bias, torch.float32),
                                          dev_ptr(col_scale, torch.float32), dev_ptr(col_add, torch.float32), qconst,
                                          dev_ptr(out_f32, torch.float32), out_f32.stride(0),
                                          dev_ptr(out_bf16, torch.bfloat16), out_bf16.stride(0),
                                          dev_ptr(out_q, torch.float64), dev_ptr(err, torch.int32),
                                          _stream_handle(stream)))


def ouu_kernel_kl_project(m, N, nn, W, rm, bias, xi, err=None, stream=None):
    """Fused FP64-field KL projection xi = bf16(m) W^T + bias (kernel-level test entry)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    check(load().ouu_kernel_kl_project(dev_ptr(m, torch.float64), N, nn, dev_ptr(W, torch.bfloat16), W.stride(0), rm,
                                       dev_ptr(bias, torch.float32), dev_ptr(xi, torch.float32),
                                       dev_ptr(err, torch.int32), _stream_handle(stream)))


def dino_desc(**kw) -> DinoDesc:
    d = DinoDesc()
    load().ouu_default_dino_desc(ctypes.byref(d))
    for k, v in kw.items():
        setattr(d, k, v)
    return d


class Dino:
    """Owns an ouu_dino_t (the MR-DINO network).  Methods are one-to-one with the C calls."""

    def __init__(self, stream=None, **desc):
        import torch
        self.desc = dino_desc(**desc)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(load().ouu_dino_create(ctypes.byref(self.desc), _stream_handle(self.stream), ctypes.byref(h)))
        self.handle = h
        self.n_params = load().ouu_dino_num_params(h)
        self.d_z = self.desc.lattice_L ** 2

    def close(self):
        if getattr(self, "handle", None):
            load().ouu_dino_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ouu_dino_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(load().ouu_dino_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    def ouu_dino_get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        check(load().ouu_dino_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def ouu_dino_set_bases(self, phi_dev, ubar_dev):
        import torch
        check(load().ouu_dino_set_bases(self.handle, dev_ptr(phi_dev, torch.float64), dev_ptr(ubar_dev, torch.float64)))

    def ouu_dino_build_bases(self, u_dev, n_states):
        eig = np.zeros(n_states)
        import torch
        check(load().ouu_dino_build_bases(self.handle, dev_ptr(u_dev, torch.float64), n_states,
                                          eig.ctypes.data_as(_dp)))
        return eig

    def ouu_dino_set_output_scale(self, s):
        s = np.ascontiguousarray(s, dtype=np.float32)
        if s.size != self.desc.r_u:
            raise ValueError(f"output scale: {s.size} entries, r_u = {self.desc.r_u}")
        check(load().ouu_dino_set_output_scale(self.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def ouu_dino_get_output_scale(self):
        s = np.zeros(self.desc.r_u, dtype=np.float32)
        check(load().ouu_dino_get_output_scale(self.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return s

    def ouu_kernel_dino_network(self, xi, n_samples, z, mode, q=None, phi=None, gradq=None):
        """The evaluation network alone from device FP32 projection coordinates xi [N][r_M], in
        network mode `mode` (kernel-level test entry)."""
        import numpy as np
        import torch
        zz = np.ascontiguousarray(z, dtype=np.float64)
        if zz.size != self.d_z:
            raise ValueError(f"z: {zz.size} entries, d_Z = {self.d_z}")
        need(xi, n_samples * self.desc.r_m, "xi")
        need(q, n_samples, "q")
        need(phi, n_samples * self.desc.r_u, "phi")
        need(gradq, n_samples * self.d_z, "gradq")
        check(load().ouu_kernel_dino_network(self.handle, dev_ptr(xi, torch.float32), n_samples,
                                             zz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(mode),
                                             dev_ptr(q, torch.float64), dev_ptr(phi, torch.float32),
                                             dev_ptr(gradq, torch.float64)))

    def ouu_dino_validate(self, problem, m_dev, n_samples, risks, zs, risk_tol=0.01, grad_tol=0.05):
        """Held-out check against the plain path at the controls zs [n_z][d_Z]; returns
        (largest relative risk error, largest relative gradient error, passed).  While passed,
        BACKEND_AUTO evaluations of `problem` use this network."""
        import torch
        zz = np.ascontiguousarray(np.atleast_2d(zs), dtype=np.float64)
        if zz.ndim != 2 or zz.shape[1] != self.d_z:
            raise ValueError(f"zs: shape {zz.shape}, expected (n_z, {self.d_z})")
        need(m_dev, n_samples * self.desc.n * self.desc.n, "m_dev")
        arr = (RiskDesc * len(risks))(*risks)
        er, eg, ok = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        check(load().ouu_dino_validate(problem.handle, self.handle, dev_ptr(m_dev, torch.float64), n_samples, arr,
                                       len(risks), zz.ctypes.data_as(_dp), zz.shape[0], float(risk_tol),
                                       float(grad_tol), ctypes.byref(er), ctypes.byref(eg), ctypes.byref(ok)))
        return er.value, eg.value, bool(ok.value)

    def ouu_dino_save(self, path):
        """Checkpoint of the whole network state (parameters, Adam state, output scale, bases)."""
        check(load().ouu_dino_save(self.handle, os.fsencode(os.fspath(path))))

    def ouu_dino_load(self, path):
        """Restores a checkpoint written by ouu_dino_save for a network of these sizes and prior."""
        check(load().ouu_dino_load(self.handle, os.fsencode(os.fspath(path))))

    def ouu_dino_set_fused_network(self, mode):
        """0: per-layer GEMM kernels, 1: one kernel per 128-sample tile, 2: 4-CTA clusters."""
        check(load().ouu_dino_set_fused_network(self.handle, int(mode)))

    def ouu_dino_set_graphs(self, enable):
        check(load().ouu_dino_set_graphs(self.handle, int(enable)))

    def ouu_dino_get_bases(self, phi_dev, ubar_dev):
        import torch
        check(load().ouu_dino_get_bases(self.handle, dev_ptr(phi_dev, torch.float64), dev_ptr(ubar_dev, torch.float64)))

    def ouu_dino_project_fields(self, m_dev, n, xi_dev):
        import torch
        check(load().ouu_dino_project_fields(self.handle, dev_ptr(m_dev, torch.float64), n,
                                             dev_ptr(xi_dev, torch.float32)))

    def ouu_dino_project_states(self, u_dev, n, y_dev):
        import torch
        check(load().ouu_dino_project_states(self.handle, dev_ptr(u_dev, torch.float64), n,
                                             dev_ptr(y_dev, torch.float32)))

    def ouu_dino_set_jacobian_route(self, route):
        """0: the route with fewer solves (default), 1: forward, 2: adjoint."""
        check(load().ouu_dino_set_jacobian_route(self.handle, route))

    def ouu_dino_jacobian_data(self, problem, m_dev, u_dev, n, jy_dev):
        import torch
        check(load().ouu_dino_jacobian_data(problem.handle, self.handle, dev_ptr(m_dev, torch.float64),
                                            dev_ptr(u_dev, torch.float64), n, dev_ptr(jy_dev, torch.float32)))

    def ouu_dino_train_step(self, xi, z, y, jy, idx, batch, lr, want_loss=False):
        import torch
        loss = np.zeros(1)
        check(load().ouu_dino_train_step(self.handle, dev_ptr(xi, torch.float32), dev_ptr(z, torch.float32),
                                         dev_ptr(y, torch.float32), dev_ptr(jy, torch.float32),
                                         dev_ptr(idx, torch.int32), batch, lr,
                                         loss.ctypes.data_as(_dp) if want_loss else None))
        return float(loss[0]) if want_loss else None

    def ouu_dino_loss_grad(self, xi, z, y, jy, idx, batch):
        import torch
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1)
        check(load().ouu_dino_loss_grad(self.handle, dev_ptr(xi, torch.float32), dev_ptr(z, torch.float32),
                                        dev_ptr(y, torch.float32), dev_ptr(jy, torch.float32),
                                        dev_ptr(idx, torch.int32), batch,
                                        g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), loss.ctypes.data_as(_dp)))
        return float(loss[0]), g

    def ouu_dino_eval(self, m_dev, n, z_host, phi_dev=None, jphi_dev=None, q_dev=None, gradq_dev=None, u_dev=None):
        import torch
        z = np.ascontiguousarray(z_host, dtype=np.float64)
        if z.size != self.d_z:
            raise ValueError(f"z: {z.size} entries, d_Z = {self.d_z}")
        d, nn = self.desc, self.desc.n * self.desc.n
        for t, count, name in ((m_dev, n * nn, "m_dev"), (phi_dev, n * d.r_u, "phi_dev"),
                               (jphi_dev, n * self.d_z * d.r_u, "jphi_dev"), (q_dev, n, "q_dev"),
                               (gradq_dev, n * self.d_z, "gradq_dev"), (u_dev, n * nn, "u_dev")):
            need(t, count, name)
        check(load().ouu_dino_eval(self.handle, dev_ptr(m_dev, torch.float64), n, z.ctypes.data_as(_dp),
                                   dev_ptr(phi_dev, torch.float32), dev_ptr(jphi_dev, torch.float32),
                                   dev_ptr(q_dev, torch.float64), dev_ptr(gradq_dev, torch.float64),
                                   dev_ptr(u_dev, torch.float32)))

    def ouu_dino_decode(self, phi_dev, n, u_dev, q_dev=None):
        """u_w = Phi phi + ubar (FP32 [n][n][n]) and the decoded QoI (FP64 [n], optional)."""
        import torch
        nn = self.desc.n * self.desc.n
        for t, count, name in ((phi_dev, n * self.desc.r_u, "phi_dev"), (u_dev, n * nn, "u_dev"), (q_dev, n, "q_dev")):
            need(t, count, name)
        check(load().ouu_dino_decode(self.handle, dev_ptr(phi_dev, torch.float32), n, dev_ptr(u_dev, torch.float32),
                                     dev_ptr(q_dev, torch.float64)))


def flatten_params(Ws, bs):
    """Flat FP32 parameter vector [W0, b0, W1, b1, ...] (W row-major [out][in])."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])
                           for W, b in zip(Ws, bs)])


def unflatten_params(p, widths):
    """Inverse of flatten_params for layer widths [n_in, h1, ..., n_out]."""
    Ws, bs, o = [], [], 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        Ws.append(np.asarray(p[o:o + fi * fo], np.float64).reshape(fo, fi))
        o += fi * fo
        bs.append(np.asarray(p[o:o + fo], np.float64))
        o += fo
    return Ws, bs


class Batch:
    """Owns an ouu_batch_t: many problems evaluated together (one CUDA graph per batch).
    items: sequence of dicts with keys problem (Problem), backend (BACKEND_PDE, _DINO or _AUTO),
    dino (Dino or None), m (device FP64 fields), n (samples), risks (list of RiskDesc)."""

    def __init__(self, items, autotune=False):
        import torch
        self._keep = []
        arr = (BatchItem * len(items))()
        self.d_z, self.n_risks = [], []
        for k, it in enumerate(items):
            rk = (RiskDesc * len(it["risks"]))(*it["risks"])
            self._keep += [it["problem"], it.get("dino"), it["m"], rk]
            arr[k].problem = it["problem"].handle
            arr[k].backend = it["backend"]
            arr[k].dino = it["dino"].handle if it.get("dino") is not None else None
            need(it["m"], it["n"] * it["problem"].n * it["problem"].n, f"items[{k}]['m']")
            arr[k].m_dev = dev_ptr(it["m"], torch.float64)
            arr[k].n_samples = it["n"]
            arr[k].risks = rk
            arr[k].n_risks = len(it["risks"])
            self.d_z.append(it["problem"].d_z)
            self.n_risks.append(len(it["risks"]))
        h = ctypes.c_void_p()
        check(load().ouu_batch_create(arr, len(items), 1 if autotune else 0, ctypes.byref(h)))
        self.handle = h
        self.n_items = len(items)

    def close(self):
        if getattr(self, "handle", None):
            load().ouu_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, zs):
        """One evaluation of every item at its control zs[k].  Returns (results, item_ms,
        total_ms); results[k] = (risk[n_risks], grad_z[n_risks, d_Z], grad_t[n_risks], t[n_risks])."""
        K = self.n_items
        z = [np.ascontiguousarray(zs[k], dtype=np.float64) for k in range(K)]
        risk = [np.zeros(self.n_risks[k]) for k in range(K)]
        grad = [np.zeros((self.n_risks[k], self.d_z[k])) for k in range(K)]
        gt = [np.zeros(self.n_risks[k]) for k in range(K)]
        t = [np.zeros(self.n_risks[k]) for k in range(K)]
        ptrs = lambda arrs: (_dp * K)(*[a.ctypes.data_as(_dp) for a in arrs])
        ms = np.zeros(K)
        total = np.zeros(1)
        check(load().ouu_batch_run(self.handle, ptrs(z), ptrs(risk), ptrs(grad), ptrs(gt), ptrs(t),
                                   ms.ctypes.data_as(_dp), total.ctypes.data_as(_dp)))
        return [(risk[k], grad[k], gt[k], t[k]) for k in range(K)], ms, float(total[0])
