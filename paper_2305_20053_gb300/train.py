"""MR-DINO construction driver (Sec. 3.4, Sec. 4.2): training data from the plain
batched solver, POD basis, and training by the library's own kernels.

Host-side orchestration only (epoch loop, learning-rate schedule, minibatch
index arrays); every computation is a call into libouu.so.

  python -m paper_2305_20053_gb300.train [--n 129] [--train 1024] [--epochs 200] [--save net.npz]

A trained surrogate is kept with save_surrogate / load_surrogate (an .npz archive of the
parameters, output scale and POD basis, checked against the handle's sizes and prior).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from dataclasses import dataclass

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_20053_gb300 import capi  # noqa: E402
from synthetic_inputs import (SEED_EVAL_Z, SEED_HELDOUT, SEED_NET, SEED_SAA, SEED_TRAIN_FIELDS,  # noqa: E402
                              SEED_TRAIN_Z, controls, epoch_orders, glorot_uniform_mlp)


@dataclass
class TrainData:
    xi: object       # [N][r_m] FP32 device
    z: object        # [N][d_Z] FP32 device
    y: object        # [N][r_u] FP32 device
    jy: object       # [N][d_Z][r_u] FP32 device
    eig: np.ndarray  # POD eigenvalues
    times: dict


def make_problem(n, L, max_samples):
    return capi.Problem(n=n, lattice_L=L, max_samples=max_samples)


def make_dino(n, L, r=200, width=400, max_batch=256, max_eval=4096, jac_weight=1.0):
    return capi.Dino(n=n, lattice_L=L, r_m=r, r_u=r, width=width, max_batch=max_batch, max_eval=max_eval,
                     jac_weight=jac_weight)


def init_params(D, seed=SEED_NET):
    d = D.desc
    widths = [d.r_m + d.lattice_L ** 2, d.width, d.width, d.width, d.r_u]
    Ws, bs = glorot_uniform_mlp(widths, seed=seed)
    D.ouu_dino_set_params(capi.flatten_params(Ws, bs))
    return widths


def generate_training_data(P, D, n_train, seed_fields=SEED_TRAIN_FIELDS, seed_z=SEED_TRAIN_Z, bases=True,
                           pod_states=1024):
    """States for per-sample controls z_i ~ U(-1, 1)^d_Z, the POD basis from the first
    min(n_train, pod_states) of them (unless bases=False), the network inputs, the reduced
    state targets and the reduced control Jacobians."""
    import torch
    n, dz = P.n, P.d_z
    t = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = torch.empty(n_train, n, n, dtype=torch.float64, device="cuda")
    for f in range(0, n_train, 65535):   # the sampling call takes up to 65535 fields
        P.ouu_sample_fields(seed_fields, f, min(65535, n_train - f), m[f:])
    z = torch.tensor(controls(seed_z, n_train, dz), device="cuda")
    u = torch.empty(n_train, n, n, dtype=torch.float64, device="cuda")
    q = torch.empty(n_train, dtype=torch.float64, device="cuda")
    st = torch.empty(n_train, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, n_train, z, dz, u, q, st)
    torch.cuda.synchronize()
    t["states_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    eig = D.ouu_dino_build_bases(u, min(n_train, pod_states)) if bases else None
    torch.cuda.synchronize()
    t["pod_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    r_m, r_u = D.desc.r_m, D.desc.r_u
    xi = torch.empty(n_train, r_m, dtype=torch.float32, device="cuda")
    y = torch.empty(n_train, r_u, dtype=torch.float32, device="cuda")
    jy = torch.empty(n_train, dz, r_u, dtype=torch.float32, device="cuda")
    D.ouu_dino_project_fields(m, n_train, xi)
    D.ouu_dino_project_states(u, n_train, y)
    D.ouu_dino_jacobian_data(P, m, u, n_train, jy)
    torch.cuda.synchronize()
    t["jacobian_s"] = time.perf_counter() - t0
    return TrainData(xi, z.float(), y, jy, eig, t)


def lr_at(ep, epochs, lr0=1e-3, lr1=2.5e-4, lr_final=None):
    """lr0 for the first half of the epochs, then lr1 (Sec. 4.2); with lr_final the second
    half decays geometrically from lr1 to lr_final instead of staying at lr1."""
    half = epochs // 2
    if ep < half:
        return lr0
    if lr_final is None or epochs - half <= 1:
        return lr1
    return lr1 * (lr_final / lr1) ** ((ep - half) / (epochs - half - 1))


def train(D, data, epochs=200, batch=256, lr0=1e-3, lr1=2.5e-4, seed=SEED_NET, log_every=0, lr_final=None):
    """Adam over `epochs` passes of seeded shuffles with the rate of lr_at.
    Returns (seconds, per-epoch losses sampled)."""
    import torch
    n_train = data.xi.shape[0]
    steps = n_train // batch
    orders = torch.tensor(epoch_orders(n_train, epochs, seed=seed + 1000).astype(np.int32), device="cuda")
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        lr = lr_at(ep, epochs, lr0, lr1, lr_final)
        for s in range(steps):
            idx = orders[ep, s * batch:(s + 1) * batch]
            want = log_every and (ep % log_every == 0 or ep == epochs - 1) and s == steps - 1
            loss = D.ouu_dino_train_step(data.xi, data.z, data.y, data.jy, idx, batch, lr, want_loss=bool(want))
            if want:
                losses.append((ep, loss))
    torch.cuda.synchronize()
    return time.perf_counter() - t0, losses


def heldout_errors(P, D, n_hold=256, seed=SEED_HELDOUT, seed_z=SEED_EVAL_Z + 100):
    """Relative state and control-Jacobian errors of the surrogate on held-out pairs (m, z),
    in the reduced coordinates (the M-orthogonal projection of the truth): Sec. 4.2's test errors."""
    import torch
    n, dz = P.n, P.d_z
    m = torch.empty(n_hold, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(seed, 0, n_hold, m)
    zs = controls(seed_z, n_hold, dz)
    u = torch.empty(n_hold, n, n, dtype=torch.float64, device="cuda")
    q = torch.empty(n_hold, dtype=torch.float64, device="cuda")
    st = torch.empty(n_hold, dtype=torch.int32, device="cuda")
    P.ouu_pde_solve_batch(m, n_hold, torch.tensor(zs, device="cuda"), dz, u, q, st)
    r_u = D.desc.r_u
    y = torch.empty(n_hold, r_u, dtype=torch.float32, device="cuda")
    jy = torch.empty(n_hold, dz, r_u, dtype=torch.float32, device="cuda")
    D.ouu_dino_project_states(u, n_hold, y)
    D.ouu_dino_jacobian_data(P, m, u, n_hold, jy)
    y, jy = y.cpu().numpy(), jy.cpu().numpy()
    es, ej = [], []
    phi = torch.empty(1, r_u, dtype=torch.float32, device="cuda")
    jphi = torch.empty(1, dz, r_u, dtype=torch.float32, device="cuda")
    for i in range(n_hold):
        D.ouu_dino_eval(m[i:i + 1], 1, zs[i], phi, jphi, None, None)
        p, J = phi.cpu().numpy()[0], jphi.cpu().numpy()[0]
        es.append(np.linalg.norm(p - y[i]) / np.linalg.norm(y[i]))
        ej.append(np.linalg.norm(J - jy[i]) / np.linalg.norm(jy[i]))
    return float(np.mean(es)), float(np.mean(ej))


def risk_errors(P, D, n_samples, zs, risks):
    """Relative risk and gradient errors of the MR-DINO SAA against the plain PDE SAA
    (same fields, same z), maximum over the controls zs."""
    import torch
    n = P.n
    m = torch.empty(n_samples, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(SEED_SAA, 0, n_samples, m)
    worst_r = np.zeros(len(risks))
    worst_g = np.zeros(len(risks))
    rows = []
    for z in zs:
        v0, g0, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m, n_samples, risks, z)
        v1, g1, _, _, _ = P.ouu_risk_and_grad(capi.BACKEND_DINO, D, m, n_samples, risks, z)
        er = np.abs(v1 - v0) / np.abs(v0)
        eg = np.linalg.norm(g1 - g0, axis=1) / np.linalg.norm(g0, axis=1)
        worst_r = np.maximum(worst_r, er)
        worst_g = np.maximum(worst_g, eg)
        rows.append({"risk_pde": v0.tolist(), "risk_dino": v1.tolist(), "rel_risk": er.tolist(),
                     "rel_grad": eg.tolist()})
    return worst_r, worst_g, rows


def validate_surrogate(P, D, n_hold=256, n_controls=3, risk_tol=0.01, grad_tol=0.05, seed=SEED_HELDOUT,
                       seed_z=SEED_EVAL_Z + 200):
    """Held-out check of the trained network with the plain path as the reference: n_hold fields
    not used for training, n_controls controls, both risks of the bench.  While it passes,
    BACKEND_AUTO evaluations of P use the network; otherwise they fall back to the plain path.
    Returns (largest relative risk error, largest relative gradient error, passed)."""
    import torch
    n = P.n
    m = torch.empty(n_hold, n, n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(seed, 0, n_hold, m)
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
    return D.ouu_dino_validate(P, m, n_hold, risks, controls(seed_z, n_controls, P.d_z), risk_tol, grad_tol)


# ----------------------------------------------------------------------------- persistence
# What defines a surrogate besides its arrays: the sizes and the prior (the KL projection rows
# follow from n, r_m and the prior, and are rebuilt when a handle is created).
SURROGATE_KEYS = ("n", "lattice_L", "r_m", "r_u", "width", "gamma", "delta", "m_mean")


def _surrogate_meta(desc):
    return np.array([float(getattr(desc, k)) for k in SURROGATE_KEYS])


def write_surrogate(path, desc, params, out_scale, phi, ubar):
    """Stores a trained surrogate as an .npz archive at `path` (written as given, no suffix
    added): the sizes and prior of `desc`, the flat FP32 parameter vector, the FP32 output
    scale [r_u] and the FP64 POD basis [r_u][n][n] with its mean state [n][n]."""
    n, r_u = int(desc.n), int(desc.r_u)
    params = np.ascontiguousarray(params, dtype=np.float32).ravel()
    out_scale = np.ascontiguousarray(out_scale, dtype=np.float32)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ubar = np.ascontiguousarray(ubar, dtype=np.float64)
    if out_scale.shape != (r_u,) or phi.shape != (r_u, n, n) or ubar.shape != (n, n):
        raise ValueError("surrogate arrays do not match the descriptor's n and r_u")
    with open(path, "wb") as fh:
        np.savez(fh, meta=_surrogate_meta(desc), params=params, out_scale=out_scale, phi=phi, ubar=ubar)


def read_surrogate(path, desc):
    """The arrays of write_surrogate, after checking that the archive holds a surrogate of the
    sizes and prior of `desc` (ValueError otherwise)."""
    with np.load(path) as f:
        meta, want = f["meta"], _surrogate_meta(desc)
        if meta.shape != want.shape or not np.array_equal(meta, want):
            bad = [k for k, a, b in zip(SURROGATE_KEYS, meta, want) if a != b] if meta.shape == want.shape else []
            raise ValueError(f"surrogate archive {path} was written for other sizes or prior {bad}")
        return {k: f[k] for k in ("params", "out_scale", "phi", "ubar")}


def save_surrogate(D, path):
    """Writes the trained state of the handle D (parameters, output scale, POD basis)."""
    import torch
    d = D.desc
    phi = torch.empty(d.r_u, d.n, d.n, dtype=torch.float64, device="cuda")
    ubar = torch.empty(d.n, d.n, dtype=torch.float64, device="cuda")
    D.ouu_dino_get_bases(phi, ubar)   # synchronises
    write_surrogate(path, d, D.ouu_dino_get_params(), D.ouu_dino_get_output_scale(), phi.cpu().numpy(),
                    ubar.cpu().numpy())


def load_surrogate(D, path):
    """Installs a surrogate written by save_surrogate into the handle D, created with the same
    sizes and prior (the Adam state starts afresh)."""
    import torch
    a = read_surrogate(path, D.desc)
    if a["params"].size != D.n_params:
        raise ValueError(f"surrogate archive {path}: {a['params'].size} parameters, the handle has {D.n_params}")
    D.ouu_dino_set_params(a["params"])
    phi = torch.tensor(a["phi"], device="cuda")
    ubar = torch.tensor(a["ubar"], device="cuda")
    D.ouu_dino_set_bases(phi, ubar)
    D.ouu_dino_set_output_scale(a["out_scale"])
    torch.cuda.synchronize()   # the basis copies have read phi and ubar before they are freed


def build_surrogate(n=129, L=10, n_train=1024, epochs=200, batch=256, jac_weight=1.0, max_eval=4096, log_every=0):
    """Problem + trained network; returns (P, D, report)."""
    P = make_problem(n, L, max(n_train, max_eval, 256))
    D = make_dino(n, L, max_eval=max_eval, jac_weight=jac_weight, max_batch=batch)
    init_params(D)
    data = generate_training_data(P, D, n_train)
    secs, losses = train(D, data, epochs=epochs, batch=batch, log_every=log_every)
    rep = dict(data.times)
    rep["train_s"] = secs
    rep["losses"] = losses
    rep["pod_energy_captured"] = float(np.sum(data.eig[:D.desc.r_u]) / np.sum(data.eig))
    return P, D, rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=129)
    ap.add_argument("--L", type=int, default=10)
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--jac-weight", type=float, default=1.0)
    ap.add_argument("--out", default="")
    ap.add_argument("--save", default="", help="write the trained surrogate to this .npz file")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    P, D, rep = build_surrogate(args.n, args.L, args.train, args.epochs, jac_weight=args.jac_weight,
                                max_eval=args.samples, log_every=20)
    if args.save:
        save_surrogate(D, args.save)
    es, ej = heldout_errors(P, D)
    rep["heldout_state_rel"] = es
    rep["heldout_jacobian_rel"] = ej
    vr, vg, ok = validate_surrogate(P, D)
    rep["fallback_check"] = {"risk_rel": vr, "grad_rel": vg, "network_used_by_auto": ok}
    risks = [capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=0.95, eps=1e-4, t_optimal=1),
             capi.risk_desc(capi.RISK_MEAN_VAR, kappa=1.0)]
    zs = controls(SEED_EVAL_Z, 5, args.L * args.L)
    wr, wg, rows = risk_errors(P, D, args.samples, zs, risks)
    rep["risk_rel_max"] = wr.tolist()
    rep["grad_rel_max"] = wg.tolist()
    rep["per_z"] = rows
    print(json.dumps(rep))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rep, fh, indent=1)


if __name__ == "__main__":
    main()
