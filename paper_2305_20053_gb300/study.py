"""Cost-accuracy study of Sec. 4.1-4.2: optimal controls of the CVaR OUU problem computed by
the plain PDE path with small SAA sample sets, and by MR-NO / MR-DINO surrogates trained on
growing data sets, judged by the relative optimal cost error against a reference solved by
the PDE path with a large sample set.

Cost of a solution, as the paper counts it: state PDE solves.  PDE-SAA: optimiser
evaluations x N (each evaluation solves N states); surrogate: the training samples (their
generation dominates; the surrogate's own SAA solve uses no PDE solve).

Every optimum is evaluated by the same reference evaluator (the plain path over the
reference fields, CVaR at its minimising t), so the errors compare like with like.

  python -m paper_2305_20053_gb300.study [--n 129] [--L 10] [--betas 0.9 0.95 0.99] [--out study.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_20053_gb300 import capi, ouu  # noqa: E402
from paper_2305_20053_gb300 import train as T  # noqa: E402
from synthetic_inputs import SEED_SAA  # noqa: E402

EPS = 1e-4


def _fields(P, seed, first, N):
    import torch
    m = torch.empty(N, P.n, P.n, dtype=torch.float64, device="cuda")
    P.ouu_sample_fields(seed, first, N, m)
    return m


def run(n=129, L=10, betas=(0.9, 0.95, 0.99), n_ref=4096, pde_sizes=(16, 32, 64, 128, 256),
        train_sizes=(512, 1024, 2048, 4096), n_nn=2048, epochs=1600, maxiter=200, log=print):
    import torch
    torch.cuda.set_device(0)
    capi.load()
    P = capi.Problem(n=n, lattice_L=L, max_samples=max(n_ref, max(train_sizes)))
    m_ref = _fields(P, SEED_SAA, 0, n_ref)
    # the PDE-SAA runs and the surrogates' SAA draw their fields from other index ranges of the
    # same stream than the reference set
    m_nn = _fields(P, SEED_SAA, 1_000_000, n_nn)
    out = {"n": n, "d_z": L * L, "eps": EPS, "n_ref": n_ref, "n_nn": n_nn, "epochs": epochs, "betas": {}}
    # surrogates: one data set (the largest), prefixes of it for the smaller sizes
    D = T.make_dino(n, L, max_eval=max(n_ref, n_nn))
    T.init_params(D)
    t0 = time.perf_counter()
    data = T.generate_training_data(P, D, max(train_sizes))
    out["data_s"] = time.perf_counter() - t0
    nets = {}
    for size in train_sizes:
        for kind, wj in (("mr-no", 0.0), ("mr-dino", 1.0)):
            Dk = T.make_dino(n, L, max_eval=max(n_ref, n_nn), jac_weight=wj)
            T.init_params(Dk)
            phi = torch.empty(Dk.desc.r_u, n, n, dtype=torch.float64, device="cuda")
            ub = torch.empty(n, n, dtype=torch.float64, device="cuda")
            D.ouu_dino_get_bases(phi, ub)   # the POD basis of the data set's first states
            Dk.ouu_dino_set_bases(phi, ub)
            Dk.ouu_dino_set_output_scale(D.ouu_dino_get_output_scale())
            sub = T.TrainData(data.xi[:size], data.z[:size], data.y[:size], data.jy[:size], data.eig, data.times)
            secs, _ = T.train(Dk, sub, epochs=epochs, batch=min(256, size), lr_final=1e-5)
            nets[(kind, size)] = Dk
            log(f"trained {kind} on {size} samples in {secs:.1f} s")
    del data
    for beta in betas:
        rd = capi.risk_desc(capi.RISK_CVAR_SMOOTH, beta=beta, eps=EPS)
        ref = ouu.solve(P, capi.BACKEND_PDE, None, m_ref, n_ref, rd, maxiter=maxiter)
        j_ref = ouu.reference_cost(P, m_ref, n_ref, rd, ref.z)
        row = {"reference": {"cost": j_ref, "evaluations": ref.evaluations, "converged": ref.converged},
               "pde": [], "surrogate": []}
        for k, N in enumerate(pde_sizes):
            m = _fields(P, SEED_SAA, 2_000_000 + 10_000 * k, N)
            r = ouu.solve(P, capi.BACKEND_PDE, None, m, N, rd, maxiter=maxiter)
            row["pde"].append({"N": N, "state_solves": r.evaluations * N,
                               "rel_cost_error": ouu.relative_cost_error(
                                   ouu.reference_cost(P, m_ref, n_ref, rd, r.z), j_ref)})
        for (kind, size), Dk in nets.items():
            r = ouu.solve(P, capi.BACKEND_DINO, Dk, m_nn, n_nn, rd, maxiter=maxiter)
            row["surrogate"].append({"kind": kind, "train_samples": size, "state_solves": size,
                                     "evaluations": r.evaluations,
                                     "rel_cost_error": ouu.relative_cost_error(
                                         ouu.reference_cost(P, m_ref, n_ref, rd, r.z), j_ref)})
        out["betas"][str(beta)] = row
        log(json.dumps({"beta": beta, **row}))
    for Dk in nets.values():
        Dk.close()
    D.close()
    P.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=129)
    ap.add_argument("--L", type=int, default=10)
    ap.add_argument("--betas", type=float, nargs="+", default=[0.9, 0.95, 0.99])
    ap.add_argument("--epochs", type=int, default=1600)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    res = run(args.n, args.L, tuple(args.betas), epochs=args.epochs)
    print(json.dumps(res))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
