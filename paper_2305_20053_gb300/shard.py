"""One SAA risk + gradient evaluation over a sample set spread across ranks (one process per GPU).

Sec. 2.2 defines the risk over ONE fixed sample set and Sec. 2.3 its gradient as ONE weighted
sum over it.  Rank k holds the contiguous block [first_k, first_k + n_k) of the n_total
samples.  Every weight depends on all QoIs (through the mean and, for CVaR, t*), so one
evaluation is: the library's phase 1 on every rank (QoIs of its block), an all-gather of the
QoIs (8 n_total bytes), the library's phase 2 on every rank (risk values, d rho / dt and t
from all QoIs, the same on every rank; this rank's part of the weighted gradient sum), and an
FP64 all-reduce (sum) of the n_risks x d_Z gradient parts.  The collectives go through
torch.distributed (NCCL between GPUs, gloo on CPU); this module only moves the numbers.
"""
from __future__ import annotations

import numpy as np


class ShardedSAA:
    """The exchange plan of one sample set spread over the ranks of `group` (torch.distributed;
    a single process when it is not initialised).  The block sizes are exchanged once here;
    each evaluate() then takes one all-gather and one all-reduce."""

    def __init__(self, n_local, device, group=None):
        import torch
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.device = torch.device(device)
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.world = self.dist.get_world_size(group) if self.dist else 1
        counts = torch.tensor([int(n_local)], dtype=torch.int64, device=self.device)
        if self.dist:
            parts = [torch.zeros_like(counts) for _ in range(self.world)]
            self.dist.all_gather(parts, counts, group=group)
            counts = torch.cat(parts)
        self.counts = [int(c) for c in counts.cpu()]
        self.n_local = int(n_local)
        self.first = sum(self.counts[:self.rank])
        self.n_total = sum(self.counts)
        self.n_max = max(self.counts)

    def gather_q(self, q_local):
        """The QoIs of all ranks in rank order, [n_total] float64 on self.device."""
        import torch
        if self.dist is None:
            return q_local[:self.n_local]
        buf = torch.zeros(self.n_max, dtype=torch.float64, device=self.device)
        buf[:self.n_local] = q_local[:self.n_local]
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf, group=self.group)
        return torch.cat([p[:c] for p, c in zip(parts, self.counts)])

    def sum_over_ranks(self, grad_part):
        """FP64 sum of every rank's gradient part (host array in, host array out)."""
        import torch
        if self.dist is None:
            return np.array(grad_part, dtype=np.float64)
        g = torch.tensor(np.ascontiguousarray(grad_part, dtype=np.float64), device=self.device)
        self.dist.all_reduce(g, op=self.dist.ReduceOp.SUM, group=self.group)
        return g.cpu().numpy()

    def evaluate(self, qoi, partial):
        """qoi() -> this rank's QoIs (tensor [n_local] on self.device);
        partial(q_all, n_total, first) -> (risk, grad_part, grad_t, t).
        Returns (risk, grad_z, grad_t, t) of the whole sample set, the same on every rank."""
        q_all = self.gather_q(qoi())
        risk, grad_part, grad_t, t = partial(q_all, self.n_total, self.first)
        return risk, self.sum_over_ranks(grad_part), grad_t, t


def risk_and_grad(problem, backend, dino, m_local, risks, z_host, plan: ShardedSAA, q_local=None):
    """ouu_risk_and_grad over the sample set spread as `plan` says, this rank's fields in
    m_local [n_local][n][n] (device): the library's two phases around the two exchanges."""
    import torch
    if q_local is None:
        q_local = torch.empty(plan.n_local, dtype=torch.float64, device=plan.device)

    def qoi():
        problem.ouu_shard_qoi(backend, dino, m_local, plan.n_local, z_host, q_local)
        return q_local

    def partial(q_all, n_total, first):
        return problem.ouu_shard_risk_partial(dino, q_all, n_total, first, risks)

    return plan.evaluate(qoi, partial)
