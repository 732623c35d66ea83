// One sample average spread over ranks (ouu_shard_qoi, ouu_shard_risk_partial).
//
// Sec. 2.2 defines the SAA risk over ONE fixed sample set and Sec. 2.3 its gradient as ONE
// weighted sum over that set.  When the set is split into contiguous blocks, one per rank
// (GPU), the only quantities that need every sample are the QoIs: the mean (and variance)
// and the CVaR minimiser t* depend on all Q_i, and through them every weight w_i.  So one
// evaluation is
//   phase 1  each rank: Q_i of its block (state solves, or the network)        [device]
//   exchange all-gather of the Q_i (8 N bytes)                                  [caller]
//   phase 2  each rank: moments, t*, risk values and d rho/dt from all Q_i (the same on
//            every rank), the weights of its block, and its part of the gradient
//            sum_{i in block} w_i grad_z Q_i (plain: adjoint solves of its samples with a
//            nonzero weight; network: its reverse-mode gradients)              [device]
//   exchange FP64 all-reduce (sum) of the n_risks x d_Z gradient parts          [caller]
// The collectives belong to the caller (NCCL between GPUs, gloo in the CPU tests); the
// library stays one process on one GPU.
#include <algorithm>
#include <cstring>

#include "dino.cuh"
#include "ouu_internal.cuh"

static int grid_for_solver(ouu_problem* p, int n) { return std::max(1, std::min(p->nslots, n)); }

static ouu_status sample_statuses(ouu_problem* p, int n) {
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat, p->d_status, (size_t)n * 4, cudaMemcpyDeviceToHost, p->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(p->stream));
  int worst = 0, nbad = 0;
  for (int i = 0; i < n; ++i) {
    worst = std::max(worst, (int)p->h_stat[i]);
    nbad += p->h_stat[i] != 0;
  }
  if (worst == OUU_SAMPLE_NOT_CONVERGED) {
    ouu_set_error(std::to_string(nbad) + " samples did not converge");
    return OUU_ERR_NOT_CONVERGED;
  }
  if (worst == OUU_SAMPLE_NONFINITE) {
    ouu_set_error("non-finite residual in some sample");
    return OUU_ERR_NONFINITE;
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_shard_qoi(ouu_problem_t p, ouu_backend backend, ouu_dino_t dino, const double* m_dev,
                                    int n_local, const double* z_host, double* q_local_dev) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(m_dev && z_host && q_local_dev, "null argument");
  OUU_CHECK_ARG(n_local >= 1 && n_local <= p->desc.max_samples, "n_local outside [1, max_samples]");
  OUU_CHECK_ARG(backend == OUU_BACKEND_PDE || backend == OUU_BACKEND_DINO || backend == OUU_BACKEND_AUTO,
                "unknown backend");
  for (int j = 0; j < p->dz; ++j) OUU_CHECK_ARG(std::isfinite(z_host[j]), "z has a non-finite entry");
  if (backend == OUU_BACKEND_AUTO)
    backend = dino_trusted(dino, p, n_local) ? OUU_BACKEND_DINO : OUU_BACKEND_PDE;
  p->shard_backend = -1;
  if (backend == OUU_BACKEND_DINO) {
    OUU_CHECK_ARG(dino != nullptr, "DINO backend needs a trained network");
    OUU_CHECK_ARG(dino->n == p->n && dino->dz == p->dz, "problem and network grids differ");
    OUU_CHECK_ARG(n_local <= dino->maxE, "n_local exceeds the network's max_eval");
    if (!dino->bases_ready) {
      ouu_set_error("network bases not built");
      return OUU_ERR_STATE;
    }
    if (ouu_status st = dino_eval_core(dino, m_dev, n_local, z_host, true)) return st;
    OUU_CUDA_TRY(cudaMemcpyAsync(q_local_dev, dino->Qe, (size_t)n_local * 8, cudaMemcpyDeviceToDevice, dino->stream));
    OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat, dino->d_err, 4, cudaMemcpyDeviceToHost, dino->stream));
    OUU_CUDA_TRY(cudaStreamSynchronize(dino->stream));
    if (p->h_stat[0]) {
      cudaMemsetAsync(dino->d_err, 0, 4, dino->stream);
      cudaMemsetAsync(dino->d_klp_ctr, 0, (OUU_KLP_MAX_TILES + 1) * sizeof(int), dino->stream);
      ouu_set_error("tensor-core GEMM pipeline wait timed out");
      return OUU_ERR_CUDA;
    }
  } else {
    std::memcpy(p->h_out, z_host, (size_t)p->dz * 8);
    OUU_CUDA_TRY(cudaMemcpyAsync(p->d_z, p->h_out, (size_t)p->dz * 8, cudaMemcpyHostToDevice, p->stream));
    PdeArgs a = ouu_base_args(p, n_local);
    a.m = m_dev;
    a.z = p->d_z;
    a.z_stride = 0;
    a.u = p->d_u;
    a.q = p->d_q;
    OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
    launch_pde_state(a, grid_for_solver(p, n_local), p->stream);
    OUU_CUDA_TRY(cudaGetLastError());
    OUU_CUDA_TRY(cudaMemcpyAsync(q_local_dev, p->d_q, (size_t)n_local * 8, cudaMemcpyDeviceToDevice, p->stream));
    if (ouu_status st = sample_statuses(p, n_local)) return st;
  }
  p->shard_backend = backend;
  p->shard_m = m_dev;
  p->shard_n = n_local;
  p->shard_dino = backend == OUU_BACKEND_DINO ? dino : nullptr;
  p->shard_dino_eval = backend == OUU_BACKEND_DINO ? dino->eval_count : 0;
  return OUU_OK;
}

extern "C" ouu_status ouu_shard_risk_partial(ouu_problem_t p, ouu_dino_t dino, const double* q_all_dev, int n_total,
                                             int64_t first_local, const ouu_risk_desc* risks, int n_risks,
                                             double* risk_out, double* grad_part_out, double* grad_t_out,
                                             double* t_out) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(q_all_dev && risk_out && grad_part_out && grad_t_out, "null argument");
  if (p->shard_backend < 0) {
    ouu_set_error("no pending ouu_shard_qoi on this problem");
    return OUU_ERR_STATE;
  }
  const int n_local = p->shard_n, backend = p->shard_backend;
  OUU_CHECK_ARG(backend != OUU_BACKEND_DINO || dino == p->shard_dino, "not the network of the pending ouu_shard_qoi");
  if (backend == OUU_BACKEND_DINO && dino->eval_count != p->shard_dino_eval) {
    // its per-sample gradients now belong to a later evaluation: each rank needs its own network
    p->shard_backend = -1;
    ouu_set_error("the network evaluated other samples since this problem's ouu_shard_qoi");
    return OUU_ERR_STATE;
  }
  OUU_CHECK_ARG(n_total >= n_local && first_local >= 0 && first_local + n_local <= (int64_t)n_total,
                "the block [first_local, first_local + n_local) must lie in [0, n_total)");
  if (ouu_status st = ouu_check_risks(risks, n_risks)) return st;
  p->shard_backend = -1;   // phase 2 consumes phase 1's per-sample state
  RiskDev rd[OUU_MAX_RISKS];
  ouu_risk_dev(risks, n_risks, n_total, rd);
  const int dz = p->dz, first = (int)first_local;
  double* d_res = p->d_out;
  double* d_grad = p->d_out + 3 * OUU_MAX_RISKS;
  const size_t out_bytes = (size_t)(OUU_MAX_RISKS * (3 + dz) + 8) * 8;
  cudaStream_t s;
  if (backend == OUU_BACKEND_DINO) {
    s = dino->stream;
    if (ouu_status st = ouu_upload_risks(p, rd, n_risks, s)) return st;
    launch_risk_weights(q_all_dev, n_total, p->d_risks, n_risks, p->d_w, d_res, p->d_rscr, s, dino->GQe,
                        (dz + 7) / 8 * 8, dz, d_grad, first, n_local);
  } else {
    s = p->stream;
    if (ouu_status st = ouu_upload_risks(p, rd, n_risks, s)) return st;
    int* d_solved = (int*)(p->d_out + OUU_MAX_RISKS * (3 + dz));
    launch_risk_weights(q_all_dev, n_total, p->d_risks, n_risks, p->d_w, d_res, p->d_rscr, s, nullptr, 0, 0,
                        nullptr, first, n_local);
    PdeArgs a = ouu_base_args(p, n_local);
    a.m = p->shard_m;
    a.z = p->d_z;
    a.z_stride = 0;
    a.u = p->d_u;
    a.q = p->d_q;
    a.w = p->d_w;   // [n_risks][n_local]: the weights of this block
    a.n_w = n_risks;
    a.solved = d_solved;
    OUU_CUDA_TRY(cudaMemsetAsync(d_solved, 0, 4, s));
    OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, s));
    launch_pde_adjoint(a, grid_for_solver(p, n_local), s);
    launch_reduce_slots_and_gradient(p->d_slots, p->lay, grid_for_solver(p, n_local), p->n, p->L, n_risks, p->d_gx,
                                     p->d_gy, p->gscale, p->d_s, d_grad, s);
  }
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_out, p->d_out, out_bytes, cudaMemcpyDeviceToHost, s));
  OUU_CUDA_TRY(cudaStreamSynchronize(s));
  for (int r = 0; r < n_risks; ++r) {
    risk_out[r] = p->h_out[3 * r + 0];
    grad_t_out[r] = p->h_out[3 * r + 1];
    if (t_out) t_out[r] = p->h_out[3 * r + 2];
    std::memcpy(grad_part_out + (size_t)r * dz, p->h_out + 3 * OUU_MAX_RISKS + (size_t)r * dz, (size_t)dz * 8);
  }
  if (backend == OUU_BACKEND_PDE) return sample_statuses(p, n_local);
  return OUU_OK;
}
