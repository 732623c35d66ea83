// Uneven batches of OUU problems evaluated together (ouu_batch_* in ouu.h): the plain
// problems' state and adjoint solves each in one persistent launch over all their samples
// (tasks ordered largest grid first, so the long tasks start early and the short ones fill
// the tail), every MR-DINO problem on a concurrent branch, the whole batch one CUDA graph.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dino.cuh"
#include "ouu_internal.cuh"
#include "tc_gemm.cuh"

#define BATCH_SIDE_STREAMS 8

// Global-timer stamp (ns) written by one thread: graph nodes that mark phases for timing.
__global__ void k_stamp(unsigned long long* at) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *at = t;
}

struct BatchEntry {
  ouu_batch_item it;
  ouu_risk_desc risks[OUU_MAX_RISKS];
  int pde_pos = -1;                         // position in the plain-problem table
  int dino_pos = -1;                        // MR-DINO branch number
};

struct ouu_batch {
  std::vector<BatchEntry> items;
  std::vector<int> pde, dino;                 // item indices (pde: largest grid first)
  cudaStream_t stream = nullptr;                // runs: the first item's problem stream
  cudaStream_t cap = nullptr;                   // private stream the graph is captured on
  cudaStream_t side[BATCH_SIDE_STREAMS] = {};
  cudaEvent_t fork = nullptr, join[BATCH_SIDE_STREAMS] = {};
  unsigned long long* d_stamp = nullptr;        // [2 + 2 n_dino] ns: batch start/end, branch start/end
  unsigned long long* h_stamp = nullptr;
  PdeArgs* d_args = nullptr;
  int2* d_tasks = nullptr;
  int n_tasks = 0;
  char* d_slots = nullptr;
  int64_t slot_bytes = 0, smem_bytes = 0;
  int nslots = 0;
  int* d_counter = nullptr;                   // [2]: state, adjoint
  unsigned long long* d_cycles = nullptr;     // [2][n_pde]
  unsigned long long* h_cycles = nullptr;     // pinned mirror
  double* h_z = nullptr;                      // pinned staging of the plain problems' controls
  std::vector<size_t> zoff;
  cudaGraphExec_t gexec = nullptr;
  double clock_khz = 0.0;
};

static void free_batch(ouu_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->d_args);
  cudaFree(b->d_tasks);
  cudaFree(b->d_slots);
  cudaFree(b->d_counter);
  cudaFree(b->d_cycles);
  if (b->h_cycles) cudaFreeHost(b->h_cycles);
  if (b->h_z) cudaFreeHost(b->h_z);
  cudaFree(b->d_stamp);
  if (b->h_stamp) cudaFreeHost(b->h_stamp);
  for (int s = 0; s < BATCH_SIDE_STREAMS; ++s) {
    if (b->side[s]) cudaStreamDestroy(b->side[s]);
    if (b->join[s]) cudaEventDestroy(b->join[s]);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

static ouu_status check_item(const ouu_batch_item& it) {
  OUU_CHECK_ARG(it.problem && it.m_dev, "batch item: problem and fields are required");
  ouu_problem* p = it.problem;
  OUU_CHECK_ARG(it.n_samples >= 1 && it.n_samples <= p->desc.max_samples, "batch item: n_samples outside [1, max_samples]");
  if (ouu_status st = ouu_check_risks(it.risks, it.n_risks)) return st;
  OUU_CHECK_ARG(it.backend == OUU_BACKEND_PDE || it.backend == OUU_BACKEND_DINO, "batch item: unknown backend");
  if (it.backend == OUU_BACKEND_DINO) {
    ouu_dino* d = it.dino;
    OUU_CHECK_ARG(d != nullptr, "batch item: MR-DINO item without a network");
    OUU_CHECK_ARG(d->n == p->n && d->dz == p->dz, "batch item: network and problem grids differ");
    OUU_CHECK_ARG(it.n_samples <= d->maxE, "batch item: n_samples exceeds the network's max_eval");
    if (!d->bases_ready) {
      ouu_set_error("batch item: network bases not built");
      return OUU_ERR_STATE;
    }
  }
  return OUU_OK;
}

#define BATCH_TRY(expr)            \
  do {                             \
    ouu_status st_ = (expr);       \
    if (st_ != OUU_OK) {           \
      free_batch(b);               \
      return st_;                  \
    }                              \
  } while (0)

#define BATCH_CUDA(expr)                                                         \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ouu_set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));         \
      free_batch(b);                                                             \
      return OUU_ERR_CUDA;                                                       \
    }                                                                            \
  } while (0)

extern "C" ouu_status ouu_batch_create(const ouu_batch_item* items_in, int n_items, int autotune, ouu_batch_t* out) {
  OUU_CHECK_ARG(items_in && out && n_items >= 1, "need items and an output handle");
  *out = nullptr;
  // AUTO items take their backend now: the network if it passed its held-out check for the
  // item's problem, else the plain path
  std::vector<ouu_batch_item> resolved(items_in, items_in + n_items);
  for (ouu_batch_item& it : resolved)
    if (it.backend == OUU_BACKEND_AUTO) {
      it.backend = dino_trusted(it.dino, it.problem, it.n_samples) ? OUU_BACKEND_DINO : OUU_BACKEND_PDE;
      if (it.backend == OUU_BACKEND_PDE) it.dino = nullptr;
    }
  const ouu_batch_item* items = resolved.data();
  for (int k = 0; k < n_items; ++k) {
    if (ouu_status st = check_item(items[k])) return st;
    for (int j = 0; j < k; ++j) {
      OUU_CHECK_ARG(items[j].problem != items[k].problem, "batch items must not share a problem");
      OUU_CHECK_ARG(items[k].backend != OUU_BACKEND_DINO || items[j].backend != OUU_BACKEND_DINO ||
                        items[j].dino != items[k].dino,
                    "batch items must not share a network (concurrent branches would share its buffers)");
    }
  }
  ouu_batch* b = new ouu_batch();
  b->stream = items[0].problem->stream;
  b->items.resize(n_items);
  size_t zsum = 0;
  for (int k = 0; k < n_items; ++k) {
    BatchEntry& e = b->items[k];
    e.it = items[k];
    std::memcpy(e.risks, items[k].risks, sizeof(ouu_risk_desc) * items[k].n_risks);
    e.it.risks = e.risks;
    (e.it.backend == OUU_BACKEND_DINO ? b->dino : b->pde).push_back(k);
    b->zoff.push_back(zsum);
    zsum += (size_t)items[k].problem->dz;
    // risk descriptors for this item's N go to its problem's arena once
    RiskDev rd[OUU_MAX_RISKS];
    for (int r = 0; r < e.it.n_risks; ++r) {
      rd[r].kind = e.risks[r].kind;
      rd[r].kappa = e.risks[r].kappa;
      rd[r].beta = e.risks[r].beta;
      rd[r].eps = e.risks[r].eps;
      rd[r].t = e.risks[r].t;
      rd[r].t_optimal = e.risks[r].t_optimal;
      risk_dev_finish(rd[r], e.it.n_samples);
    }
    BATCH_CUDA(cudaMemcpy(e.it.problem->d_risks, rd, sizeof(RiskDev) * e.it.n_risks, cudaMemcpyHostToDevice));
    e.it.problem->rd_n = -1;   // ouu_risk_and_grad's record of the uploaded descriptors is stale
    if (e.it.backend == OUU_BACKEND_DINO) e.dino_pos = (int)b->dino.size() - 1;
  }
  for (int s = 0; s < BATCH_SIDE_STREAMS; ++s) {
    BATCH_CUDA(cudaStreamCreateWithFlags(&b->side[s], cudaStreamNonBlocking));
    BATCH_CUDA(cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming));
  }
  BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  BATCH_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  BATCH_CUDA(cudaMalloc((void**)&b->d_stamp, (2 + 2 * b->dino.size()) * 8));
  BATCH_CUDA(cudaMallocHost((void**)&b->h_stamp, (2 + 2 * b->dino.size()) * 8));
  BATCH_CUDA(cudaMallocHost((void**)&b->h_z, std::max<size_t>(zsum, 1) * 8));
  int dev = 0, sms = 1, clk = 0;
  BATCH_CUDA(cudaGetDevice(&dev));
  BATCH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  cudaGetLastError();
  b->clock_khz = clk > 0 ? (double)clk : 2.0e6;
  // plain problems: argument table, task list, shared slot pool
  if (!b->pde.empty()) {
    std::stable_sort(b->pde.begin(), b->pde.end(), [&](int x, int y) {
      const ouu_problem* px = b->items[x].it.problem;
      const ouu_problem* py = b->items[y].it.problem;
      return px->n != py->n ? px->n > py->n : b->items[x].it.n_samples > b->items[y].it.n_samples;
    });
    std::vector<PdeArgs> args;
    std::vector<int2> tasks;
    for (int j = 0; j < (int)b->pde.size(); ++j) {
      BatchEntry& e = b->items[b->pde[j]];
      ouu_problem* p = e.it.problem;
      e.pde_pos = j;
      PdeArgs a = ouu_base_args(p, e.it.n_samples);
      a.m = e.it.m_dev;
      a.z = p->d_z;
      a.z_stride = 0;
      a.u = p->d_u;
      a.q = p->d_q;
      a.w = p->d_w;
      a.n_w = e.it.n_risks;
      a.acc_out = p->d_s;
      a.slots = nullptr;   // the batch pool
      a.counter = nullptr;
      args.push_back(a);
      b->slot_bytes = std::max<int64_t>(b->slot_bytes, p->lay.bytes);
      b->smem_bytes = std::max<int64_t>(b->smem_bytes, p->lay.smem_bytes);
      for (int i = 0; i < e.it.n_samples; ++i) tasks.push_back(make_int2(j, i));
    }
    b->slot_bytes = (b->slot_bytes + 255) / 256 * 256;
    b->n_tasks = (int)tasks.size();
    // the persistent launch holds its SMs until it ends: leave some to the MR-DINO branches
    const int reserve = b->dino.empty() ? 0 : std::min(16, sms / 4);
    b->nslots = std::max(1, std::min(sms - reserve, b->n_tasks));
    BATCH_CUDA(cudaMalloc((void**)&b->d_args, sizeof(PdeArgs) * args.size()));
    BATCH_CUDA(cudaMemcpy(b->d_args, args.data(), sizeof(PdeArgs) * args.size(), cudaMemcpyHostToDevice));
    BATCH_CUDA(cudaMalloc((void**)&b->d_tasks, sizeof(int2) * tasks.size()));
    BATCH_CUDA(cudaMemcpy(b->d_tasks, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice));
    BATCH_CUDA(cudaMalloc((void**)&b->d_slots, (size_t)b->slot_bytes * b->nslots));
    BATCH_CUDA(cudaMalloc((void**)&b->d_counter, 16));
  }
  const size_t np = std::max<size_t>(b->pde.size(), 1);
  BATCH_CUDA(cudaMalloc((void**)&b->d_cycles, 2 * np * 8));
  BATCH_CUDA(cudaMallocHost((void**)&b->h_cycles, 2 * np * 8));
  // Autotuning of every MR-DINO problem's evaluation: the per-layer GEMM path with its N tiles
  // timed per layer shape, against the one-kernel networks (one CTA per 128 samples, and 4-CTA
  // clusters per 128 samples); the fastest is kept.
  if (autotune && !b->dino.empty()) {
    ouu_status st = OUU_OK;
    cudaEvent_t t0, t1;
    BATCH_CUDA(cudaEventCreate(&t0));
    BATCH_CUDA(cudaEventCreate(&t1));
    for (int k : b->dino) {
      BatchEntry& e = b->items[k];
      ouu_dino* d = e.it.dino;
      std::vector<double> z0(e.it.problem->dz, 0.0);
      float ms[3] = {1e30f, 1e30f, 1e30f};
      const int fits[3] = {1, mlp_fused_fits(d) ? 1 : 0, mlp_cluster_fits(d) ? 1 : 0};
      for (int mode = 0; mode < 3 && st == OUU_OK; ++mode) {
        if (!fits[mode]) continue;
        d->fused_mlp = mode;
        if (mode == 0) ouu_gemm_set_autotune(1);
        for (int rep = 0; rep < 2 && st == OUU_OK; ++rep) {   // the second run is timed
          cudaEventRecord(t0, d->stream);
          st = dino_enqueue_risk(e.it.problem, d, e.it.m_dev, e.it.n_samples, e.it.n_risks, z0.data());
          cudaEventRecord(t1, d->stream);
          if (st == OUU_OK && cudaEventSynchronize(t1) != cudaSuccess) st = OUU_ERR_CUDA;
          if (st == OUU_OK && rep == 1) cudaEventElapsedTime(&ms[mode], t0, t1);
        }
        ouu_gemm_set_autotune(0);
      }
      int best = 0;
      for (int mode = 1; mode < 3; ++mode)
        if (fits[mode] && ms[mode] < ms[best]) best = mode;
      d->fused_mlp = best;
      if (d->gexec) {   // the network's own captured evaluation may hold the other path
        cudaGraphExecDestroy(d->gexec);
        d->gexec = nullptr;
      }
      if (st != OUU_OK) break;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    BATCH_TRY(st);
  }
  *out = b;
  return OUU_OK;
}

extern "C" void ouu_batch_destroy(ouu_batch_t b) { free_batch(b); }

// The whole batch, enqueued on the capture stream (captured into the graph by the first run).
static ouu_status enqueue_batch(ouu_batch* b, const double* const* z_hosts) {
  cudaStream_t ms = b->cap;
  k_stamp<<<1, 1, 0, ms>>>(b->d_stamp);
  for (int k : b->pde) {
    ouu_problem* p = b->items[k].it.problem;
    OUU_CUDA_TRY(cudaMemcpyAsync(p->d_z, b->h_z + b->zoff[k], (size_t)p->dz * 8, cudaMemcpyHostToDevice, ms));
  }
  if (!b->pde.empty()) {
    OUU_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, 8, ms));
    OUU_CUDA_TRY(cudaMemsetAsync(b->d_cycles, 0, 2 * b->pde.size() * 8, ms));
    for (int k : b->pde) {
      const BatchEntry& e = b->items[k];
      ouu_problem* p = e.it.problem;
      OUU_CUDA_TRY(cudaMemsetAsync(p->d_s, 0, (size_t)e.it.n_risks * p->n * p->n * 8, ms));
    }
  }
  // MR-DINO problems on branches
  OUU_CUDA_TRY(cudaEventRecord(b->fork, ms));
  const int nbr = std::min<int>((int)b->dino.size(), BATCH_SIDE_STREAMS);
  for (int s = 0; s < nbr; ++s) OUU_CUDA_TRY(cudaStreamWaitEvent(b->side[s], b->fork, 0));
  for (int j = 0; j < (int)b->dino.size(); ++j) {
    BatchEntry& e = b->items[b->dino[j]];
    ouu_dino* d = e.it.dino;
    cudaStream_t ss = b->side[j % BATCH_SIDE_STREAMS];
    cudaStream_t own = d->stream;
    d->stream = ss;
    d->capturing = true;
    k_stamp<<<1, 1, 0, ss>>>(b->d_stamp + 2 + 2 * j);
    const ouu_status st = dino_enqueue_risk(e.it.problem, d, e.it.m_dev, e.it.n_samples, e.it.n_risks,
                                            z_hosts[b->dino[j]]);
    if (st == OUU_OK) k_stamp<<<1, 1, 0, ss>>>(b->d_stamp + 3 + 2 * j);
    d->stream = own;
    d->capturing = false;
    if (st != OUU_OK) return st;
  }
  // plain problems: one persistent launch per solve kind over all their samples
  if (!b->pde.empty()) {
    launch_pde_batch(b->d_args, b->d_tasks, b->n_tasks, b->d_slots, b->slot_bytes, b->smem_bytes, b->nslots,
                     b->d_counter, b->d_cycles, false, ms);
    for (int k : b->pde) {
      const BatchEntry& e = b->items[k];
      ouu_problem* p = e.it.problem;
      launch_risk_weights(p->d_q, e.it.n_samples, p->d_risks, e.it.n_risks, p->d_w, p->d_out, p->d_rscr, ms);
    }
    launch_pde_batch(b->d_args, b->d_tasks, b->n_tasks, b->d_slots, b->slot_bytes, b->smem_bytes, b->nslots,
                     b->d_counter + 1, b->d_cycles + b->pde.size(), true, ms);
    for (int k : b->pde) {
      const BatchEntry& e = b->items[k];
      ouu_problem* p = e.it.problem;
      launch_sources_transpose(p->n, p->L, e.it.n_risks, p->d_gx, p->d_gy, p->gscale, p->d_s,
                               p->d_out + 3 * OUU_MAX_RISKS, ms);
      const size_t ob = (size_t)(OUU_MAX_RISKS * (3 + p->dz) + 8) * 8;
      OUU_CUDA_TRY(cudaMemcpyAsync(p->h_out, p->d_out, ob, cudaMemcpyDeviceToHost, ms));
      OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat, p->d_status, (size_t)e.it.n_samples * 4, cudaMemcpyDeviceToHost, ms));
    }
    OUU_CUDA_TRY(cudaMemcpyAsync(b->h_cycles, b->d_cycles, 2 * b->pde.size() * 8, cudaMemcpyDeviceToHost, ms));
  }
  for (int s = 0; s < nbr; ++s) {
    OUU_CUDA_TRY(cudaEventRecord(b->join[s], b->side[s]));
    OUU_CUDA_TRY(cudaStreamWaitEvent(ms, b->join[s], 0));
  }
  k_stamp<<<1, 1, 0, ms>>>(b->d_stamp + 1);
  OUU_CUDA_TRY(cudaMemcpyAsync(b->h_stamp, b->d_stamp, (2 + 2 * b->dino.size()) * 8, cudaMemcpyDeviceToHost, ms));
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

extern "C" ouu_status ouu_batch_run(ouu_batch_t b, const double* const* z_hosts, double* const* risk_out,
                                    double* const* grad_z_out, double* const* grad_t_out, double* const* t_out,
                                    double* item_ms, double* total_ms) {
  OUU_CHECK_ARG(b && z_hosts && risk_out && grad_z_out && grad_t_out, "null argument");
  const int nk = (int)b->items.size();
  for (int k = 0; k < nk; ++k) {
    OUU_CHECK_ARG(z_hosts[k] && risk_out[k] && grad_z_out[k] && grad_t_out[k], "null per-item pointer");
    const int dz = b->items[k].it.problem->dz;
    for (int j = 0; j < dz; ++j) OUU_CHECK_ARG(std::isfinite(z_hosts[k][j]), "z has a non-finite entry");
  }
  // controls: plain problems through the staging copy nodes, MR-DINO ones through the
  // networks' pinned z buffers (the copy nodes of their branches read them)
  for (int k : b->pde)
    std::memcpy(b->h_z + b->zoff[k], z_hosts[k], (size_t)b->items[k].it.problem->dz * 8);
  for (int k : b->dino) {
    float* zh = (float*)b->items[k].it.dino->h_pin;
    for (int j = 0; j < b->items[k].it.problem->dz; ++j) zh[j] = (float)z_hosts[k][j];
  }
  if (!b->gexec) {
    cudaGraph_t g = nullptr;
    OUU_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const ouu_status st = enqueue_batch(b, z_hosts);
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (st != OUU_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ce != cudaSuccess || !g) {
      ouu_set_error(std::string("batch graph capture failed: ") + cudaGetErrorString(ce));
      cudaGetLastError();
      return OUU_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      b->gexec = nullptr;
      ouu_set_error(std::string("batch graph instantiation failed: ") + cudaGetErrorString(ie));
      return OUU_ERR_CUDA;
    }
  }
  for (int k : b->dino) ++b->items[k].it.dino->eval_count;   // their per-sample buffers are rewritten
  OUU_CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(b->stream));
  int worst = 0;
  for (int k = 0; k < nk; ++k) {
    const BatchEntry& e = b->items[k];
    ouu_problem* p = e.it.problem;
    const int dz = p->dz;
    if (e.it.backend == OUU_BACKEND_DINO) {
      if (p->h_out[OUU_OUT_FLAG(dz)] != 0.0) {
        cudaMemsetAsync(e.it.dino->d_err, 0, 4, b->stream);
        ouu_set_error("tensor-core GEMM pipeline wait timed out");
        return OUU_ERR_CUDA;
      }
    } else {
      for (int i = 0; i < e.it.n_samples; ++i) worst = std::max(worst, (int)p->h_stat[i]);
    }
    for (int r = 0; r < e.it.n_risks; ++r) {
      risk_out[k][r] = p->h_out[3 * r + 0];
      grad_t_out[k][r] = p->h_out[3 * r + 1];
      if (t_out && t_out[k]) t_out[k][r] = p->h_out[3 * r + 2];
      std::memcpy(grad_z_out[k] + (size_t)r * dz, p->h_out + 3 * OUU_MAX_RISKS + (size_t)r * dz, (size_t)dz * 8);
    }
    if (item_ms) {
      if (e.it.backend == OUU_BACKEND_DINO) {
        item_ms[k] = 1e-6 * (double)(b->h_stamp[3 + 2 * e.dino_pos] - b->h_stamp[2 + 2 * e.dino_pos]);
      } else {
        const unsigned long long cyc = b->h_cycles[e.pde_pos] + b->h_cycles[b->pde.size() + e.pde_pos];
        item_ms[k] = (double)cyc / b->clock_khz / (double)b->nslots;
      }
    }
  }
  if (total_ms) *total_ms = 1e-6 * (double)(b->h_stamp[1] - b->h_stamp[0]);
  if (worst == OUU_SAMPLE_NOT_CONVERGED) {
    ouu_set_error("some samples of a plain problem did not converge");
    return OUU_ERR_NOT_CONVERGED;
  }
  if (worst == OUU_SAMPLE_NONFINITE) {
    ouu_set_error("non-finite residual in some sample of a plain problem");
    return OUU_ERR_NONFINITE;
  }
  return OUU_OK;
}
