// C ABI: problem handle, argument checks, launches, host results.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "dino.cuh"
#include "ouu_internal.cuh"

static thread_local std::string g_last_error;

void ouu_set_error(const std::string& msg) { g_last_error = msg; }

cudaError_t ouu_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;   // (device, kernel) -> limit set so far
  int dev = 0;
  if (const cudaError_t e = cudaGetDevice(&dev)) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (cur >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

extern "C" size_t ouu_last_error(char* buf, size_t len) {
  if (buf && len > 0) {
    const size_t k = std::min(len - 1, g_last_error.size());
    std::memcpy(buf, g_last_error.data(), k);
    buf[k] = 0;
  }
  return g_last_error.size();
}

int ouu_num_levels(int n) {
  int l = 1;
  while (n > 3) {
    n = (n + 1) / 2;
    ++l;
  }
  return l;
}

static bool grid_ok(int n) {
  if (n < 5 || n > 1025) return false;
  const int m = n - 1;
  return (m & (m - 1)) == 0;
}

extern "C" void ouu_default_problem_desc(ouu_problem_desc* d) {
  if (!d) return;
  d->n = 129;
  d->reaction_r = 1.0;
  d->gamma = 0.1;
  d->delta = 1.0;
  d->m_mean = 0.0;
  d->lattice_L = 10;
  d->bump_width = 0.05;
  d->newton_rtol = 1e-10;
  d->newton_maxit = 30;
  d->cg_rtol = 1e-6;
  d->cg_maxit = 200;
  d->max_samples = 4096;
}

static SlotLayout make_layout(int n, int nlev, int L) {
  SlotLayout s;
  std::memset(&s, 0, sizeof(s));
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off += (bytes + 255) & ~int64_t(255);
    return o;
  };
  const int64_t nn = (int64_t)n * n;
  s.E = take(nn * 8);
  s.f = take(nn * 8);
  s.tmp = take((int64_t)std::max(L, 1) * n * 8);
  s.lam = take(nn * 8);
  s.acc = take((int64_t)OUU_MAX_RISKS * nn * 8);
  s.kx = take(nn * 4);
  s.ky = take(nn * 4);
  s.D = take(nn * 4);
  s.x = take(nn * 4);
  s.r = take(nn * 4);
  s.z = take(nn * 4);
  s.p = take(nn * 4);
  s.q = take(nn * 4);
  s.t = take(nn * 4);
  int nl = n;
  int64_t soff = 0;
  for (int l = 0; l < OUU_MAX_LEVELS; ++l) {
    s.lev[l] = -1;
    s.smem_lev[l] = -1;
  }
  for (int l = 0; l < nlev; ++l) {
    if (l > 0) {
      const int64_t blk = 6 * ouu_level_array_bytes(nl);
      if (nl <= OUU_SMEM_MAX_N) {
        s.smem_lev[l] = soff;
        soff += blk;
      } else {
        s.lev[l] = take(blk);
      }
    }
    nl = (nl + 1) / 2;
  }
  s.smem_bytes = soff;
  s.bytes = off;
  return s;
}

static ouu_status check_desc(const ouu_problem_desc* d) {
  OUU_CHECK_ARG(d != nullptr, "desc is null");
  OUU_CHECK_ARG(grid_ok(d->n), "n must be 2^k + 1 with 5 <= n <= 1025");
  OUU_CHECK_ARG(d->lattice_L >= 1 && d->lattice_L <= 64, "lattice_L must be in [1, 64]");
  OUU_CHECK_ARG(d->bump_width > 0 && std::isfinite(d->bump_width), "bump_width must be positive");
  OUU_CHECK_ARG(d->gamma > 0 && d->delta > 0, "gamma and delta must be positive");
  OUU_CHECK_ARG(d->reaction_r >= 0 && std::isfinite(d->reaction_r), "reaction_r must be >= 0");
  OUU_CHECK_ARG(std::isfinite(d->m_mean), "m_mean must be finite");
  OUU_CHECK_ARG(d->newton_rtol > 0 && d->newton_maxit >= 1, "bad Newton tolerance/cap");
  OUU_CHECK_ARG(d->cg_rtol > 0 && d->cg_rtol < 1 && d->cg_maxit >= 1, "bad CG tolerance/cap");
  OUU_CHECK_ARG(d->max_samples >= 1, "max_samples must be >= 1");
  return OUU_OK;
}

static void free_problem(ouu_problem* p) {
  if (!p) return;
  cudaFree(p->d_gx);
  cudaFree(p->d_gy);
  cudaFree(p->d_ut);
  cudaFree(p->d_V);
  cudaFree(p->d_invlam);
  cudaFree(p->d_slots);
  cudaFree(p->d_counter);
  cudaFree(p->d_u);
  cudaFree(p->d_q);
  cudaFree(p->d_status);
  cudaFree(p->d_iters);
  cudaFree(p->d_w);
  cudaFree(p->d_s);
  cudaFree(p->d_out);
  cudaFree(p->d_risks);
  cudaFree(p->d_z);
  cudaFree(p->d_rscr);
  cudaFreeHost(p->h_out);
  cudaFreeHost(p->h_stat);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
}

#define OUU_ALLOC(ptr, bytes)                                                           \
  do {                                                                                  \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                           \
      cudaGetLastError();                                                               \
      free_problem(p);                                                                  \
      ouu_set_error("cudaMalloc failed for " #ptr);                                     \
      return OUU_ERR_OOM;                                                               \
    }                                                                                   \
  } while (0)

extern "C" ouu_status ouu_create_problem(const ouu_problem_desc* desc, void* cuda_stream, ouu_problem_t* out) {
  OUU_CHECK_ARG(out != nullptr, "out is null");
  *out = nullptr;
  if (ouu_status st = check_desc(desc)) return st;
  ouu_problem* p = new ouu_problem();
  static std::atomic<uint64_t> next_serial{1};
  p->serial = next_serial++;
  p->desc = *desc;
  p->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    ouu_set_error("no CUDA device");
    return OUU_ERR_CUDA;
  }
  const int n = desc->n, L = desc->lattice_L;
  p->n = n;
  p->L = L;
  p->dz = L * L;
  p->nlev = ouu_num_levels(n);
  p->h = 1.0 / (n - 1);
  const double w = desc->bump_width;
  p->gscale = 1.0 / (w * std::sqrt(2.0 * M_PI));
  p->lay = make_layout(n, p->nlev, L);
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  if (p->lay.smem_bytes + 1024 > smem_optin) {
    delete p;
    ouu_set_error("multigrid shared-memory levels exceed the device limit");
    return OUU_ERR_INVALID_ARG;
  }
  if ((int64_t)L * n * (int64_t)sizeof(double) > smem_optin) {   // the G^T s reduction stages [L][n] in shared memory
    delete p;
    ouu_set_error("lattice_L * n too large for the gradient reduction's shared memory");
    return OUU_ERR_INVALID_ARG;
  }
  p->nslots = std::min(p->num_sms, desc->max_samples);
  const int64_t nn = (int64_t)n * n;
  const int64_t N = desc->max_samples;
  // host tables
  std::vector<double> gx((size_t)L * n), gy((size_t)L * n), ut(nn), V(nn), invlam(nn), mu(n);
  for (int j = 0; j < L; ++j) {
    const double c = (j + 0.5) / L;
    for (int i = 0; i < n; ++i) {
      const double x = i * p->h;
      const double g = std::exp(-((x - c) * (x - c)) / (2.0 * w * w));
      gx[(size_t)j * n + i] = g;
      gy[(size_t)j * n + i] = g;
    }
  }
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix)
      ut[(size_t)iy * n + ix] = std::sin(M_PI * (ix / (double)(n - 1))) * std::sin(M_PI * (iy / (double)(n - 1)));
  for (int k = 0; k < n; ++k) {
    const double s = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int j = 0; j < n; ++j) V[(size_t)k * n + j] = s * std::cos(M_PI * k * (j + 0.5) / n);
    const double sn = std::sin(M_PI * k / (2.0 * n));
    mu[k] = 4.0 * n * n * (sn * sn);
  }
  for (int k2 = 0; k2 < n; ++k2)
    for (int k1 = 0; k1 < n; ++k1)
      invlam[(size_t)k2 * n + k1] = 1.0 / (desc->delta + desc->gamma * (mu[k1] + mu[k2]));
  OUU_ALLOC(p->d_gx, gx.size() * 8);
  OUU_ALLOC(p->d_gy, gy.size() * 8);
  OUU_ALLOC(p->d_ut, nn * 8);
  OUU_ALLOC(p->d_V, nn * 8);
  OUU_ALLOC(p->d_invlam, nn * 8);
  OUU_ALLOC(p->d_slots, (size_t)p->lay.bytes * p->nslots);
  OUU_ALLOC(p->d_counter, 64);
  OUU_ALLOC(p->d_u, (size_t)N * nn * 8);
  OUU_ALLOC(p->d_q, (size_t)N * 8);
  OUU_ALLOC(p->d_status, (size_t)N * 4);
  OUU_ALLOC(p->d_iters, (size_t)N * 3 * 4);
  OUU_ALLOC(p->d_w, (size_t)OUU_MAX_RISKS * N * 8);
  OUU_ALLOC(p->d_s, (size_t)OUU_MAX_RISKS * nn * 8);
  OUU_ALLOC(p->d_out, (size_t)(OUU_MAX_RISKS * (3 + p->dz) + 8) * 8);
  OUU_ALLOC(p->d_risks, sizeof(RiskDev) * OUU_MAX_RISKS);
  OUU_ALLOC(p->d_z, (size_t)p->dz * 8);
  OUU_ALLOC(p->d_rscr, (size_t)OUU_RISK_SCRATCH * 8);
  OUU_CUDA_TRY(cudaMemset(p->d_rscr, 0, (size_t)OUU_RISK_SCRATCH * 8));
  if (cudaMallocHost((void**)&p->h_out, (size_t)(OUU_MAX_RISKS * (3 + p->dz) + 8) * 8) != cudaSuccess ||
      cudaMallocHost((void**)&p->h_stat, (size_t)N * 4 * 4 + 64) != cudaSuccess) {
    cudaGetLastError();
    free_problem(p);
    ouu_set_error("cudaMallocHost failed");
    return OUU_ERR_OOM;
  }
  OUU_CUDA_TRY(cudaMemcpy(p->d_gx, gx.data(), gx.size() * 8, cudaMemcpyHostToDevice));
  OUU_CUDA_TRY(cudaMemcpy(p->d_gy, gy.data(), gy.size() * 8, cudaMemcpyHostToDevice));
  OUU_CUDA_TRY(cudaMemcpy(p->d_ut, ut.data(), nn * 8, cudaMemcpyHostToDevice));
  OUU_CUDA_TRY(cudaMemcpy(p->d_V, V.data(), nn * 8, cudaMemcpyHostToDevice));
  OUU_CUDA_TRY(cudaMemcpy(p->d_invlam, invlam.data(), nn * 8, cudaMemcpyHostToDevice));
  OUU_CUDA_TRY(cudaMemset(p->d_slots, 0, (size_t)p->lay.bytes * p->nslots));
  OUU_CUDA_TRY(cudaMemset(p->d_u, 0, (size_t)N * nn * 8));
  for (auto& e : p->ev) OUU_CUDA_TRY(cudaEventCreate(&e));
  OUU_CUDA_TRY(cudaDeviceSynchronize());
  *out = p;
  return OUU_OK;
}

extern "C" ouu_status ouu_destroy_problem(ouu_problem_t p) {
  if (!p) return OUU_OK;
  cudaStreamSynchronize(p->stream);
  free_problem(p);
  return OUU_OK;
}

extern "C" int ouu_problem_slots(ouu_problem_t p) { return p ? p->nslots : 0; }

extern "C" ouu_status ouu_sample_fields(ouu_problem_t p, uint64_t seed, int64_t first_index, int n_samples,
                                        double* m_dev) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(n_samples >= 0 && first_index >= 0, "negative sample range");
  if (n_samples == 0) return OUU_OK;
  OUU_CHECK_ARG(m_dev != nullptr, "m_dev is null");
  OUU_CHECK_ARG(n_samples <= 65535, "at most 65535 samples per call");
  launch_sample_fields(p->n, seed, first_index, n_samples, p->d_invlam, p->d_V, p->desc.m_mean, m_dev, p->stream);
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

PdeArgs ouu_base_args(ouu_problem* p, int n_samples) {
  PdeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = p->n;
  a.nlev = p->nlev;
  a.L = p->L;
  a.n_samples = n_samples;
  a.rr = p->desc.reaction_r;
  a.gscale = p->gscale;
  a.newton_rtol = p->desc.newton_rtol;
  a.newton_maxit = p->desc.newton_maxit;
  a.cg_rtol = p->desc.cg_rtol;
  a.cg_maxit = p->desc.cg_maxit;
  a.refine_rtol = 1e-12;
  a.refine_maxit = 12;
  a.gx = p->d_gx;
  a.gy = p->d_gy;
  a.ut = p->d_ut;
  a.slots = p->d_slots;
  a.lay = p->lay;
  a.counter = p->d_counter;
  a.status = p->d_status;
  a.iters = p->d_iters;
  return a;
}

static int solver_grid(ouu_problem* p, int n_samples) { return std::max(1, std::min(p->nslots, n_samples)); }

// Reads back per-sample statuses and turns them into a call status.
static ouu_status check_statuses(ouu_problem* p, int n_samples) {
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat, p->d_status, (size_t)n_samples * 4, cudaMemcpyDeviceToHost, p->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(p->stream));
  int worst = 0, bad = -1;
  for (int i = 0; i < n_samples; ++i)
    if (p->h_stat[i] > worst) {
      worst = p->h_stat[i];
      bad = i;
    }
  if (worst == OUU_SAMPLE_NOT_CONVERGED) {
    ouu_set_error("sample " + std::to_string(bad) + " did not converge");
    return OUU_ERR_NOT_CONVERGED;
  }
  if (worst == OUU_SAMPLE_NONFINITE) {
    ouu_set_error("non-finite residual in sample " + std::to_string(bad));
    return OUU_ERR_NONFINITE;
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_pde_solve_batch(ouu_problem_t p, const double* m_dev, int n_samples, const double* z_dev,
                                          int64_t z_stride, double* u_dev, double* q_dev, int32_t* status_dev) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(n_samples >= 0 && n_samples <= p->desc.max_samples, "n_samples outside [0, max_samples]");
  if (n_samples == 0) return OUU_OK;
  OUU_CHECK_ARG(m_dev && z_dev && q_dev, "m_dev, z_dev and q_dev are required");
  OUU_CHECK_ARG(z_stride == 0 || z_stride >= p->dz, "z_stride must be 0 or >= d_Z");
  PdeArgs a = ouu_base_args(p, n_samples);
  a.m = m_dev;
  a.z = z_dev;
  a.z_stride = z_stride;
  a.u = u_dev ? u_dev : p->d_u;
  a.q = q_dev;
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
  launch_pde_state(a, solver_grid(p, n_samples), p->stream);
  OUU_CUDA_TRY(cudaGetLastError());
  if (status_dev)
    OUU_CUDA_TRY(cudaMemcpyAsync(status_dev, p->d_status, (size_t)n_samples * 4, cudaMemcpyDeviceToDevice,
                                 p->stream));
  return check_statuses(p, n_samples);
}

extern "C" ouu_status ouu_adjoint_batch(ouu_problem_t p, const double* m_dev, const double* u_dev, int n_samples,
                                        double* lambda_dev, double* gradq_dev) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(n_samples >= 0 && n_samples <= p->desc.max_samples, "n_samples outside [0, max_samples]");
  if (n_samples == 0 || (!lambda_dev && !gradq_dev)) return OUU_OK;
  OUU_CHECK_ARG(m_dev && u_dev, "m_dev and u_dev are required");
  PdeArgs a = ouu_base_args(p, n_samples);
  a.m = m_dev;
  a.u = const_cast<double*>(u_dev);
  a.lam_out = lambda_dev;
  a.grad_out = gradq_dev;
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, (size_t)n_samples * 4, p->stream));
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_iters, 0, (size_t)n_samples * 12, p->stream));
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
  launch_pde_adjoint(a, solver_grid(p, n_samples), p->stream);
  OUU_CUDA_TRY(cudaGetLastError());
  return check_statuses(p, n_samples);
}

ouu_status ouu_check_risks(const ouu_risk_desc* risks, int n_risks) {
  OUU_CHECK_ARG(risks != nullptr && n_risks >= 1 && n_risks <= OUU_MAX_RISKS, "need 1..4 risk descriptors");
  for (int r = 0; r < n_risks; ++r) {
    const ouu_risk_desc& R = risks[r];
    OUU_CHECK_ARG(R.kind == OUU_RISK_MEAN_VAR || R.kind == OUU_RISK_CVAR_SMOOTH, "unknown risk kind");
    if (R.kind == OUU_RISK_MEAN_VAR) OUU_CHECK_ARG(std::isfinite(R.kappa), "kappa must be finite");
    else {
      OUU_CHECK_ARG(R.beta >= 0 && R.beta < 1, "beta must be in [0, 1)");
      OUU_CHECK_ARG(R.eps > 0 && std::isfinite(R.eps), "eps must be positive");
      OUU_CHECK_ARG(std::isfinite(R.t), "t must be finite");
    }
  }
  return OUU_OK;
}

void ouu_risk_dev(const ouu_risk_desc* risks, int n_risks, int N, RiskDev* rd) {
  std::memset(rd, 0, sizeof(RiskDev) * OUU_MAX_RISKS);   // padding too: descriptors are compared bytewise
  for (int r = 0; r < n_risks; ++r) {
    rd[r].kind = risks[r].kind;
    rd[r].kappa = risks[r].kappa;
    rd[r].beta = risks[r].beta;
    rd[r].eps = risks[r].eps;
    rd[r].t = risks[r].t;
    rd[r].t_optimal = risks[r].t_optimal;
    risk_dev_finish(rd[r], N);
  }
}

ouu_status ouu_upload_risks(ouu_problem* p, const RiskDev* rd, int n_risks, cudaStream_t us) {
  if (n_risks != p->rd_n || us != p->rd_stream || std::memcmp(rd, p->rd_last, sizeof(RiskDev) * n_risks) != 0) {
    p->rd_n = -1;   // stays invalid if the upload fails
    OUU_CUDA_TRY(cudaMemcpyAsync(p->d_risks, rd, sizeof(RiskDev) * n_risks, cudaMemcpyHostToDevice, us));
    std::memcpy(p->rd_last, rd, sizeof(RiskDev) * n_risks);
    p->rd_n = n_risks;
    p->rd_stream = us;
  }
  return OUU_OK;
}

// The MR-DINO risk evaluation as one stream-ordered sequence on dino->stream: projection +
// network + reduced QoI + reverse-mode gradient, risk weights with the weighted gradient
// sum, results (and the GEMM error flag) to the problem's pinned host mirror.  The risk
// descriptors must already be in p->d_risks.
ouu_status dino_enqueue_risk(ouu_problem* p, ouu_dino* dino, const double* m_dev, int n_samples, int n_risks,
                             const double* z_host) {
  const int dz = p->dz;
  double* d_res = p->d_out;
  double* d_grad = p->d_out + 3 * OUU_MAX_RISKS;
  const size_t ob = (size_t)(OUU_MAX_RISKS * (3 + dz) + 8) * 8;
  bool split = false;
  if (ouu_status st = dino_eval_forward(dino, m_dev, n_samples, z_host, &split)) return st;
  if (split) {
    // Q is complete: the moments and t* (which read only Q) on the side stream, beside the
    // network's reverse mode on the main one; joined before the weighted sums
    OUU_CUDA_TRY(cudaEventRecord(dino->ev_fork, dino->stream));
    OUU_CUDA_TRY(cudaStreamWaitEvent(dino->side, dino->ev_fork, 0));
    // (the moments from the forward launch's per-tile sums)
    launch_risk_select(dino->Qe, n_samples, p->d_risks, n_risks, d_res, p->d_rscr, dino->side, d_grad, n_risks * dz,
                       dino->Qmom, (n_samples + 127) / 128);
    OUU_CUDA_TRY(cudaEventRecord(dino->ev_join, dino->side));
    if (ouu_status st = dino_eval_reverse(dino, n_samples)) return st;
    OUU_CUDA_TRY(cudaStreamWaitEvent(dino->stream, dino->ev_join, 0));
  }
  if (!dino->capturing) OUU_CUDA_TRY(cudaEventRecord(p->ev[1], dino->stream));
  // weights, risk values and sum_i w_i grad Q_i in one pass over the samples
  if (split)
    launch_risk_apply(dino->Qe, n_samples, p->d_risks, n_risks, p->d_w, p->d_rscr, dino->stream, dino->GQe,
                      (dz + 7) / 8 * 8, dz, d_grad, 0, -1, dino->d_err, p->d_out + OUU_OUT_FLAG(dz));
  else
    launch_risk_weights(dino->Qe, n_samples, p->d_risks, n_risks, p->d_w, d_res, p->d_rscr, dino->stream,
                        dino->GQe, (dz + 7) / 8 * 8, dz, d_grad, 0, -1, dino->d_err, p->d_out + OUU_OUT_FLAG(dz));
  if (!dino->capturing) OUU_CUDA_TRY(cudaEventRecord(p->ev[2], dino->stream));
  OUU_CUDA_TRY(cudaGetLastError());
  // one read-back: the results and (in them) the network's status flag
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_out, p->d_out, ob, cudaMemcpyDeviceToHost, dino->stream));
  return OUU_OK;
}

// One risk evaluation on the given backend (OUU_BACKEND_PDE or OUU_BACKEND_DINO).
static ouu_status risk_and_grad_on(ouu_problem_t p, ouu_backend backend, ouu_dino_t dino, const double* m_dev,
                                   int n_samples, const ouu_risk_desc* risks, int n_risks, const double* z_host,
                                   double* risk_out, double* grad_z_out, double* grad_t_out, double* t_out,
                                   ouu_eval_stats* stats) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(n_samples >= 1 && n_samples <= p->desc.max_samples, "n_samples outside [1, max_samples]");
  OUU_CHECK_ARG(m_dev && z_host && risk_out && grad_z_out && grad_t_out, "null argument");
  if (ouu_status st = ouu_check_risks(risks, n_risks)) return st;
  for (int j = 0; j < p->dz; ++j) OUU_CHECK_ARG(std::isfinite(z_host[j]), "z has a non-finite entry");
  RiskDev rd[OUU_MAX_RISKS];
  ouu_risk_dev(risks, n_risks, n_samples, rd);
  const int dz = p->dz;
  double* d_res = p->d_out;                         // [n_risks][3]
  double* d_grad = p->d_out + 3 * OUU_MAX_RISKS;    // [n_risks][dz]
  int* d_solved = (int*)(p->d_out + OUU_MAX_RISKS * (3 + dz));
  if (backend == OUU_BACKEND_DINO) {
    OUU_CHECK_ARG(dino != nullptr, "DINO backend needs a trained network");
    OUU_CHECK_ARG(dino->n == p->n && dino->dz == p->dz, "problem and network grids differ");
    OUU_CHECK_ARG(n_samples <= dino->maxE, "n_samples exceeds the network's max_eval");
    if (!dino->bases_ready) {
      ouu_set_error("network bases not built");
      return OUU_ERR_STATE;
    }
  }
  // The risk descriptors go up on the stream that reads them, and only when they differ from
  // the last ones sent there (every call ends synchronised, so an upload on the same stream
  // has been performed).  z: the plain path reads it from d_z (staged in the pinned h_out,
  // which the results overwrite only later in the same stream); the MR-DINO evaluation copies
  // it itself.  No synchronisation before the work is enqueued.
  cudaStream_t us = backend == OUU_BACKEND_DINO ? dino->stream : p->stream;
  if (ouu_status st = ouu_upload_risks(p, rd, n_risks, us)) return st;
  if (backend != OUU_BACKEND_DINO) {
    std::memcpy(p->h_out, z_host, (size_t)dz * 8);
    OUU_CUDA_TRY(cudaMemcpyAsync(p->d_z, p->h_out, (size_t)dz * 8, cudaMemcpyHostToDevice, p->stream));
  }
  if (backend == OUU_BACKEND_DINO) {
    cudaStream_t ds = dino->stream;
    ++dino->eval_count;   // a graph replay, too, overwrites the network's per-sample buffers
    auto enqueue = [&]() -> ouu_status { return dino_enqueue_risk(p, dino, m_dev, n_samples, n_risks, z_host); };
    const bool replay = dino->use_graphs && dino->gexec && dino->gkey_p == p && dino->gkey_m == m_dev &&
                        dino->gkey_N == n_samples && dino->gkey_nr == n_risks;
    OUU_CUDA_TRY(cudaEventRecord(p->ev[0], ds));
    if (replay) {
      float* zh = (float*)dino->h_pin;   // the graph's copy node reads z from here
      for (int j = 0; j < dz; ++j) zh[j] = (float)z_host[j];
      OUU_CUDA_TRY(cudaGraphLaunch(dino->gexec, ds));
    } else {
      if (ouu_status st = enqueue()) return st;
      if (dino->use_graphs) {
        // capture the same sequence for the next calls with this (problem, fields, N, risks)
        if (dino->gexec) {
          cudaGraphExecDestroy(dino->gexec);
          dino->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        dino->capturing = true;
        dino->stream = dino->cap;
        ouu_status cst = OUU_OK;
        if (cudaStreamBeginCapture(dino->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          cst = enqueue();
          if (cudaStreamEndCapture(dino->cap, &g) != cudaSuccess) g = nullptr;
        }
        dino->stream = ds;
        dino->capturing = false;
        cudaGetLastError();
        if (cst == OUU_OK && g) {
          cudaGraphExec_t ex = nullptr;
          if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
            dino->gexec = ex;
            dino->gkey_p = p;
            dino->gkey_m = m_dev;
            dino->gkey_N = n_samples;
            dino->gkey_nr = n_risks;
          }
          cudaGetLastError();
        }
        if (g) cudaGraphDestroy(g);
      }
    }
    OUU_CUDA_TRY(cudaEventRecord(p->ev[3], ds));
    OUU_CUDA_TRY(cudaStreamSynchronize(ds));
    if (p->h_out[OUU_OUT_FLAG(dz)] != 0.0) {
      cudaMemsetAsync(dino->d_err, 0, 4, ds);
      // an interrupted projection may have left its tile counters non-zero
      cudaMemsetAsync(dino->d_klp_ctr, 0, (OUU_KLP_MAX_TILES + 1) * sizeof(int), ds);
      ouu_set_error("tensor-core GEMM pipeline wait timed out");
      return OUU_ERR_CUDA;
    }
    for (int r = 0; r < n_risks; ++r) {
      risk_out[r] = p->h_out[3 * r + 0];
      grad_t_out[r] = p->h_out[3 * r + 1];
      if (t_out) t_out[r] = p->h_out[3 * r + 2];
      std::memcpy(grad_z_out + (size_t)r * dz, p->h_out + 3 * OUU_MAX_RISKS + (size_t)r * dz, (size_t)dz * 8);
    }
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      cudaEventElapsedTime(&stats->ms_total, p->ev[0], p->ev[3]);
      // the projection's marks are event nodes of the graph too
      if (replay && dino->graph_marks) cudaEventElapsedTime(&stats->ms_project, dino->ev[0], dino->ev[2]);
      if (!replay) {   // the other phase marks exist only for an eagerly enqueued evaluation
        cudaEventElapsedTime(&stats->ms_state, p->ev[0], p->ev[1]);
        cudaEventElapsedTime(&stats->ms_weights, p->ev[1], p->ev[2]);
        cudaEventElapsedTime(&stats->ms_reduce, p->ev[2], p->ev[3]);
        cudaEventElapsedTime(&stats->ms_project, dino->ev[0], dino->ev[2]);
        cudaEventElapsedTime(&stats->ms_network, dino->ev[2], dino->ev[3]);
      }
    }
    return OUU_OK;
  }
  OUU_CHECK_ARG(backend == OUU_BACKEND_PDE, "unknown backend");
  PdeArgs a = ouu_base_args(p, n_samples);
  a.m = m_dev;
  a.z = p->d_z;
  a.z_stride = 0;
  a.u = p->d_u;
  a.q = p->d_q;
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
  OUU_CUDA_TRY(cudaMemsetAsync(d_solved, 0, 4, p->stream));
  OUU_CUDA_TRY(cudaEventRecord(p->ev[0], p->stream));
  launch_pde_state(a, solver_grid(p, n_samples), p->stream);
  OUU_CUDA_TRY(cudaEventRecord(p->ev[1], p->stream));
  launch_risk_weights(p->d_q, n_samples, p->d_risks, n_risks, p->d_w, d_res, p->d_rscr, p->stream);
  OUU_CUDA_TRY(cudaEventRecord(p->ev[2], p->stream));
  a.w = p->d_w;
  a.n_w = n_risks;
  a.solved = d_solved;
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
  launch_pde_adjoint(a, solver_grid(p, n_samples), p->stream);
  OUU_CUDA_TRY(cudaEventRecord(p->ev[3], p->stream));
  launch_reduce_slots_and_gradient(p->d_slots, p->lay, solver_grid(p, n_samples), p->n, p->L, n_risks, p->d_gx,
                                   p->d_gy, p->gscale, p->d_s, d_grad, p->stream);
  OUU_CUDA_TRY(cudaEventRecord(p->ev[4], p->stream));
  OUU_CUDA_TRY(cudaGetLastError());
  const size_t out_bytes = (size_t)(OUU_MAX_RISKS * (3 + dz) + 8) * 8;
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_out, p->d_out, out_bytes, cudaMemcpyDeviceToHost, p->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat, p->d_status, (size_t)n_samples * 4, cudaMemcpyDeviceToHost, p->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(p->h_stat + n_samples, p->d_iters, (size_t)n_samples * 12, cudaMemcpyDeviceToHost,
                               p->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(p->stream));
  for (int r = 0; r < n_risks; ++r) {
    risk_out[r] = p->h_out[3 * r + 0];
    grad_t_out[r] = p->h_out[3 * r + 1];
    if (t_out) t_out[r] = p->h_out[3 * r + 2];
    std::memcpy(grad_z_out + (size_t)r * dz, p->h_out + 3 * OUU_MAX_RISKS + (size_t)r * dz, (size_t)dz * 8);
  }
  int worst = 0, nbad = 0;
  const int32_t* it = p->h_stat + n_samples;
  if (stats) {
    stats->newton_min = 1 << 30;
    stats->newton_max = 0;
    stats->newton_mean = 0;
    stats->cg_total = 0;
  }
  for (int i = 0; i < n_samples; ++i) {
    worst = std::max(worst, (int)p->h_stat[i]);
    nbad += p->h_stat[i] != 0;
    if (stats) {
      stats->newton_min = std::min(stats->newton_min, (int)it[3 * i]);
      stats->newton_max = std::max(stats->newton_max, (int)it[3 * i]);
      stats->newton_mean += it[3 * i];
      stats->cg_total += it[3 * i + 1];
    }
  }
  if (stats) {
    cudaEventElapsedTime(&stats->ms_state, p->ev[0], p->ev[1]);
    cudaEventElapsedTime(&stats->ms_weights, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&stats->ms_adjoint, p->ev[2], p->ev[3]);
    cudaEventElapsedTime(&stats->ms_reduce, p->ev[3], p->ev[4]);
    cudaEventElapsedTime(&stats->ms_total, p->ev[0], p->ev[4]);
    stats->newton_mean /= n_samples;
    stats->adjoint_solves = *(const int*)(p->h_out + OUU_MAX_RISKS * (3 + dz));
    stats->n_not_converged = nbad;
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

// The network may stand in for the plain path: it passed its held-out check against this
// problem and can take this many samples.
bool dino_trusted(const ouu_dino* d, const ouu_problem* p, int n_samples) {
  return d && p && d->val_ok && d->val_serial == p->serial && d->bases_ready && n_samples <= d->maxE;
}

extern "C" ouu_status ouu_risk_and_grad(ouu_problem_t p, ouu_backend backend, ouu_dino_t dino, const double* m_dev,
                                        int n_samples, const ouu_risk_desc* risks, int n_risks, const double* z_host,
                                        double* risk_out, double* grad_z_out, double* grad_t_out, double* t_out,
                                        ouu_eval_stats* stats) {
  OUU_CHECK_ARG(p != nullptr, "problem is null");
  OUU_CHECK_ARG(backend == OUU_BACKEND_PDE || backend == OUU_BACKEND_DINO || backend == OUU_BACKEND_AUTO,
                "unknown backend");
  if (backend == OUU_BACKEND_AUTO)
    backend = dino_trusted(dino, p, n_samples) ? OUU_BACKEND_DINO : OUU_BACKEND_PDE;
  const ouu_status st = risk_and_grad_on(p, backend, dino, m_dev, n_samples, risks, n_risks, z_host, risk_out,
                                         grad_z_out, grad_t_out, t_out, stats);
  if (st == OUU_OK) p->last_backend = backend;
  return st;
}

extern "C" int ouu_last_backend(ouu_problem_t p) { return p ? p->last_backend : -1; }

// Relative error |a - b| / |b| (0 when both are zero; NaN stays NaN).
static double rel_err(double a, double b) {
  const double d = std::fabs(a - b), s = std::fabs(b);
  return s > 0 ? d / s : (d == 0 ? 0.0 : INFINITY);
}

extern "C" ouu_status ouu_dino_validate(ouu_problem_t p, ouu_dino_t d, const double* m_dev, int n_samples,
                                        const ouu_risk_desc* risks, int n_risks, const double* z_host, int n_z,
                                        double risk_tol, double grad_tol, double* risk_err_out, double* grad_err_out,
                                        int* passed_out) {
  OUU_CHECK_ARG(p && d && m_dev && z_host, "null argument");
  OUU_CHECK_ARG(n_z >= 1, "need at least one control");
  OUU_CHECK_ARG(std::isfinite(risk_tol) && std::isfinite(grad_tol) && risk_tol >= 0 && grad_tol >= 0,
                "tolerances must be finite and >= 0");
  OUU_CHECK_ARG(n_risks >= 1 && n_risks <= OUU_MAX_RISKS, "need 1..4 risk descriptors");
  d->val_ok = 0;   // a check that fails or stops part-way leaves the network untrusted
  const int dz = p->dz;
  std::vector<double> r0(n_risks), r1(n_risks), g0((size_t)n_risks * dz), g1((size_t)n_risks * dz),
      t0(n_risks), t1(n_risks);
  double er = 0.0, eg = 0.0;
  for (int k = 0; k < n_z; ++k) {
    const double* z = z_host + (size_t)k * dz;
    if (ouu_status st = risk_and_grad_on(p, OUU_BACKEND_PDE, nullptr, m_dev, n_samples, risks, n_risks, z,
                                         r0.data(), g0.data(), t0.data(), nullptr, nullptr))
      return st;
    if (ouu_status st = risk_and_grad_on(p, OUU_BACKEND_DINO, d, m_dev, n_samples, risks, n_risks, z, r1.data(),
                                         g1.data(), t1.data(), nullptr, nullptr))
      return st;
    for (int r = 0; r < n_risks; ++r) {
      const double e = rel_err(r1[r], r0[r]);
      if (!(e <= er)) er = e;   // a NaN error sticks
      double dd = 0.0, nn = 0.0;
      for (int j = 0; j < dz; ++j) {
        const double a = g1[(size_t)r * dz + j], b = g0[(size_t)r * dz + j];
        dd += (a - b) * (a - b);
        nn += b * b;
      }
      const double eg_r = nn > 0 ? std::sqrt(dd / nn) : (dd == 0 ? 0.0 : INFINITY);
      if (!(eg_r <= eg)) eg = eg_r;
    }
  }
  const bool passed = er <= risk_tol && eg <= grad_tol;
  if (passed) {
    d->val_ok = 1;
    d->val_serial = p->serial;
  }
  if (risk_err_out) *risk_err_out = er;
  if (grad_err_out) *grad_err_out = eg;
  if (passed_out) *passed_out = passed ? 1 : 0;
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_jacobian_data(ouu_problem_t p, ouu_dino_t d, const double* m_dev, const double* u_dev,
                                             int n_samples, float* jy_dev) {
  OUU_CHECK_ARG(p && d && m_dev && u_dev && jy_dev, "null argument");
  OUU_CHECK_ARG(p->n == d->n && p->dz == d->dz, "problem and network grids differ");
  OUU_CHECK_ARG(n_samples >= 0 && n_samples <= p->desc.max_samples, "n_samples outside [0, max_samples]");
  if (!d->bases_ready) {
    ouu_set_error("network bases not built");
    return OUU_ERR_STATE;
  }
  if (n_samples == 0) return OUU_OK;
  PdeArgs a = ouu_base_args(p, n_samples);
  a.m = m_dev;
  a.u = const_cast<double*>(u_dev);
  OUU_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, 4, p->stream));
  // Sec. 3.4: the forward route takes d_Z linearised solves per sample, the adjoint route r_u
  const int route = d->jac_route == 1 ? 0 : d->jac_route == 2 ? 1 : (d->dz <= d->ru ? 0 : 1);
  launch_pde_jacobian_data(a, solver_grid(p, n_samples), d->d_phi, d->ru, jy_dev, route, p->stream);
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_set_jacobian_route(ouu_dino_t d, int route) {
  OUU_CHECK_ARG(d != nullptr, "null argument");
  OUU_CHECK_ARG(route >= 0 && route <= 2, "route: 0 the cheaper, 1 forward, 2 adjoint");
  d->jac_route = route;
  return OUU_OK;
}
