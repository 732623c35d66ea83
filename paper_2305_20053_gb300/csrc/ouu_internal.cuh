// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "ouu.h"
#include "pde_core.cuh"

// ------------------------------------------------------------------ errors
void ouu_set_error(const std::string& msg);

// Raises kernel fn's dynamic shared memory limit to at least `bytes` (never lowers it), under
// one lock, so that launches of the same kernel with different sizes from concurrent handles
// cannot undo each other's limit.  Kept per device (the current one).
cudaError_t ouu_smem_limit(const void* fn, size_t bytes);

// Checks 1..OUU_MAX_RISKS risk descriptors (known kind; finite kappa; beta in [0, 1), eps > 0
// and finite t for the smoothed CVaR); INVALID_ARG with a message otherwise.
ouu_status ouu_check_risks(const ouu_risk_desc* risks, int n_risks);

// ------------------------------------------------------------------ programmatic dependent launch
// Kernels launched with launch_pdl may start while the previous kernel in the stream drains
// (their set-up overlaps its tail); each calls pdl_wait() before it reads or writes global
// memory that earlier kernels touch.  No kernel triggers its dependents early, so a kernel's
// completion still implies the completion of every kernel before it.
static __device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define OUU_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ouu_set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));               \
      return OUU_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define OUU_CHECK_ARG(cond, msg)                                                        \
  do {                                                                                  \
    if (!(cond)) {                                                                      \
      ouu_set_error(msg);                                                               \
      return OUU_ERR_INVALID_ARG;                                                       \
    }                                                                                   \
  } while (0)

// ------------------------------------------------------------------ CTA context
// One CTA cooperates on one sample: warps own grid rows, lanes own columns.
struct CtaCtx {
  double* red;   // shared scratch of >= 33 doubles
  __device__ __forceinline__ int row0() const { return threadIdx.x >> 5; }
  __device__ __forceinline__ int rowstep() const { return blockDim.x >> 5; }
  __device__ __forceinline__ int col0() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int colstep() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ double sum_d(double v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
      double s = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
  }
  // FP32 partial sums per thread and per warp, FP64 across warps.
  __device__ double sum_f(float v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = (double)v;
    __syncthreads();
    if (w == 0) {
      double s = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
  }
};

// ------------------------------------------------------------------ solver launch data
#define OUU_SMEM_MAX_N 65      // multigrid levels with n_l <= this live in shared memory
#define OUU_SOLVER_THREADS 1024
#define OUU_MAX_RISKS 4

// Bytes of one array of a multigrid level (n x n floats, padded to 16 bytes).
__host__ __device__ inline int64_t ouu_level_array_bytes(int n) {
  return (((int64_t)n * n * 4 + 15) / 16) * 16;
}

struct SlotLayout {
  int64_t bytes;                         // bytes per slot
  int64_t E, f, tmp, lam, acc;           // FP64 arrays (offsets in bytes)
  int64_t kx, ky, D, x, r, z, p, q, t;   // level-0 FP32 arrays
  int64_t lev[OUU_MAX_LEVELS];           // global coarse level blocks (6 arrays), -1 if in smem
  int64_t smem_lev[OUU_MAX_LEVELS];      // shared-memory offsets of smem levels, -1 if global
  int64_t smem_bytes;
};

struct PdeArgs {
  int n, nlev, L, n_samples;
  double rr, gscale, newton_rtol, cg_rtol, refine_rtol;
  int newton_maxit, cg_maxit, refine_maxit;
  const double* m;            // [N][n*n]
  const double* z;            // z for sample i at z + i * z_stride
  int64_t z_stride;
  const double* gx;           // [L][n]
  const double* gy;           // [L][n]
  const double* ut;           // [n*n]
  double* u;                  // [N][n*n]: output of the state kernel, input of the adjoint kernel
  double* q;                  // [N]
  int32_t* status;            // [N]
  int32_t* iters;             // [N][3]: newton steps, cg iterations, refinement steps
  int* solved;                // adjoint kernel: count of samples solved (may be null)
  // adjoint kernel
  const double* w;            // [n_w][N] risk weights (null: per-sample outputs only)
  int n_w;
  double* lam_out;            // [N][n*n] or null
  double* grad_out;           // [N][L*L] or null
  char* slots;
  SlotLayout lay;
  int* counter;
  double* acc_out;            // batch adjoint: [n_w][n*n] sums the slots are flushed into
};

struct ouu_problem;
PdeArgs ouu_base_args(ouu_problem* p, int n_samples);
void launch_pde_state(const PdeArgs& a, int nslots, cudaStream_t s);
// One persistent launch over tasks (problem, sample) of many problems (probs_dev: device
// array of per-problem arguments; tasks_dev: device int2 array).  adjoint: adjoint solves
// with weighted sums flushed into probs[p].acc_out (zeroed beforehand); else state solves.
void launch_pde_batch(const PdeArgs* probs_dev, const int2* tasks_dev, int n_tasks, char* slots, int64_t slot_bytes,
                      int64_t smem_bytes, int nslots, int* counter, unsigned long long* cycles, bool adjoint,
                      cudaStream_t s);
void launch_pde_adjoint(const PdeArgs& a, int nslots, cudaStream_t s);

// Sum the per-slot FP64 accumulators [slot][n_w][n*n] into s_out [n_w][n*n], then
// grad[r][j] = scale * sum_{iy,ix} gy[jy][iy] gx[jx][ix] s[r][iy*n+ix].
// grad[r][j] = gscale * sum_{iy,ix} gy[jy][iy] gx[jx][ix] s[r][iy*n+ix] for r < n_w.
void launch_sources_transpose(int n, int L, int n_w, const double* gx, const double* gy, double gscale,
                              const double* s, double* grad, cudaStream_t st);
void launch_reduce_slots_and_gradient(const char* slots, const SlotLayout& lay, int nslots, int n, int L,
                                      int n_w, const double* gx, const double* gy, double gscale,
                                      double* s_out, double* grad, cudaStream_t st);

// ------------------------------------------------------------------ risk weights
struct RiskDev {
  int kind;
  double kappa, beta, eps, t;
  int t_optimal;
  // set on the host for the call's N (risk_dev_finish), so that no device thread divides in
  // FP64: K = N (1 - beta), the rank kq = floor(K) + 1 (clamped to [1, N]) of the sample that
  // opens the CVaR window, 1 / eps, 1 / K and 1 / N
  double K, inv_eps, inv_K, inv_N;
  int kq;
};

inline void risk_dev_finish(RiskDev& r, int N) {
  r.K = (double)N * (1.0 - r.beta);
  int kq = (int)(r.K) + 1;   // floor for K >= 0
  r.kq = kq > N ? N : (kq < 1 ? 1 : kq);
  r.inv_eps = r.eps > 0.0 ? 1.0 / r.eps : 0.0;
  r.inv_K = r.K > 0.0 ? 1.0 / r.K : 0.0;
  r.inv_N = 1.0 / (double)N;
}

// Per-risk weights w[r][i], value[r], dt[r], t[r] from q[N] (moments on many CTAs, t*
// selection on one, weights on many).  out layout: value[r], dt[r], t[r] at out[3r+0..2].
// With per-sample gradients gq [N][ldg] (FP32), also grad_out[r][j] = sum_i w[r][i] gq[i][j].
// A window (wfirst, wcount >= 0) restricts the weights written and the gradient sum to the
// samples [wfirst, wfirst + wcount): w then holds [n_risks][wcount] and gq has wcount rows
// (one rank's block of a sample set spread over ranks); the risk values, t and d rho / dt
// still come from all N QoIs.  wcount < 0: the whole set.
// scratch: OUU_RISK_SCRATCH doubles of device memory.
#define OUU_RISK_SCRATCH 2048
// The results block d_out of a problem: [OUU_MAX_RISKS][3] values, [OUU_MAX_RISKS][d_Z] gradients,
// then 8 doubles: the plain path's solved-sample count (an int) and the network's status flag.
#define OUU_OUT_FLAG(dz) (OUU_MAX_RISKS * (3 + (dz)) + 1)
void launch_risk_weights(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* out,
                         double* scratch, cudaStream_t s, const float* gq = nullptr, int ldg = 0, int dz = 0,
                         double* grad_out = nullptr, int wfirst = 0, int wcount = -1,
                         const int* flag_src = nullptr, double* flag_dst = nullptr);
// launch_risk_weights as its two stream-ordered parts: launch_risk_select (moments, t* and
// the risk values into out, reading only q; zeroes grad_out [n_grad] for the sums to come) and
// launch_risk_apply (weights and weighted gradient sums), with the same scratch.  Work that
// touches neither q, out nor the scratch may run between them, on another stream.  mom_part
// [mom_n][2] (sum Q, sum Q^2 over disjoint parts of the samples), when given, stands in for
// the moments pass.
void launch_risk_select(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* out,
                        double* scratch, cudaStream_t s, double* grad_out, int n_grad,
                        const double* mom_part = nullptr, int mom_n = 0);
// flag_src / flag_dst: the weighted pass also copies an int status flag (set by earlier
// kernels) into a double of the results, so that one read-back carries both.
void launch_risk_apply(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* scratch,
                       cudaStream_t s, const float* gq, int ldg, int dz, double* grad_out, int wfirst = 0,
                       int wcount = -1, const int* flag_src = nullptr, double* flag_dst = nullptr);

// ------------------------------------------------------------------ fields
void launch_sample_fields(int n, uint64_t seed, int64_t first, int count, const double* invlam,
                          const double* V, double m_mean, double* m, cudaStream_t s);

// ------------------------------------------------------------------ handle
struct ouu_problem {
  ouu_problem_desc desc;
  cudaStream_t stream;
  int device, num_sms, n, nlev, L, dz, nslots;
  double h, gscale;
  double* d_gx = nullptr;     // [L][n]
  double* d_gy = nullptr;     // [L][n]
  double* d_ut = nullptr;     // [n*n]
  double* d_V = nullptr;      // DCT-II [n][n]
  double* d_invlam = nullptr; // [n*n] 1/lambda
  char* d_slots = nullptr;
  SlotLayout lay;
  int* d_counter = nullptr;
  // per-call buffers (capacity max_samples)
  double* d_u = nullptr;
  double* d_q = nullptr;
  int32_t* d_status = nullptr;
  int32_t* d_iters = nullptr;
  double* d_w = nullptr;      // [OUU_MAX_RISKS][max_samples]
  double* d_s = nullptr;      // [OUU_MAX_RISKS][n*n]
  double* d_out = nullptr;    // results: [OUU_MAX_RISKS][3] + grads [OUU_MAX_RISKS][dz] + misc
  RiskDev* d_risks = nullptr;
  RiskDev rd_last[OUU_MAX_RISKS];   // host copy of what d_risks holds, uploaded on rd_stream
  int rd_n = -1;
  cudaStream_t rd_stream = nullptr;
  double* d_z = nullptr;      // [dz] shared control of the current evaluation
  double* d_rscr = nullptr;   // [OUU_RISK_SCRATCH] risk-weight scratch
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // evaluation phase timers
  double* h_out = nullptr;    // pinned mirror of d_out
  int32_t* h_stat = nullptr;  // pinned: per-sample status/iters copy (max_samples * 4)
  uint64_t serial = 0;        // unique per created problem (a network's held-out check names it)
  int last_backend = -1;      // backend of the last ouu_risk_and_grad that returned OUU_OK
  // phase 1 of a sharded evaluation (ouu_shard_qoi) that phase 2 continues
  int shard_backend = -1;     // -1: none pending
  const double* shard_m = nullptr;
  int shard_n = 0;
  const ouu_dino* shard_dino = nullptr;
  uint64_t shard_dino_eval = 0;   // the network's evaluation that phase 1 ran
};

// Uploads the risk descriptors to p->d_risks on stream `us` unless they equal the last ones
// sent there (every call ends synchronised, so an earlier upload on the same stream is done).
ouu_status ouu_upload_risks(ouu_problem* p, const RiskDev* rd, int n_risks, cudaStream_t us);
// Device form of the descriptors for a sample average over N samples.
void ouu_risk_dev(const ouu_risk_desc* risks, int n_risks, int N, RiskDev* rd);

int ouu_num_levels(int n);
