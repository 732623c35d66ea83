// Persistent per-sample PDE kernels: one CTA solves one sample at a time and pulls
// the next sample index from a global counter (samples differ in Newton/CG
// iteration counts, so the work is balanced dynamically).  A CTA's fine-grid
// vectors live in its own workspace slot (about 1.5 MB at 129 x 129, of which the
// FP32 CG working set is 0.6 MB, so that set of all 152 resident CTAs stays in the
// 126 MB L2); multigrid levels of at most 65 x 65 nodes live in shared memory.
#include "ouu_internal.cuh"
#include "dino.cuh"

static __device__ void build_hierarchy(const PdeArgs& a, char* slot, unsigned char* smem, Hierarchy& H) {
  H.nlev = a.nlev;
  int n = a.n;
  float ih2 = (float)(n - 1) * (float)(n - 1);
  for (int l = 0; l < a.nlev; ++l) {
    MgLevel& L = H.lev[l];
    L.n = n;
    L.inv_h2 = ih2;
    if (l == 0) {
      L.kx = (float*)(slot + a.lay.kx);
      L.ky = (float*)(slot + a.lay.ky);
      L.D = (float*)(slot + a.lay.D);
      L.x = (float*)(slot + a.lay.z);   // preconditioner output z
      L.b = (float*)(slot + a.lay.r);   // CG residual
      L.r = (float*)(slot + a.lay.t);   // scratch
    } else {
      char* base = a.lay.smem_lev[l] >= 0 ? (char*)smem + a.lay.smem_lev[l] : slot + a.lay.lev[l];
      const int64_t sz = ouu_level_array_bytes(n);
      L.kx = (float*)(base);
      L.ky = (float*)(base + sz);
      L.D = (float*)(base + 2 * sz);
      L.x = (float*)(base + 3 * sz);
      L.b = (float*)(base + 4 * sz);
      L.r = (float*)(base + 5 * sz);
    }
    n = (n + 1) / 2;
    ih2 *= 0.25f;
  }
}

static __device__ __forceinline__ int next_sample(int* counter, int* s_idx) {
  if (threadIdx.x == 0) *s_idx = atomicAdd(counter, 1);
  __syncthreads();
  const int i = *s_idx;
  __syncthreads();
  return i;
}

static __device__ void zero_smem(unsigned char* smem, int64_t bytes) {
  float4* p = (float4*)smem;
  for (int64_t k = threadIdx.x; k < bytes / 16; k += blockDim.x) p[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
}

// State solve + QoI of sample i (Sec. 4.2 state equation, Newton), collective over the CTA.
static __device__ void state_task(const PdeArgs& a, CtaCtx& c, Hierarchy& H, char* slot, int i) {
  double* E = (double*)(slot + a.lay.E);
  double* f = (double*)(slot + a.lay.f);
  double* tmp = (double*)(slot + a.lay.tmp);
  float* x = (float*)(slot + a.lay.x);
  float* p = (float*)(slot + a.lay.p);
  float* q = (float*)(slot + a.lay.q);
  const int n = a.n;
  const int64_t nn = (int64_t)n * n;
  const double* m = a.m + (int64_t)i * nn;
  double* u = a.u + (int64_t)i * nn;
  build_fine_coeffs(c, n, m, E, H.lev[0]);
  c.sync();
  setup_coarse_coeffs(c, H);
  build_forcing(c, n, a.L, a.gx, a.gy, a.gscale, a.z + (int64_t)i * a.z_stride, tmp, f);
  for (int64_t k = threadIdx.x; k < nn; k += blockDim.x) u[k] = 0.0;
  c.sync();
  NewtonResult nr = newton_solve(c, H, a.rr, E, f, u, x, p, q, a.newton_rtol, a.newton_maxit, a.cg_rtol, a.cg_maxit);
  const double Q = qoi_and_grad(c, n, u, a.ut, (double*)nullptr);
  if (threadIdx.x == 0) {
    a.q[i] = Q;
    a.status[i] = nr.status;
    a.iters[3 * i + 0] = nr.newton_iters;
    a.iters[3 * i + 1] = nr.cg_iters;
    a.iters[3 * i + 2] = 0;
  }
  c.sync();
}

// State solves of every sample of one problem.
__global__ void __launch_bounds__(OUU_SOLVER_THREADS, 1) k_pde_state(PdeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[40];
  __shared__ int s_idx;
  CtaCtx c{red};
  zero_smem(smem, a.lay.smem_bytes);
  char* slot = a.slots + (int64_t)blockIdx.x * a.lay.bytes;
  Hierarchy H;
  build_hierarchy(a, slot, smem, H);
  for (;;) {
    const int i = next_sample(a.counter, &s_idx);
    if (i >= a.n_samples) break;
    state_task(a, c, H, slot, i);
  }
}

// Adjoint solve (Sec. 2.3) of sample i: J(u_i) lam_i = h^2 (u_i - u_t).  With risk
// weights w[r][i], a sample whose weights are all zero is skipped and sum_i w[r][i] lam_i
// is accumulated in the slot; per-sample lam_i and grad_z Q_i = G^T lam_i are written when
// requested.  Collective over the CTA.
static __device__ void adjoint_task(const PdeArgs& a, CtaCtx& c, Hierarchy& H, char* slot, int i) {
  double* E = (double*)(slot + a.lay.E);
  double* b = (double*)(slot + a.lay.f);
  double* tmp = (double*)(slot + a.lay.tmp);
  double* lam_slot = (double*)(slot + a.lay.lam);
  double* acc = (double*)(slot + a.lay.acc);
  float* x = (float*)(slot + a.lay.x);
  float* p = (float*)(slot + a.lay.p);
  float* q = (float*)(slot + a.lay.q);
  const int n = a.n, L = a.L;
  const int64_t nn = (int64_t)n * n;
  bool need = a.lam_out != nullptr || a.grad_out != nullptr;
  if (a.w)
    for (int r = 0; r < a.n_w; ++r) need = need || a.w[(int64_t)r * a.n_samples + i] != 0.0;
  if (!need) return;
  const double* m = a.m + (int64_t)i * nn;
  const double* u = a.u + (int64_t)i * nn;
  build_fine_coeffs(c, n, m, E, H.lev[0]);
  c.sync();
  setup_coarse_coeffs(c, H);
  setup_jacobian(c, H, a.rr, u);
  qoi_and_grad(c, n, u, a.ut, b);
  double* lam = a.lam_out ? a.lam_out + (int64_t)i * nn : lam_slot;
  for (int64_t k = threadIdx.x; k < nn; k += blockDim.x) lam[k] = 0.0;
  c.sync();
  NewtonResult rr = refine_solve(c, H, a.rr, E, u, b, lam, x, p, q, a.refine_rtol, a.refine_maxit, a.cg_rtol,
                                 a.cg_maxit);
  if (a.w) {
    for (int r = 0; r < a.n_w; ++r) {
      const double wr = a.w[(int64_t)r * a.n_samples + i];
      if (wr == 0.0) continue;
      double* ar = acc + (int64_t)r * nn;
      OUU_FOR_INTERIOR(c, n, iy, ix) {
        const int k = iy * n + ix;
        ar[k] += wr * lam[k];
      }
    }
  }
  if (a.grad_out) {
    // tmp[jx][iy] = sum_ix gx[jx][ix] lam[iy][ix]; grad[jy L + jx] = s sum_iy gy[jy][iy] tmp[jx][iy]
    for (int jx = c.row0(); jx < L; jx += c.rowstep())
      for (int iy = c.col0(); iy < n; iy += c.colstep()) {
        double s = 0.0;
        for (int ix = 1; ix < n - 1; ++ix) s += a.gx[jx * n + ix] * lam[iy * n + ix];
        tmp[jx * n + iy] = s;
      }
    c.sync();
    for (int j = threadIdx.x; j < L * L; j += blockDim.x) {
      const int jy = j / L, jx = j % L;
      double s = 0.0;
      for (int iy = 1; iy < n - 1; ++iy) s += a.gy[jy * n + iy] * tmp[jx * n + iy];
      a.grad_out[(int64_t)i * L * L + j] = a.gscale * s;
    }
  }
  if (threadIdx.x == 0) {
    if (a.solved) atomicAdd(a.solved, 1);
    if (rr.status > a.status[i]) a.status[i] = rr.status;
    a.iters[3 * i + 2] = rr.newton_iters;
    a.iters[3 * i + 1] += rr.cg_iters;
  }
  c.sync();
}

// Adjoint solves of every sample of one problem; the slot accumulators are summed over the
// slots afterwards (launch_reduce_slots_and_gradient).
__global__ void __launch_bounds__(OUU_SOLVER_THREADS, 1) k_pde_adjoint(PdeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[40];
  __shared__ int s_idx;
  CtaCtx c{red};
  zero_smem(smem, a.lay.smem_bytes);
  char* slot = a.slots + (int64_t)blockIdx.x * a.lay.bytes;
  Hierarchy H;
  build_hierarchy(a, slot, smem, H);
  if (a.w) {
    double* acc = (double*)(slot + a.lay.acc);
    for (int64_t k = threadIdx.x; k < (int64_t)a.n_w * a.n * a.n; k += blockDim.x) acc[k] = 0.0;
  }
  __syncthreads();
  for (;;) {
    const int i = next_sample(a.counter, &s_idx);
    if (i >= a.n_samples) break;
    adjoint_task(a, c, H, slot, i);
  }
}

// ------------------------------------------------------------------ many problems, one launch
// Tasks (problem, sample) of many problems of different grids, control counts and sample
// counts, pulled from one counter by persistent CTAs.  A CTA's slot (sized for the largest
// grid) and shared-memory levels are re-zeroed and the multigrid hierarchy rebuilt whenever
// its next task belongs to another problem.  Per task, the SM clock cycles it took are
// added to cycles[problem] (the problem's share of the launch).
static __device__ void zero_region(char* p, int64_t bytes) {
  float4* q = (float4*)p;
  for (int64_t k = threadIdx.x; k < bytes / 16; k += blockDim.x) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
}

// Adds the slot's weighted-adjoint accumulators into the problem's sum (FP64 atomics).
static __device__ void flush_acc(const PdeArgs& a, char* slot) {
  const double* acc = (const double*)(slot + a.lay.acc);
  const int64_t cnt = (int64_t)a.n_w * a.n * a.n;
  for (int64_t k = threadIdx.x; k < cnt; k += blockDim.x)
    if (acc[k] != 0.0) atomicAdd(&a.acc_out[k], acc[k]);
  __syncthreads();
}

template <bool ADJOINT>
__global__ void __launch_bounds__(OUU_SOLVER_THREADS, 1)
    k_pde_batch(const PdeArgs* __restrict__ probs, const int2* __restrict__ tasks, int n_tasks, char* slots,
                int64_t slot_bytes, int* counter, unsigned long long* cycles) {
  constexpr bool adjoint = ADJOINT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[40];
  __shared__ int s_idx;
  CtaCtx c{red};
  char* slot = slots + (int64_t)blockIdx.x * slot_bytes;
  Hierarchy H;
  int cur = -1;
  for (;;) {
    const int t = next_sample(counter, &s_idx);
    if (t >= n_tasks) break;
    const int2 tk = tasks[t];
    if (tk.x != cur) {
      if (adjoint && cur >= 0 && probs[cur].w) flush_acc(probs[cur], slot);
      cur = tk.x;
      const PdeArgs& a = probs[cur];
      zero_region(slot, a.lay.bytes);
      zero_region((char*)smem, a.lay.smem_bytes);
      build_hierarchy(a, slot, smem, H);
    }
    const long long t0 = clock64();
    if (adjoint) adjoint_task(probs[cur], c, H, slot, tk.y);
    else state_task(probs[cur], c, H, slot, tk.y);
    if (threadIdx.x == 0) atomicAdd(&cycles[cur], (unsigned long long)(clock64() - t0));
  }
  if (adjoint && cur >= 0 && probs[cur].w) flush_acc(probs[cur], slot);
}

void launch_pde_batch(const PdeArgs* probs_dev, const int2* tasks_dev, int n_tasks, char* slots, int64_t slot_bytes,
                      int64_t smem_bytes, int nslots, int* counter, unsigned long long* cycles, bool adjoint,
                      cudaStream_t s) {
  if (adjoint) {
    ouu_smem_limit((const void*)k_pde_batch<true>, (size_t)smem_bytes);
    k_pde_batch<true><<<nslots, OUU_SOLVER_THREADS, (size_t)smem_bytes, s>>>(probs_dev, tasks_dev, n_tasks, slots,
                                                                              slot_bytes, counter, cycles);
  } else {
    ouu_smem_limit((const void*)k_pde_batch<false>, (size_t)smem_bytes);
    k_pde_batch<false><<<nslots, OUU_SOLVER_THREADS, (size_t)smem_bytes, s>>>(probs_dev, tasks_dev, n_tasks, slots,
                                                                               slot_bytes, counter, cycles);
  }
}

static void set_smem(const void* fn, int64_t bytes) { ouu_smem_limit(fn, (size_t)bytes); }

void launch_pde_state(const PdeArgs& a, int nslots, cudaStream_t s) {
  set_smem((const void*)k_pde_state, a.lay.smem_bytes);
  k_pde_state<<<nslots, OUU_SOLVER_THREADS, (size_t)a.lay.smem_bytes, s>>>(a);
}

void launch_pde_adjoint(const PdeArgs& a, int nslots, cudaStream_t s) {
  set_smem((const void*)k_pde_adjoint, a.lay.smem_bytes);
  k_pde_adjoint<<<nslots, OUU_SOLVER_THREADS, (size_t)a.lay.smem_bytes, s>>>(a);
}

// ------------------------------------------------------------------ slot reduction + G^T s
__global__ void k_reduce_slots(const char* slots, int64_t slot_bytes, int64_t acc_off, int nslots, int64_t count,
                               double* s_out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int sl = 0; sl < nslots; ++sl) s += ((const double*)(slots + sl * slot_bytes + acc_off))[k];
    s_out[k] = s;
  }
}

__global__ void k_sources_transpose_apply(int n, int L, const double* gx, const double* gy, double gscale,
                                          const double* s, double* grad) {
  extern __shared__ double tmp[];   // [L][n]
  const int r = blockIdx.x;
  const double* sr = s + (int64_t)r * n * n;
  for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
    const int jx = e / n, iy = e % n;
    double a = 0.0;
    for (int ix = 0; ix < n; ++ix) a += gx[jx * n + ix] * sr[iy * n + ix];
    tmp[e] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < L * L; j += blockDim.x) {
    const int jy = j / L, jx = j % L;
    double a = 0.0;
    for (int iy = 0; iy < n; ++iy) a += gy[jy * n + iy] * tmp[jx * n + iy];
    grad[(int64_t)r * L * L + j] = gscale * a;
  }
}

void launch_sources_transpose(int n, int L, int n_w, const double* gx, const double* gy, double gscale,
                              const double* s, double* grad, cudaStream_t st) {
  const size_t sm = (size_t)L * n * sizeof(double);
  if (sm > 48 * 1024) ouu_smem_limit((const void*)k_sources_transpose_apply, sm);
  k_sources_transpose_apply<<<n_w, 256, sm, st>>>(n, L, gx, gy, gscale, s, grad);
}

void launch_reduce_slots_and_gradient(const char* slots, const SlotLayout& lay, int nslots, int n, int L, int n_w,
                                      const double* gx, const double* gy, double gscale, double* s_out,
                                      double* grad, cudaStream_t st) {
  const int64_t count = (int64_t)n_w * n * n;
  k_reduce_slots<<<(int)((count + 255) / 256), 256, 0, st>>>(slots, lay.bytes, lay.acc, nslots, count, s_out);
  const size_t sm = (size_t)L * n * sizeof(double);
  if (sm > 48 * 1024) ouu_smem_limit((const void*)k_sources_transpose_apply, sm);
  k_sources_transpose_apply<<<n_w, 256, sm, st>>>(n, L, gx, gy, gscale, s_out, grad);
}

// ------------------------------------------------------------------ Jacobian data (Sec. 3.4)
// For each sample: one operator set-up J(u_i), then d_Z forward linearised solves
// J w_j = g_j (MG-PCG, FP32) and their projections jy[i][j][r] = h^2 Phi_r . w_j.
// Projected control Jacobians (Sec. 3.4): jy[i][j][r] = h^2 Phi_r . J(u_i)^-1 g_j.  Forward
// route (route 0): one linearised solve per control, J x = g_j, then the r_u projections.
// Adjoint route (route 1): one solve per POD mode, J lam_r = h^2 Phi_r (J is symmetric), then
// jy[i][j][r] = g_j . lam_r by the separable sources: t[jy][ix] = sum_iy gy[jy][iy] lam[iy][ix],
// g_j . lam = gscale sum_ix gx[jx][ix] t[jy][ix].  min(d_Z, r_u) solves per sample either way.
__global__ void __launch_bounds__(OUU_SOLVER_THREADS, 1)
    k_pde_jacobian_data(PdeArgs a, const float* __restrict__ phi, int ru, float* __restrict__ jy, int route) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[40];
  __shared__ int s_idx;
  CtaCtx c{red};
  zero_smem(smem, a.lay.smem_bytes);
  char* slot = a.slots + (int64_t)blockIdx.x * a.lay.bytes;
  Hierarchy H;
  build_hierarchy(a, slot, smem, H);
  double* E = (double*)(slot + a.lay.E);
  float* x = (float*)(slot + a.lay.x);
  float* p = (float*)(slot + a.lay.p);
  float* q = (float*)(slot + a.lay.q);
  const int n = a.n, L = a.L, dz = a.L * a.L;
  const int64_t nn = (int64_t)n * n;
  const float h2 = (float)(1.0 / ((double)(n - 1) * (n - 1)));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (;;) {
    const int i = next_sample(a.counter, &s_idx);
    if (i >= a.n_samples) break;
    build_fine_coeffs(c, n, a.m + (int64_t)i * nn, E, H.lev[0]);
    c.sync();
    setup_coarse_coeffs(c, H);
    setup_jacobian(c, H, a.rr, a.u + (int64_t)i * nn);
    int cg_total = 0;
    if (route == 1) {
      float* t = (float*)(slot + a.lay.tmp);   // [L][n] partial contractions
      for (int r = 0; r < ru; ++r) {
        const float* pr = phi + (int64_t)r * nn;
        double acc = 0.0;
        OUU_FOR_INTERIOR(c, n, iy, ix) {
          const float v = h2 * pr[iy * n + ix];
          H.lev[0].b[iy * n + ix] = v;
          acc = fma((double)v, (double)v, acc);
        }
        const double bnorm = sqrt(c.sum_d(acc));
        CgResult cg = pcg_solve(c, H, x, p, q, bnorm, a.cg_rtol, a.cg_maxit);
        cg_total += cg.iters;
        c.sync();
        for (int jyy = warp; jyy < L; jyy += nwarps)
          for (int ix = lane; ix < n; ix += 32) {
            float sum = 0.f;
            for (int iy = 1; iy < n - 1; ++iy) sum = fmaf((float)a.gy[jyy * n + iy], x[iy * n + ix], sum);
            t[jyy * n + ix] = sum;
          }
        c.sync();
        const float sc = (float)(a.gscale * cg.scale);
        for (int j = warp; j < dz; j += nwarps) {
          const int jx = j % L, jyy = j / L;
          float sum = 0.f;
          for (int ix = lane; ix < n; ix += 32) sum = fmaf((float)a.gx[jx * n + ix], t[jyy * n + ix], sum);
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0) jy[((int64_t)i * dz + j) * ru + r] = sc * sum;
        }
        c.sync();
      }
    }
    for (int j = 0; j < (route == 1 ? 0 : dz); ++j) {
      const int jx = j % L, jyy = j / L;
      float acc = 0.f;
      OUU_FOR_INTERIOR(c, n, iy, ix) {
        const float v = (float)(a.gscale * a.gx[jx * n + ix] * a.gy[jyy * n + iy]);
        H.lev[0].b[iy * n + ix] = v;
        acc += v * v;
      }
      const double bnorm = sqrt(c.sum_f(acc));
      CgResult cg = pcg_solve(c, H, x, p, q, bnorm, a.cg_rtol, a.cg_maxit);
      cg_total += cg.iters;
      const float sc = h2 * (float)cg.scale;
      for (int r = warp; r < ru; r += nwarps) {
        const float* pr = phi + (int64_t)r * nn;
        float s = 0.f;
        for (int64_t k = lane; k < nn; k += 32) s += pr[k] * x[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) jy[((int64_t)i * dz + j) * ru + r] = sc * s;
      }
      c.sync();
    }
    if (threadIdx.x == 0) a.iters[3 * i + 1] = cg_total;
    c.sync();
  }
}

void launch_pde_jacobian_data(const PdeArgs& a, int nslots, const float* phi, int ru, float* jy, int route,
                              cudaStream_t s) {
  set_smem((const void*)k_pde_jacobian_data, a.lay.smem_bytes);
  k_pde_jacobian_data<<<nslots, OUU_SOLVER_THREADS, (size_t)a.lay.smem_bytes, s>>>(a, phi, ru, jy, route);
}
