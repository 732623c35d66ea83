// MR-DINO: reduced-basis neural operator with forward-mode control Jacobian
// (Sec. 3.2-3.4): KL projection, dense GELU net, DINO loss and its gradient,
// Adam, and the surrogate risk evaluation.  Dense contractions run on the
// tcgen05 GEMM (tc_gemm.cu); the kernels here are the element-wise glue.
//
// Training rows are stacked: rows [0, B) carry the values of the B samples,
// rows B + b*dz + j carry the tangent d/dz_j of sample b, so one GEMM moves a
// layer's values or tangents, and one GEMM over all B + B*dz rows forms the
// weight gradient of the value and Jacobian terms together.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "dino.cuh"
#include "gelu.cuh"
#include "ouu_kernels.h"

static int pad8(int x) { return (x + 7) / 8 * 8; }
static int pad64(int x) { return (x + 63) / 64 * 64; }


#define GRID_STRIDE(e, total) \
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (total); e += (int64_t)gridDim.x * blockDim.x)

static int grid_for(int64_t total, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 152 * 16));
}

// ------------------------------------------------------------------ element-wise kernels
// x0[b] = [xi[src]; z[src]; 0-pad], src = idx ? idx[b] : b (z_stride 0: one shared z).
__global__ void k_build_x0(const float* __restrict__ xi, const int* __restrict__ idx, const float* __restrict__ z,
                           int64_t z_stride, int rm, int dz, int in0p, int B, __nv_bfloat16* __restrict__ x0,
                           __nv_bfloat16* __restrict__ x0t) {
  // four consecutive columns per thread (in0p is a multiple of 8): one 8-byte store
  pdl_wait();
  const int q4 = in0p >> 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * q4; e += gridDim.x * blockDim.x) {
    const int b = e / q4, k0 = 4 * (e - b * q4);
    const int64_t src = idx ? idx[b] : b;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + j;
      v[j] = k < rm ? xi[src * rm + k] : (k < rm + dz ? z[src * z_stride + (k - rm)] : 0.f);
    }
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(x0 + (int64_t)b * in0p + k0) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
    if (x0t) {
      x0t[(int64_t)(k0 + 0) * B + b] = p0.x;
      x0t[(int64_t)(k0 + 1) * B + b] = p0.y;
      x0t[(int64_t)(k0 + 2) * B + b] = p1.x;
      x0t[(int64_t)(k0 + 3) * B + b] = p1.y;
    }
  }
}

// First-layer tangents: hdot_1[(b, j), n] = gelu'(a_1[b, n]) * W0[n, rm + j].
__global__ void k_tangent1(const float* __restrict__ a1, const float* __restrict__ W0, int in0, int rm, int dz,
                           int wd, int wdp, int B, __nv_bfloat16* __restrict__ hs_t) {
  GRID_STRIDE(e, (int64_t)B * dz * wd) {
    const int64_t t = e / wd;
    const int n = (int)(e % wd);
    const int b = (int)(t / dz), j = (int)(t % dz);
    hs_t[t * wdp + n] = __float2bfloat16(gelu_d1(a1[(int64_t)b * wd + n]) * W0[(int64_t)n * in0 + rm + j]);
  }
}

// out[c][r] = in[r][c] for r < rows, c < cols (32 x 32 tiles).
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int64_t ld_in, int rows, int cols,
                                 __nv_bfloat16* __restrict__ out, int64_t ld_out) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(int64_t)r * ld_in + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * ld_out + r] = tile[threadIdx.x][k];
  }
}

static void transpose_bf16(const __nv_bfloat16* in, int64_t ld_in, int rows, int cols, __nv_bfloat16* out,
                           int64_t ld_out, cudaStream_t s) {
  dim3 g((cols + 31) / 32, (rows + 31) / 32), b(32, 8);
  k_transpose_bf16<<<g, b, 0, s>>>(in, ld_in, rows, cols, out, ld_out);
}

// DINO loss of Sec. 3.4 and its gradient w.r.t. the stacked outputs.
// Value rows: e = phi - y; tangent rows (b, j): e = d phi / d z_j - Y_b[:, j].
#define LOSS_BLOCKS 256
__global__ void k_loss_out(const float* __restrict__ out, int ldo, const float* __restrict__ y,
                           const float* __restrict__ jy, const int* __restrict__ idx, int B, int dz, int ru, float wj,
                           const float* __restrict__ oscale, __nv_bfloat16* __restrict__ go, int ldgo,
                           float* __restrict__ gov, double* part) {
  __shared__ double red[40];
  double acc = 0.0;
  GRID_STRIDE(e, (int64_t)(B + (int64_t)B * dz) * ru) {
    const int64_t row = e / ru;
    const int r = (int)(e % ru);
    float ev, g;
    if (row < B) {
      const int64_t src = idx[row];
      ev = out[row * ldo + r] - y[src * ru + r];
      g = 2.f * ev / B * oscale[r];     // gradient w.r.t. the unscaled output W3 h3 + b3
      acc += (double)ev * ev / B;
      gov[row * ru + r] = g;
    } else {
      const int64_t t = row - B;
      const int64_t b = t / dz, j = t % dz;
      const int64_t src = idx[b];
      ev = out[row * ldo + r] - jy[(src * dz + j) * ru + r];
      g = 2.f * wj * ev / B * oscale[r];
      acc += (double)wj * ev * ev / B;
    }
    go[row * ldgo + r] = __float2bfloat16(g);
  }
  CtaCtx c{red};
  const double s = c.sum_d(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* part, int n, double* out) {
  __shared__ double red[40];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  CtaCtx c{red};
  const double s = c.sum_d(a);
  if (threadIdx.x == 0) out[0] = s;
}

// Backward through a GELU layer for the stacked rows.
// value row b:   ga[b, n] = s'(a) gh[b, n] + s''(a) sum_j ghdot[(b, j), n] adot[(b, j), n]
// tangent (b,j): gadot[(b, j), n] = s'(a[b, n]) ghdot[(b, j), n]
// adot = AD (layers 2, 3) or W0[n, rm + j] (layer 1).
__global__ void k_bwd_layer(const float* __restrict__ gh, const float* __restrict__ a,
                            const __nv_bfloat16* __restrict__ ad, int wdp, const float* __restrict__ W0, int in0,
                            int rm, int dz, int wd, int B, __nv_bfloat16* __restrict__ ga, float* __restrict__ gav) {
  GRID_STRIDE(e, (int64_t)(B + (int64_t)B * dz) * wd) {
    const int64_t row = e / wd;
    const int n = (int)(e % wd);
    if (row < B) {
      const float av = a[row * wd + n];
      float s = 0.f;
      for (int j = 0; j < dz; ++j) {
        const int64_t t = row * dz + j;
        const float adot = ad ? __bfloat162float(ad[t * wdp + n]) : W0[(int64_t)n * in0 + rm + j];
        s += gh[(B + t) * wd + n] * adot;
      }
      const float g = gelu_d1(av) * gh[row * wd + n] + gelu_d2(av) * s;
      ga[row * wdp + n] = __float2bfloat16(g);
      gav[row * wd + n] = g;
    } else {
      const int64_t b = (row - B) / dz;
      ga[row * wdp + n] = __float2bfloat16(gelu_d1(a[b * wd + n]) * gh[row * wd + n]);
    }
  }
}

// dW0[n, rm + j] += sum_b s'(a_1[b, n]) ghdot_1[(b, j), n]  (first-layer tangent term).
__global__ void k_dw0z(const float* __restrict__ a1, const float* __restrict__ gh, int B, int dz, int wd, int rm,
                       int in0, float* __restrict__ dW0) {
  GRID_STRIDE(e, (int64_t)dz * wd) {
    const int j = (int)(e / wd), n = (int)(e % wd);
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += gelu_d1(a1[(int64_t)b * wd + n]) * gh[(B + (int64_t)b * dz + j) * wd + n];
    dW0[(int64_t)n * in0 + rm + j] += s;
  }
}

// out[c] = sum_r X[r][c]
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols, int ld, float* __restrict__ out) {
  GRID_STRIDE(c, cols) {
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += X[(int64_t)r * ld + c];
    out[c] = s;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  GRID_STRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 copies of one weight matrix W [out][in]: Wb [out][inp], WTb [in][outp].
__global__ void k_weight_bf16(const float* __restrict__ W, int out, int in, int inp, int outp,
                              __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ WTb) {
  GRID_STRIDE(e, (int64_t)out * inp) {
    const int o = (int)(e / inp), i = (int)(e % inp);
    const __nv_bfloat16 v = __float2bfloat16(i < in ? W[(int64_t)o * in + i] : 0.f);
    Wb[e] = v;
    if (i < in) WTb[(int64_t)i * outp + o] = v;
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ in, int ld_in, int rows, int cols, double* __restrict__ out) {
  GRID_STRIDE(e, (int64_t)rows * cols) {
    const int64_t r = e / cols;
    const int c = (int)(e % cols);
    out[e] = in[r * ld_in + c];
  }
}

__global__ void k_copy_rows_f32(const float* __restrict__ in, int ld_in, int rows, int cols, float* __restrict__ out,
                                int ld_out) {
  GRID_STRIDE(e, (int64_t)rows * cols) {
    const int64_t r = e / cols;
    const int c = (int)(e % cols);
    out[r * ld_out + c] = in[r * ld_in + c];
  }
}

// y[i][r] = h^2 sum_p Phi[r][p] (u_i[p] - ubar[p])  (FP32, 32 x 32 output tiles).
__global__ void k_project_states(const double* __restrict__ u, const double* __restrict__ ubar,
                                 const float* __restrict__ phi, int nn, int ru, int N, float h2, float* __restrict__ y) {
  __shared__ float su[32][33], sp[32][33];
  const int i0 = blockIdx.y * 32, r0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int p0 = 0; p0 < nn; p0 += 32) {
    for (int k = ty; k < 32; k += 8) {
      const int i = i0 + k, r = r0 + k, p = p0 + tx;
      su[k][tx] = (i < N && p < nn) ? (float)(u[(int64_t)i * nn + p] - ubar[p]) : 0.f;
      sp[k][tx] = (r < ru && p < nn) ? phi[(int64_t)r * nn + p] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int pp = 0; pp < 32; ++pp) {
      const float b = sp[tx][pp];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += su[ty + 8 * q][pp] * b;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, r = r0 + tx;
    if (i < N && r < ru) y[(int64_t)i * ru + r] = h2 * acc[q];
  }
}

// c[r] = h^2 sum_p Phi[r][p] (ubar[p] - ut[p]) and sum_p h^2 (ubar - ut)^2 (FP64).
__global__ void k_reduced_qoi_terms(const double* __restrict__ phi64, const double* __restrict__ ubar,
                                    const double* __restrict__ ut, int n, int ru, double* __restrict__ c,
                                    double* __restrict__ norm2) {
  __shared__ double red[40];
  CtaCtx cc{red};
  const double h2 = 1.0 / ((double)(n - 1) * (n - 1));
  const int r = blockIdx.x;
  double s = 0.0;
  for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
    const int iy = p / n, ix = p % n;
    if (iy == 0 || ix == 0 || iy == n - 1 || ix == n - 1) continue;
    const double d = ubar[p] - ut[p];
    s += r < ru ? phi64[(int64_t)r * n * n + p] * d : d * d;
  }
  const double t = cc.sum_d(s);
  if (threadIdx.x == 0) {
    if (r < ru) c[r] = h2 * t;
    else *norm2 = h2 * t;
  }
}

__global__ void k_phi_to_f32(const double* __restrict__ in, int64_t count, float* __restrict__ out) {
  GRID_STRIDE(e, count) out[e] = (float)in[e];
}

// ------------------------------------------------------------------ host helpers
#define DINO_TRY(expr)                        \
  do {                                        \
    ouu_status st_ = (expr);                  \
    if (st_ != OUU_OK) return st_;            \
  } while (0)

static EpiParams epi(int mode) {
  EpiParams e;
  std::memset(&e, 0, sizeof(e));
  e.mode = mode;
  e.alpha = 1.f;
  e.aux_rdiv = 1;
  return e;
}

static ouu_status gemm(ouu_dino* d, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                       int K, const EpiParams& ep) {
  return ouu_gemm_bf16(A, lda, B, ldb, M, N, K, ep, d->d_err, d->stream);
}

// out [M][N] (leading dimension N) = A B^T with K split over CTAs so that the few output tiles of
// a weight gradient (M, N <= 400, K = batch x (1 + d_Z)) fill the GPU: the slices' FP32 partial
// products are added atomically into the zeroed output.
static ouu_status gemm_wgrad(ouu_dino* d, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
                             int N, int K, float* out) {
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128), kb = (K + 63) / 64;
  int splits = std::max(1, std::min(std::min(64, kb), d->num_sms / std::max(1, tiles)));
  while (splits > 1 && (splits - 1) * ((kb + splits - 1) / splits) >= kb) --splits;   // no empty slice
  EpiParams e = epi(EPI_LINEAR);
  e.out_f32 = out;
  e.ld_f32 = N;
  if (splits > 1) OUU_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)M * N * 4, d->stream));
  return ouu_gemm_bf16(A, lda, B, ldb, M, N, K, e, d->d_err, d->stream, splits);
}

extern "C" void ouu_default_dino_desc(ouu_dino_desc* d) {
  if (!d) return;
  d->n = 129;
  d->lattice_L = 10;
  d->r_m = 200;
  d->r_u = 200;
  d->width = 400;
  d->max_batch = 256;
  d->max_eval = 4096;
  d->gamma = 0.1;
  d->delta = 1.0;
  d->m_mean = 0.0;
  d->jac_weight = 1.0;
}

static void free_dino(ouu_dino* d) {
  if (!d) return;
  void* ptrs[] = {d->d_params, d->d_grad, d->d_adam_m, d->d_adam_v, d->d_phi, d->d_phi64, d->d_ubar, d->d_ut,
                  d->d_c, d->d_cf, d->d_wkl, d->d_kl_order, d->X0, d->X0T, d->OUT, d->GO, d->GOT, d->GH, d->GA, d->GAT,
                  d->GAv, d->GA1T, d->d_loss_part, d->d_loss, d->XIe, d->X0e, d->He0, d->He1, d->OUTe,
                  d->Ge, d->GQe, d->Qe, d->Qpart, d->Qmom, d->d_zf, d->d_err, d->d_klp_ctr, d->d_gov, d->d_oscale,
                  d->d_klbias, d->d_dec_b, d->d_dec_a, d->d_ubarf, d->d_utf, d->d_qdec};
  for (void* p : ptrs) cudaFree(p);
  for (int l = 0; l < 4; ++l) {
    cudaFree(d->A[l]);
    cudaFree(d->HS[l]);
    cudaFree(d->HST[l]);
    cudaFree(d->AD[l]);
    cudaFree(d->Ae[l]);
    cudaFree(d->Wb[l]);
    cudaFree(d->WTb[l]);
  }
  cudaFreeHost(d->h_pin);
  for (auto& e : d->ev)
    if (e) cudaEventDestroy(e);
  if (d->gexec) cudaGraphExecDestroy(d->gexec);
  if (d->cap) cudaStreamDestroy(d->cap);
  if (d->side) cudaStreamDestroy(d->side);
  if (d->ev_fork) cudaEventDestroy(d->ev_fork);
  if (d->ev_join) cudaEventDestroy(d->ev_join);
  delete d;
}

extern "C" ouu_status ouu_dino_destroy(ouu_dino_t d) {
  if (!d) return OUU_OK;
  cudaStreamSynchronize(d->stream);
  free_dino(d);
  return OUU_OK;
}

extern "C" size_t ouu_dino_num_params(ouu_dino_t d) { return d ? d->n_params : 0; }

extern "C" ouu_status ouu_dino_create(const ouu_dino_desc* desc, void* cuda_stream, ouu_dino_t* out) {
  OUU_CHECK_ARG(desc && out, "null argument");
  *out = nullptr;
  const int n = desc->n;
  OUU_CHECK_ARG(n >= 5 && n <= 1025 && (((n - 1) & (n - 2)) == 0), "n must be 2^k + 1");
  OUU_CHECK_ARG(desc->lattice_L >= 1 && desc->lattice_L <= 64, "lattice_L must be in [1, 64]");
  OUU_CHECK_ARG(desc->r_m >= 1 && desc->r_m <= n * n && desc->r_m <= 240 && desc->r_u >= 1 && desc->r_u <= 256,
                "ranks: 1 <= r_m <= min(n^2, 240) (the projection's N tile), 1 <= r_u <= 256");
  OUU_CHECK_ARG(desc->width >= 8 && desc->width % 8 == 0 && desc->width <= 2048, "width: multiple of 8");
  OUU_CHECK_ARG(desc->max_batch >= 8 && desc->max_batch % 8 == 0, "max_batch: positive multiple of 8");
  OUU_CHECK_ARG(desc->max_eval >= 1, "max_eval must be positive");
  OUU_CHECK_ARG(desc->gamma > 0 && desc->delta > 0 && desc->jac_weight >= 0, "bad prior or loss weight");
  ouu_dino* d = new ouu_dino();
  d->desc = *desc;
  d->stream = (cudaStream_t)cuda_stream;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) d->num_sms = 148;
  }
  d->n = n;
  d->nn = n * n;
  d->nnp = pad64(n * n);
  d->dz = desc->lattice_L * desc->lattice_L;
  d->rm = desc->r_m;
  d->ru = desc->r_u;
  d->wd = desc->width;
  d->in0 = d->rm + d->dz;
  d->maxB = desc->max_batch;
  d->maxE = desc->max_eval;
  d->R = d->maxB * d->dz;
  d->BR = d->maxB + d->R;
  d->h = 1.0 / (n - 1);
  const int ins[4] = {d->in0, d->wd, d->wd, d->wd}, outs[4] = {d->wd, d->wd, d->wd, d->ru};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    d->in_l[l] = ins[l];
    d->out_l[l] = outs[l];
    d->inp_l[l] = pad8(ins[l]);
    d->outp_l[l] = pad8(outs[l]);
    d->offW[l] = off;
    off += (size_t)ins[l] * outs[l];
    d->offb[l] = off;
    off += outs[l];
  }
  d->n_params = off;
  const int wdp = d->wd, rup = pad8(d->ru), in0p = d->inp_l[0], dzp = pad8(d->dz);
  const size_t BR = d->BR, maxB = d->maxB, E = d->maxE;
  bool ok = true;
  auto al = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
    if (ok) cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
  };
  al((void**)&d->d_params, off * 4);
  al((void**)&d->d_grad, off * 4);
  al((void**)&d->d_adam_m, off * 4);
  al((void**)&d->d_adam_v, off * 4);
  for (int l = 0; l < 4; ++l) {
    al((void**)&d->Wb[l], (size_t)outs[l] * d->inp_l[l] * 2);
    al((void**)&d->WTb[l], (size_t)ins[l] * d->outp_l[l] * 2);
  }
  al((void**)&d->d_phi, (size_t)d->ru * d->nn * 4);
  al((void**)&d->d_phi64, (size_t)d->ru * d->nn * 8);
  al((void**)&d->d_ubar, (size_t)d->nn * 8);
  al((void**)&d->d_ut, (size_t)d->nn * 8);
  al((void**)&d->d_c, (size_t)d->ru * 8 + 16);
  al((void**)&d->d_cf, (size_t)d->ru * 4 + 16);
  al((void**)&d->d_oscale, (size_t)d->ru * 4);
  al((void**)&d->d_dec_b, (size_t)d->nn * 3 * rup * 2);
  al((void**)&d->d_dec_a, E * 3 * rup * 2);
  al((void**)&d->d_ubarf, (size_t)d->nn * 4);
  al((void**)&d->d_utf, (size_t)d->nn * 4);
  al((void**)&d->d_qdec, E * 8);
  al((void**)&d->d_wkl, (size_t)d->rm * d->nnp * 2);
  al((void**)&d->d_kl_order, (size_t)d->rm * 4);
  al((void**)&d->d_klbias, (size_t)d->rm * 4);
  al((void**)&d->X0, maxB * in0p * 2);
  al((void**)&d->X0T, (size_t)in0p * maxB * 2);
  for (int l = 1; l <= 3; ++l) {
    al((void**)&d->A[l], maxB * d->wd * 4);
    al((void**)&d->HS[l], BR * wdp * 2);
    al((void**)&d->HST[l], (size_t)d->wd * BR * 2);
    if (l >= 2) al((void**)&d->AD[l], (size_t)d->R * wdp * 2);
  }
  al((void**)&d->OUT, BR * rup * 4);
  al((void**)&d->GO, BR * rup * 2);
  al((void**)&d->GOT, (size_t)d->ru * BR * 2);
  al((void**)&d->d_gov, maxB * d->ru * 4);
  al((void**)&d->GH, BR * d->wd * 4);
  al((void**)&d->GA, BR * wdp * 2);
  al((void**)&d->GAT, (size_t)d->wd * BR * 2);
  al((void**)&d->GAv, maxB * d->wd * 4);
  al((void**)&d->GA1T, (size_t)d->wd * maxB * 2);
  al((void**)&d->d_loss_part, LOSS_BLOCKS * 8);
  al((void**)&d->d_loss, 16);
  al((void**)&d->XIe, E * d->rm * 4);
  al((void**)&d->X0e, E * in0p * 2);
  for (int l = 1; l <= 3; ++l) al((void**)&d->Ae[l], E * d->wd * 4);
  al((void**)&d->He0, E * wdp * 2);
  al((void**)&d->He1, E * wdp * 2);
  al((void**)&d->OUTe, E * rup * 4);
  al((void**)&d->Ge, E * rup * 2);
  al((void**)&d->GQe, E * dzp * 4);
  al((void**)&d->Qe, E * 8);
  al((void**)&d->Qpart, E * 4 * 4);
  al((void**)&d->Qmom, (E / 128 + 1) * 2 * 8);
  al((void**)&d->d_zf, std::max<size_t>(maxB, 1) * d->dz * 4 + 64);
  al((void**)&d->d_err, 16);
  al((void**)&d->d_klp_ctr, (OUU_KLP_MAX_TILES + 1) * sizeof(int));   // zeroed by al()
  if (ok && cudaMallocHost((void**)&d->h_pin, (size_t)(4 * 3 + 4 * d->dz + 64) * 8 + 4096) != cudaSuccess) ok = false;
  if (ok && cudaHostGetDevicePointer((void**)&d->h_pin_dev, d->h_pin, 0) != cudaSuccess) {
    d->h_pin_dev = nullptr;   // not mapped: the controls then go by a copy
    cudaGetLastError();
  }
  if (!ok) {
    cudaGetLastError();
    free_dino(d);
    ouu_set_error("device allocation failed in ouu_dino_create");
    return OUU_ERR_OOM;
  }
  // KL projection rows: mode order by (lambda, k1 + k2, k1); row j = (lambda_q / n) v_k1(ix) v_k2(iy).
  {
    std::vector<double> mu(n), V((size_t)n * n);
    for (int k = 0; k < n; ++k) {
      const double sn = std::sin(M_PI * k / (2.0 * n));
      mu[k] = 4.0 * n * n * (sn * sn);
      const double s = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      for (int j = 0; j < n; ++j) V[(size_t)k * n + j] = s * std::cos(M_PI * k * (j + 0.5) / n);
    }
    std::vector<int> q(n * n);
    std::iota(q.begin(), q.end(), 0);
    auto lam = [&](int qq) { return desc->delta + desc->gamma * (mu[qq % n] + mu[qq / n]); };
    std::stable_sort(q.begin(), q.end(), [&](int a, int b) {
      const double la = lam(a), lb = lam(b);
      if (la != lb) return la < lb;
      const int sa = a % n + a / n, sb = b % n + b / n;
      if (sa != sb) return sa < sb;
      return a % n < b % n;
    });
    std::vector<__nv_bfloat16> rows((size_t)d->rm * d->nnp, __float2bfloat16(0.f));
    for (int j = 0; j < d->rm; ++j) {
      const int qq = q[j], k1 = qq % n, k2 = qq / n;
      const double sc = lam(qq) / n;
      for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix)
          rows[(size_t)j * d->nnp + iy * n + ix] = __float2bfloat16((float)(sc * V[(size_t)k2 * n + iy] * V[(size_t)k1 * n + ix]));
    }
    OUU_CUDA_TRY(cudaMemcpy(d->d_wkl, rows.data(), rows.size() * 2, cudaMemcpyHostToDevice));
    std::vector<float> klb(d->rm, 0.f);
    for (int j = 0; j < d->rm; ++j) {
      double s = 0.0;
      for (int p = 0; p < d->nn; ++p) s += (double)__bfloat162float(rows[(size_t)j * d->nnp + p]);
      klb[j] = (float)(-desc->m_mean * s);
    }
    OUU_CUDA_TRY(cudaMemcpy(d->d_klbias, klb.data(), (size_t)d->rm * 4, cudaMemcpyHostToDevice));
    OUU_CUDA_TRY(cudaMemcpy(d->d_kl_order, q.data(), (size_t)d->rm * 4, cudaMemcpyHostToDevice));
    std::vector<double> ut(d->nn);
    for (int iy = 0; iy < n; ++iy)
      for (int ix = 0; ix < n; ++ix)
        ut[(size_t)iy * n + ix] = std::sin(M_PI * (ix / (double)(n - 1))) * std::sin(M_PI * (iy / (double)(n - 1)));
    OUU_CUDA_TRY(cudaMemcpy(d->d_ut, ut.data(), (size_t)d->nn * 8, cudaMemcpyHostToDevice));
    std::vector<float> ones(d->ru, 1.f);
    OUU_CUDA_TRY(cudaMemcpy(d->d_oscale, ones.data(), (size_t)d->ru * 4, cudaMemcpyHostToDevice));
  }
  for (auto& e : d->ev) OUU_CUDA_TRY(cudaEventCreate(&e));
  OUU_CUDA_TRY(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
  OUU_CUDA_TRY(cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking));
  OUU_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming));
  OUU_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming));
  OUU_CUDA_TRY(cudaDeviceSynchronize());
  *out = d;
  return OUU_OK;
}

static void refresh_bf16_weights(ouu_dino* d) {
  for (int l = 0; l < 4; ++l) {
    const int64_t tot = (int64_t)d->out_l[l] * d->inp_l[l];
    k_weight_bf16<<<grid_for(tot), 256, 0, d->stream>>>(d->d_params + d->offW[l], d->out_l[l], d->in_l[l],
                                                         d->inp_l[l], d->outp_l[l], d->Wb[l], d->WTb[l]);
  }
}

extern "C" ouu_status ouu_dino_set_params(ouu_dino_t d, const float* params_host, size_t n) {
  OUU_CHECK_ARG(d && params_host, "null argument");
  OUU_CHECK_ARG(n == d->n_params, "parameter count mismatch");
  d->val_ok = 0;   // another network: its held-out check is to be done again
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_params, params_host, n * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemsetAsync(d->d_adam_m, 0, n * 4, d->stream));
  OUU_CUDA_TRY(cudaMemsetAsync(d->d_adam_v, 0, n * 4, d->stream));
  d->adam_t = 0;
  refresh_bf16_weights(d);
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_get_params(ouu_dino_t d, float* params_host, size_t n) {
  OUU_CHECK_ARG(d && params_host, "null argument");
  OUU_CHECK_ARG(n == d->n_params, "parameter count mismatch");
  OUU_CUDA_TRY(cudaMemcpyAsync(params_host, d->d_params, n * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

// x = hi + lo with hi, lo BF16 (round to nearest): hi x hi' + hi x lo' + lo x hi' carries about
// 16 significant bits of a product of two such splits.
static __device__ __forceinline__ void bf16_split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Basis side of the decode GEMM: b[p][k] = Phi_hi, b[p][rup + k] = Phi_lo, b[p][2 rup + k] =
// Phi_hi of mode k at node p (zero for k >= ru); ubar and the target state in FP32, the latter
// zero on the boundary (the QoI sums over the interior, where Phi and ubar live).
__global__ void k_decode_basis(const double* __restrict__ phi64, const double* __restrict__ ubar,
                               const double* __restrict__ ut, int n, int ru, int rup, __nv_bfloat16* __restrict__ b,
                               float* __restrict__ ubarf, float* __restrict__ utf) {
  const int nn = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nn * rup;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / rup), k = (int)(e - (int64_t)p * rup);
    __nv_bfloat16 hi = __float2bfloat16_rn(0.f), lo = hi;
    if (k < ru) bf16_split((float)phi64[(int64_t)k * nn + p], hi, lo);
    __nv_bfloat16* row = b + (int64_t)p * 3 * rup;
    row[k] = hi;
    row[rup + k] = lo;
    row[2 * rup + k] = hi;
    if (k == 0) {
      const int ix = p % n, iy = p / n;
      const bool interior = ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1;
      ubarf[p] = (float)ubar[p];
      utf[p] = interior ? (float)ut[p] : 0.f;
    }
  }
}

// Coefficient side: a[i][k] = a[i][rup + k] = phi_hi, a[i][2 rup + k] = phi_lo (zero for k >= ru).
__global__ void k_decode_coeffs(const float* __restrict__ phi, int ldphi, int N, int ru, int rup,
                                __nv_bfloat16* __restrict__ a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * rup;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / rup), k = (int)(e - (int64_t)i * rup);
    __nv_bfloat16 hi = __float2bfloat16_rn(0.f), lo = hi;
    if (k < ru) bf16_split(phi[(int64_t)i * ldphi + k], hi, lo);
    __nv_bfloat16* row = a + (int64_t)i * 3 * rup;
    row[k] = hi;
    row[rup + k] = hi;
    row[2 * rup + k] = lo;
  }
}

ouu_status dino_decode(ouu_dino* d, const float* phi, int ldphi, int N, float* u, double* q) {
  const int rup = pad8(d->ru), K = 3 * rup;
  k_decode_coeffs<<<grid_for((int64_t)N * rup), 256, 0, d->stream>>>(phi, ldphi, N, d->ru, rup, d->d_dec_a);
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaMemsetAsync(q, 0, (size_t)N * 8, d->stream));
  EpiParams e = epi(EPI_DECODE);   // rows: the nn grid nodes; columns: the N samples
  e.out_f32 = u;
  e.ld_f32 = d->nn;
  e.col_add = d->d_ubarf;
  e.col_ref = d->d_utf;
  e.out_q = q;
  e.qconst = 0.5 * d->h * d->h;
  return gemm(d, d->d_dec_b, K, d->d_dec_a, K, d->nn, N, K, e);
}

static ouu_status check_err(ouu_dino* d);

extern "C" ouu_status ouu_dino_decode(ouu_dino_t d, const float* phi_dev, int n_samples, float* u_dev,
                                      double* q_dev) {
  OUU_CHECK_ARG(d && phi_dev && u_dev, "null argument");
  if (!d->bases_ready) {
    ouu_set_error("bases not built");
    return OUU_ERR_STATE;
  }
  OUU_CHECK_ARG(n_samples >= 1 && n_samples <= d->maxE, "n_samples outside [1, max_eval]");
  DINO_TRY(dino_decode(d, phi_dev, d->ru, n_samples, u_dev, q_dev ? q_dev : d->d_qdec));
  return check_err(d);
}

// Installs Phi (FP64 copy already in d_phi64) and ubar: FP32 copy, c and the constant, and
// the basis side of the decode GEMM.
ouu_status dino_install_bases(ouu_dino* d) {
  d->val_ok = 0;
  const int64_t cnt = (int64_t)d->ru * d->nn;
  k_phi_to_f32<<<grid_for(cnt), 256, 0, d->stream>>>(d->d_phi64, cnt, d->d_phi);
  k_decode_basis<<<grid_for((int64_t)d->nn * pad8(d->ru)), 256, 0, d->stream>>>(
      d->d_phi64, d->d_ubar, d->d_ut, d->n, d->ru, pad8(d->ru), d->d_dec_b, d->d_ubarf, d->d_utf);
  k_reduced_qoi_terms<<<d->ru + 1, 256, 0, d->stream>>>(d->d_phi64, d->d_ubar, d->d_ut, d->n, d->ru, d->d_c,
                                                         d->d_c + d->ru);
  OUU_CUDA_TRY(cudaGetLastError());
  std::vector<double> c(d->ru + 1);
  OUU_CUDA_TRY(cudaMemcpyAsync(c.data(), d->d_c, (d->ru + 1) * 8, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  double cc = 0.0;
  std::vector<float> cf(d->ru);
  for (int r = 0; r < d->ru; ++r) {
    cc += c[r] * c[r];
    cf[r] = (float)c[r];
  }
  d->qconst = 0.5 * (c[d->ru] - cc);
  OUU_CUDA_TRY(cudaMemcpy(d->d_cf, cf.data(), (size_t)d->ru * 4, cudaMemcpyHostToDevice));
  d->bases_ready = 1;
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_set_bases(ouu_dino_t d, const double* phi_dev, const double* ubar_dev) {
  OUU_CHECK_ARG(d && phi_dev && ubar_dev, "null argument");
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_phi64, phi_dev, (size_t)d->ru * d->nn * 8, cudaMemcpyDeviceToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_ubar, ubar_dev, (size_t)d->nn * 8, cudaMemcpyDeviceToDevice, d->stream));
  return dino_install_bases(d);
}

extern "C" ouu_status ouu_dino_get_bases(ouu_dino_t d, double* phi_dev, double* ubar_dev) {
  OUU_CHECK_ARG(d && d->bases_ready, "bases not built");
  if (phi_dev)
    OUU_CUDA_TRY(cudaMemcpyAsync(phi_dev, d->d_phi64, (size_t)d->ru * d->nn * 8, cudaMemcpyDeviceToDevice, d->stream));
  if (ubar_dev)
    OUU_CUDA_TRY(cudaMemcpyAsync(ubar_dev, d->d_ubar, (size_t)d->nn * 8, cudaMemcpyDeviceToDevice, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

static ouu_status check_err(ouu_dino* d) {
  int e = 0;
  OUU_CUDA_TRY(cudaMemcpyAsync(&e, d->d_err, 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  if (e) {
    cudaMemsetAsync(d->d_err, 0, 4, d->stream);
    // an interrupted projection may have left its tile counters non-zero
    cudaMemsetAsync(d->d_klp_ctr, 0, (OUU_KLP_MAX_TILES + 1) * sizeof(int), d->stream);
    ouu_set_error("tensor-core GEMM pipeline wait timed out");
    return OUU_ERR_CUDA;
  }
  return OUU_OK;
}

// KL coordinates of `count` fields (chunked BF16 cast + tensor-core projection).
// With mark, events ev[0] / ev[2] bracket the projection in an eagerly enqueued call.  With
// graph_mark as well, while a graph is captured, they become event nodes of the graph, which
// every replay records: ev[2] on the side stream, forked after the projection so that the
// next kernel on the main stream keeps its programmatic edge (the caller joins the side
// stream back before the capture ends).  With zstage, the projection launch also stages the
// controls (d_zf) from the mapped pinned buffer.
static ouu_status project_fields(ouu_dino* d, const double* m, int count, float* xi, bool mark = false,
                                 bool zstage = false, bool graph_mark = false) {
  // one fused pass over the FP64 fields (kl_project.cu); the bias -W mbar carries the prior mean
  const bool eager_mark = mark && !d->capturing, node_mark = mark && graph_mark && d->capturing;
  if (eager_mark) OUU_CUDA_TRY(cudaEventRecord(d->ev[0], d->stream));
  if (node_mark) OUU_CUDA_TRY(cudaEventRecordWithFlags(d->ev[0], d->stream, cudaEventRecordExternal));
  DINO_TRY(ouu_kl_project(m, count, d->nn, d->d_wkl, d->nnp, d->rm, d->d_klbias, xi, d->d_err, d->d_klp_ctr,
                          d->num_sms, d->stream, zstage ? d->h_pin_dev : nullptr, d->d_zf, d->dz));
  if (eager_mark) OUU_CUDA_TRY(cudaEventRecord(d->ev[2], d->stream));
  if (node_mark) {
    OUU_CUDA_TRY(cudaEventRecord(d->ev_fork, d->stream));
    OUU_CUDA_TRY(cudaStreamWaitEvent(d->side, d->ev_fork, 0));
    OUU_CUDA_TRY(cudaEventRecordWithFlags(d->ev[2], d->side, cudaEventRecordExternal));
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_project_fields(ouu_dino_t d, const double* m_dev, int n_samples, float* xi_dev) {
  OUU_CHECK_ARG(d && m_dev && xi_dev && n_samples >= 0, "bad argument");
  if (n_samples == 0) return OUU_OK;
  DINO_TRY(project_fields(d, m_dev, n_samples, xi_dev));
  return check_err(d);
}

extern "C" ouu_status ouu_dino_project_states(ouu_dino_t d, const double* u_dev, int n_samples, float* y_dev) {
  OUU_CHECK_ARG(d && u_dev && y_dev && n_samples >= 0, "bad argument");
  OUU_CHECK_ARG(d->bases_ready, "bases not built");
  if (n_samples == 0) return OUU_OK;
  dim3 g((d->ru + 31) / 32, (n_samples + 31) / 32), b(32, 8);
  k_project_states<<<g, b, 0, d->stream>>>(u_dev, d->d_ubar, d->d_phi, d->nn, d->ru, n_samples,
                                            (float)(d->h * d->h), y_dev);
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

// ------------------------------------------------------------------ forward with tangents
// Stacked forward pass for B samples (rows of xi/z/y chosen by idx): values in
// A[1..3], HS[1..3] rows [0, B), tangents in HS rows [B, B + B dz), AD[2..3];
// outputs phi in OUT rows [0, B) and J^T in jout (row (b, j) = d phi_b / d z_j).
static ouu_status forward_tangent(ouu_dino* d, const float* xi, const float* z, int64_t z_stride, const int* idx,
                                  int B, float* jout, int ld_jout, bool transposed) {
  const int wd = d->wd, wdp = d->wd, rup = pad8(d->ru), in0p = d->inp_l[0], dz = d->dz;
  const int R = B * dz, BR = B + R;
  k_build_x0<<<grid_for((int64_t)B * (in0p / 4)), 256, 0, d->stream>>>(xi, idx, z, z_stride, d->rm, dz, in0p, B, d->X0,
                                                                  transposed ? d->X0T : nullptr);
  {  // layer 0 values
    EpiParams ep = epi(EPI_GELU);
    ep.bias = d->d_params + d->offb[0];
    ep.out_f32 = d->A[1];
    ep.ld_f32 = wd;
    ep.out_bf16 = d->HS[1];
    ep.ld_bf16 = wdp;
    if (transposed) {
      ep.out_t_bf16 = d->HST[1];
      ep.ld_t = BR;
    }
    DINO_TRY(gemm(d, d->X0, in0p, d->Wb[0], d->inp_l[0], B, wd, d->in0, ep));
  }
  k_tangent1<<<grid_for((int64_t)R * wd), 256, 0, d->stream>>>(d->A[1], d->d_params + d->offW[0], d->in0, d->rm, dz,
                                                               wd, wdp, B, d->HS[1] + (int64_t)B * wdp);
  if (transposed) transpose_bf16(d->HS[1] + (int64_t)B * wdp, wdp, R, wd, d->HST[1] + B, BR, d->stream);
  for (int l = 1; l <= 2; ++l) {
    EpiParams ev = epi(EPI_GELU);
    ev.bias = d->d_params + d->offb[l];
    ev.out_f32 = d->A[l + 1];
    ev.ld_f32 = wd;
    ev.out_bf16 = d->HS[l + 1];
    ev.ld_bf16 = wdp;
    if (transposed) {
      ev.out_t_bf16 = d->HST[l + 1];
      ev.ld_t = BR;
    }
    DINO_TRY(gemm(d, d->HS[l], wdp, d->Wb[l], wdp, B, wd, wd, ev));
    EpiParams et = epi(EPI_DGELU_SCALE);
    et.aux = d->A[l + 1];
    et.ld_aux = wd;
    et.aux_rdiv = dz;
    et.out_bf16 = d->HS[l + 1] + (int64_t)B * wdp;
    et.ld_bf16 = wdp;
    if (transposed) {
      et.out_t_bf16 = d->HST[l + 1] + B;
      et.ld_t = BR;
    }
    et.out2_bf16 = d->AD[l + 1];
    et.ld2 = wdp;
    DINO_TRY(gemm(d, d->HS[l] + (int64_t)B * wdp, wdp, d->Wb[l], wdp, R, wd, wd, et));
  }
  {  // output layer: values and tangents
    EpiParams ev = epi(EPI_LINEAR);
    ev.bias = d->d_params + d->offb[3];
    ev.col_scale = d->d_oscale;
    ev.out_f32 = d->OUT;
    ev.ld_f32 = rup;
    DINO_TRY(gemm(d, d->HS[3], wdp, d->Wb[3], wdp, B, d->ru, wd, ev));
    EpiParams et = epi(EPI_LINEAR);
    et.col_scale = d->d_oscale;
    et.out_f32 = jout;
    et.ld_f32 = ld_jout;
    DINO_TRY(gemm(d, d->HS[3] + (int64_t)B * wdp, wdp, d->Wb[3], wdp, R, d->ru, wd, et));
  }
  return OUU_OK;
}

// Loss and gradient (into d_grad) for one minibatch.
static ouu_status loss_and_grad(ouu_dino* d, const float* xi, const float* z, const float* y, const float* jy,
                                const int* idx, int B) {
  const int wd = d->wd, wdp = d->wd, rup = pad8(d->ru), dz = d->dz, ru = d->ru;
  const int R = B * dz, BR = B + R;
  DINO_TRY(forward_tangent(d, xi, z, dz, idx, B, d->OUT + (int64_t)B * rup, rup, true));
  k_loss_out<<<LOSS_BLOCKS, 256, 0, d->stream>>>(d->OUT, rup, y, jy, idx, B, dz, ru, (float)d->desc.jac_weight,
                                                 d->d_oscale, d->GO, rup, d->d_gov, d->d_loss_part);
  k_sum_parts<<<1, 256, 0, d->stream>>>(d->d_loss_part, LOSS_BLOCKS, d->d_loss);
  transpose_bf16(d->GO, rup, BR, ru, d->GOT, BR, d->stream);
  float* g = d->d_grad;
  {  // output layer: dW3 = GO^T [h3; hdot3], db3 = sum_b g_phi, GH = GO W3
    DINO_TRY(gemm_wgrad(d, d->GOT, BR, d->HST[3], BR, ru, wd, BR, g + d->offW[3]));
    k_colsum<<<grid_for(ru), 256, 0, d->stream>>>(d->d_gov, B, ru, ru, g + d->offb[3]);
    EpiParams h = epi(EPI_LINEAR);
    h.out_f32 = d->GH;
    h.ld_f32 = wd;
    DINO_TRY(gemm(d, d->GO, rup, d->WTb[3], rup, BR, wd, ru, h));
  }
  for (int l = 3; l >= 2; --l) {   // activation l produced by weights l - 1
    k_bwd_layer<<<grid_for((int64_t)BR * wd), 256, 0, d->stream>>>(d->GH, d->A[l], d->AD[l], wdp, nullptr, 0, 0, dz,
                                                                   wd, B, d->GA, d->GAv);
    transpose_bf16(d->GA, wdp, BR, wd, d->GAT, BR, d->stream);
    DINO_TRY(gemm_wgrad(d, d->GAT, BR, d->HST[l - 1], BR, wd, wd, BR, g + d->offW[l - 1]));
    k_colsum<<<grid_for(wd), 256, 0, d->stream>>>(d->GAv, B, wd, wd, g + d->offb[l - 1]);
    EpiParams h = epi(EPI_LINEAR);
    h.out_f32 = d->GH;
    h.ld_f32 = wd;
    DINO_TRY(gemm(d, d->GA, wdp, d->WTb[l - 1], wdp, BR, wd, wd, h));
  }
  // first layer: value rows only feed dW0; the tangent term enters dW0's z columns.
  k_bwd_layer<<<grid_for((int64_t)B * wd), 256, 0, d->stream>>>(d->GH, d->A[1], nullptr, wdp,
                                                                d->d_params + d->offW[0], d->in0, d->rm, dz, wd, B,
                                                                d->GA, d->GAv);
  transpose_bf16(d->GA, wdp, B, wd, d->GA1T, B, d->stream);
  {
    EpiParams e = epi(EPI_LINEAR);
    e.out_f32 = g + d->offW[0];
    e.ld_f32 = d->in0;
    DINO_TRY(gemm(d, d->GA1T, B, d->X0T, B, wd, d->in0, B, e));
  }
  k_dw0z<<<grid_for((int64_t)dz * wd), 256, 0, d->stream>>>(d->A[1], d->GH, B, dz, wd, d->rm, d->in0,
                                                            g + d->offW[0]);
  k_colsum<<<grid_for(wd), 256, 0, d->stream>>>(d->GAv, B, wd, wd, g + d->offb[0]);
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

static ouu_status check_batch(ouu_dino* d, const float* xi, const float* z, const float* y, const float* jy,
                              const int32_t* idx, int batch) {
  OUU_CHECK_ARG(d && xi && z && y && jy && idx, "null argument");
  OUU_CHECK_ARG(batch >= 8 && batch <= d->maxB && batch % 8 == 0, "batch: multiple of 8 in [8, max_batch]");
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_train_step(ouu_dino_t d, const float* xi_dev, const float* z_dev, const float* y_dev,
                                          const float* jy_dev, const int32_t* idx_dev, int batch, float lr,
                                          double* loss_out) {
  DINO_TRY(check_batch(d, xi_dev, z_dev, y_dev, jy_dev, idx_dev, batch));
  OUU_CHECK_ARG(lr > 0 && std::isfinite(lr), "lr must be positive");
  d->val_ok = 0;
  DINO_TRY(loss_and_grad(d, xi_dev, z_dev, y_dev, jy_dev, idx_dev, batch));
  d->adam_t += 1;
  const double c1 = 1.0 - std::pow(0.9, d->adam_t), c2 = 1.0 - std::pow(0.999, d->adam_t);
  k_adam<<<grid_for((int64_t)d->n_params), 256, 0, d->stream>>>(d->d_params, d->d_grad, d->d_adam_m, d->d_adam_v,
                                                                 (int64_t)d->n_params, lr, 0.9f, 0.999f, 1e-8f,
                                                                 (float)c1, (float)c2);
  refresh_bf16_weights(d);
  OUU_CUDA_TRY(cudaGetLastError());
  if (loss_out) {
    OUU_CUDA_TRY(cudaMemcpyAsync(d->h_pin, d->d_loss, 8, cudaMemcpyDeviceToHost, d->stream));
    DINO_TRY(check_err(d));
    *loss_out = d->h_pin[0];
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_loss_grad(ouu_dino_t d, const float* xi_dev, const float* z_dev, const float* y_dev,
                                         const float* jy_dev, const int32_t* idx_dev, int batch, float* grad_host,
                                         double* loss_out) {
  DINO_TRY(check_batch(d, xi_dev, z_dev, y_dev, jy_dev, idx_dev, batch));
  DINO_TRY(loss_and_grad(d, xi_dev, z_dev, y_dev, jy_dev, idx_dev, batch));
  if (grad_host)
    OUU_CUDA_TRY(cudaMemcpyAsync(grad_host, d->d_grad, d->n_params * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->h_pin, d->d_loss, 8, cudaMemcpyDeviceToHost, d->stream));
  DINO_TRY(check_err(d));
  if (loss_out) *loss_out = d->h_pin[0];
  return OUU_OK;
}

// ------------------------------------------------------------------ evaluation
// Projection, forward values, reduced QoI (Qe) and, with want_grad, per-sample
// grad_z Q in GQe by reverse mode: seed phi + c through W3^T, GELU', ... , W0z^T.
static ouu_status dino_network(ouu_dino* d, int N, bool want_grad);

// The controls to the device and the projection of the fields into XIe.  With split (the risk
// evaluation's two-branch form): the projection launch carries the controls over from the
// pinned buffer (when it is mapped) instead of a copy ahead of it, and a captured graph gets
// the projection's event nodes.
static ouu_status dino_eval_inputs(ouu_dino* d, const double* m_dev, int N, const double* z_host, bool split = false) {
  ++d->eval_count;   // the per-sample buffers now belong to this evaluation
  float* zh = (float*)d->h_pin;
  for (int j = 0; j < d->dz; ++j) zh[j] = (float)z_host[j];
  const bool zstage = split && d->h_pin_dev;
  if (!zstage) OUU_CUDA_TRY(cudaMemcpyAsync(d->d_zf, zh, (size_t)d->dz * 4, cudaMemcpyHostToDevice, d->stream));
  DINO_TRY(project_fields(d, m_dev, N, d->XIe, true, zstage, split));
  return OUU_OK;
}

ouu_status dino_eval_core(ouu_dino* d, const double* m_dev, int N, const double* z_host, bool want_grad) {
  DINO_TRY(dino_eval_inputs(d, m_dev, N, z_host));
  return dino_network(d, N, want_grad);
}

ouu_status dino_eval_forward(ouu_dino* d, const double* m_dev, int N, const double* z_host, bool* split) {
  *split = d->fused_mlp == 2 && mlp_cluster_fits(d);
  if (d->capturing) d->graph_marks = *split;   // the captured graph holds the projection's event nodes
  if (!*split) return dino_eval_core(d, m_dev, N, z_host, true);
  DINO_TRY(dino_eval_inputs(d, m_dev, N, z_host, true));
  DINO_TRY(mlp_cluster_eval(d, N, 0, 4));
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

ouu_status dino_eval_reverse(ouu_dino* d, int N) {
  DINO_TRY(mlp_cluster_eval(d, N, 4, 8));
  if (!d->capturing) OUU_CUDA_TRY(cudaEventRecord(d->ev[3], d->stream));
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

// The network from the projection coordinates in XIe and the controls in d_zf.
static ouu_status dino_network(ouu_dino* d, int N, bool want_grad) {
  const int wd = d->wd, wdp = d->wd, rup = pad8(d->ru), in0p = d->inp_l[0], dz = d->dz, dzp = pad8(d->dz);
  if (want_grad && ((d->fused_mlp == 1 && mlp_fused_fits(d)) || (d->fused_mlp == 2 && mlp_cluster_fits(d)))) {
    // the whole network in one kernel
    DINO_TRY(d->fused_mlp == 2 ? mlp_cluster_eval(d, N) : mlp_fused_eval(d, N));
    if (!d->capturing) OUU_CUDA_TRY(cudaEventRecord(d->ev[3], d->stream));
    OUU_CUDA_TRY(cudaGetLastError());
    return OUU_OK;
  }
  OUU_CUDA_TRY(launch_pdl(k_build_x0, dim3(grid_for((int64_t)N * (in0p / 4))), dim3(256), 0, d->stream,
                          (const float*)d->XIe, (const int*)nullptr, (const float*)d->d_zf, (int64_t)0, d->rm, dz, in0p,
                          N, d->X0e, (__nv_bfloat16*)nullptr));
  __nv_bfloat16* hin = d->X0e;
  int ldin = in0p, kin = d->in0;
  __nv_bfloat16* hbuf[2] = {d->He0, d->He1};
  for (int l = 0; l < 3; ++l) {   // Ae[l + 1] = gelu'(a_{l+1}) for the reverse pass
    EpiParams e = epi(EPI_GELU_D);
    e.bias = d->d_params + d->offb[l];
    e.out_f32 = d->Ae[l + 1];
    e.ld_f32 = wd;
    e.out_bf16 = hbuf[l & 1];
    e.ld_bf16 = wdp;
    DINO_TRY(gemm(d, hin, ldin, d->Wb[l], d->inp_l[l], N, wd, kin, e));
    hin = hbuf[l & 1];
    ldin = wdp;
    kin = wd;
  }
  {  // output layer with the reduced QoI (Sec. 3.3): phi, Q = 1/2 ||phi + c||^2 + const, seed s (phi + c)
    EpiParams e = epi(EPI_QOI);
    e.bias = d->d_params + d->offb[3];
    e.col_scale = d->d_oscale;
    e.col_add = d->d_cf;
    e.qconst = d->qconst;
    e.out_f32 = d->OUTe;
    e.ld_f32 = rup;
    e.out_bf16 = want_grad ? d->Ge : nullptr;
    e.ld_bf16 = rup;
    e.out_q = d->Qe;
    DINO_TRY(gemm(d, hin, wdp, d->Wb[3], wdp, N, d->ru, wd, e));
  }
  if (want_grad) {
    const __nv_bfloat16* gin = d->Ge;
    int ldg = rup, kg = d->ru;
    for (int l = 3; l >= 1; --l) {   // ga_l = s'(a_l) * (g W_l)
      EpiParams e = epi(EPI_SCALE);
      e.aux = d->Ae[l];
      e.ld_aux = wd;
      e.aux_rdiv = 1;
      e.out_bf16 = hbuf[l & 1];
      e.ld_bf16 = wdp;
      DINO_TRY(gemm(d, gin, ldg, d->WTb[l], d->outp_l[l], N, wd, kg, e));
      gin = hbuf[l & 1];
      ldg = wdp;
      kg = wd;
    }
    EpiParams e = epi(EPI_LINEAR);   // grad_z Q = ga_1 W0z
    e.out_f32 = d->GQe;
    e.ld_f32 = dzp;
    DINO_TRY(gemm(d, gin, wdp, d->WTb[0] + (int64_t)d->rm * d->outp_l[0], d->outp_l[0], N, dz, wd, e));
  }
  if (!d->capturing) OUU_CUDA_TRY(cudaEventRecord(d->ev[3], d->stream));
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_eval(ouu_dino_t d, const double* m_dev, int n_samples, const double* z_host,
                                    float* phi_dev, float* jphi_dev, double* q_dev, double* gradq_dev,
                                    float* u_dev) {
  OUU_CHECK_ARG(d && m_dev && z_host, "null argument");
  OUU_CHECK_ARG(d->bases_ready, "bases not built");
  OUU_CHECK_ARG(n_samples >= 1 && n_samples <= d->maxE, "n_samples outside [1, max_eval]");
  const int rup = pad8(d->ru), dz = d->dz, dzp = pad8(d->dz);
  DINO_TRY(dino_eval_core(d, m_dev, n_samples, z_host, gradq_dev != nullptr));
  if (phi_dev)
    k_copy_rows_f32<<<grid_for((int64_t)n_samples * d->ru), 256, 0, d->stream>>>(d->OUTe, rup, n_samples, d->ru,
                                                                                 phi_dev, d->ru);
  if (q_dev) OUU_CUDA_TRY(cudaMemcpyAsync(q_dev, d->Qe, (size_t)n_samples * 8, cudaMemcpyDeviceToDevice, d->stream));
  if (gradq_dev)
    k_f32_to_f64<<<grid_for((int64_t)n_samples * dz), 256, 0, d->stream>>>(d->GQe, dzp, n_samples, dz, gradq_dev);
  if (u_dev) DINO_TRY(dino_decode(d, d->OUTe, rup, n_samples, u_dev, d->d_qdec));
  if (jphi_dev) {
    // forward-mode Jacobian in chunks of max_batch samples (tangent rows go straight to jphi)
    float* zf = d->d_zf;
    for (int s0 = 0; s0 < n_samples; s0 += d->maxB) {
      const int cnt = std::min(d->maxB, n_samples - s0);
      DINO_TRY(forward_tangent(d, d->XIe + (int64_t)s0 * d->rm, zf, 0, nullptr, cnt,
                               jphi_dev + (int64_t)s0 * dz * d->ru, d->ru, false));
    }
  }
  OUU_CUDA_TRY(cudaGetLastError());
  return check_err(d);
}

extern "C" ouu_status ouu_kernel_dino_network(ouu_dino_t d, const float* xi_dev, int n_samples, const double* z_host,
                                              int mode, double* q_dev, float* phi_dev, double* gradq_dev) {
  OUU_CHECK_ARG(d && xi_dev && z_host, "null argument");
  OUU_CHECK_ARG(d->bases_ready, "bases not built");
  OUU_CHECK_ARG(n_samples >= 1 && n_samples <= d->maxE, "n_samples outside [1, max_eval]");
  OUU_CHECK_ARG(mode >= 0 && mode <= 2, "network mode: 0, 1 or 2");
  const int rup = pad8(d->ru), dz = d->dz, dzp = pad8(d->dz);
  float* zh = (float*)d->h_pin;
  for (int j = 0; j < dz; ++j) zh[j] = (float)z_host[j];
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_zf, zh, (size_t)dz * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->XIe, xi_dev, (size_t)n_samples * d->rm * 4, cudaMemcpyDeviceToDevice, d->stream));
  ++d->eval_count;
  const int saved = d->fused_mlp;
  d->fused_mlp = mode;
  const ouu_status st = dino_network(d, n_samples, gradq_dev != nullptr);
  d->fused_mlp = saved;
  DINO_TRY(st);
  if (phi_dev)
    k_copy_rows_f32<<<grid_for((int64_t)n_samples * d->ru), 256, 0, d->stream>>>(d->OUTe, rup, n_samples, d->ru,
                                                                                 phi_dev, d->ru);
  if (q_dev) OUU_CUDA_TRY(cudaMemcpyAsync(q_dev, d->Qe, (size_t)n_samples * 8, cudaMemcpyDeviceToDevice, d->stream));
  if (gradq_dev)
    k_f32_to_f64<<<grid_for((int64_t)n_samples * dz), 256, 0, d->stream>>>(d->GQe, dzp, n_samples, dz, gradq_dev);
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return check_err(d);
}

extern "C" ouu_status ouu_dino_set_output_scale(ouu_dino_t d, const float* s_host) {
  OUU_CHECK_ARG(d && s_host, "null argument");
  for (int r = 0; r < d->ru; ++r) OUU_CHECK_ARG(s_host[r] > 0 && std::isfinite(s_host[r]), "scales must be positive");
  d->val_ok = 0;
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_oscale, s_host, (size_t)d->ru * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_get_output_scale(ouu_dino_t d, float* s_host) {
  OUU_CHECK_ARG(d && s_host, "null argument");
  OUU_CUDA_TRY(cudaMemcpyAsync(s_host, d->d_oscale, (size_t)d->ru * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

// ------------------------------------------------------------------ checkpoint
// File: the 8 bytes "OUUDINO1", a CkptHead, then FP32 parameters, Adam first and second
// moments [n_params] each, FP32 output scale [r_u], and with bases FP64 Phi [r_u][n n] and
// ubar [n n]; all little-endian, as both supported hosts (x86-64, aarch64) store them.
static const char kCkptMagic[8] = {'O', 'U', 'U', 'D', 'I', 'N', 'O', '1'};
struct CkptHead {
  int32_t version, n, lattice_L, r_m, r_u, width, adam_t, bases_ready;
  double gamma, delta, m_mean;
  uint64_t n_params;
};
static_assert(sizeof(CkptHead) == 64, "checkpoint header without padding");

extern "C" ouu_status ouu_dino_save(ouu_dino_t d, const char* path) {
  OUU_CHECK_ARG(d && path, "null argument");
  const size_t np = d->n_params, ru = (size_t)d->ru, nn = (size_t)d->nn;
  std::vector<float> prm(np), am(np), av(np), sc(ru);
  std::vector<double> phi(d->bases_ready ? ru * nn : 0), ub(d->bases_ready ? nn : 0);
  OUU_CUDA_TRY(cudaMemcpyAsync(prm.data(), d->d_params, np * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(am.data(), d->d_adam_m, np * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(av.data(), d->d_adam_v, np * 4, cudaMemcpyDeviceToHost, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(sc.data(), d->d_oscale, ru * 4, cudaMemcpyDeviceToHost, d->stream));
  if (d->bases_ready) {
    OUU_CUDA_TRY(cudaMemcpyAsync(phi.data(), d->d_phi64, ru * nn * 8, cudaMemcpyDeviceToHost, d->stream));
    OUU_CUDA_TRY(cudaMemcpyAsync(ub.data(), d->d_ubar, nn * 8, cudaMemcpyDeviceToHost, d->stream));
  }
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  CkptHead h;
  std::memset(&h, 0, sizeof(h));
  h.version = 1;
  h.n = d->n;
  h.lattice_L = d->desc.lattice_L;
  h.r_m = d->rm;
  h.r_u = d->ru;
  h.width = d->wd;
  h.adam_t = d->adam_t;
  h.bases_ready = d->bases_ready ? 1 : 0;
  h.gamma = d->desc.gamma;
  h.delta = d->desc.delta;
  h.m_mean = d->desc.m_mean;
  h.n_params = np;
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    ouu_set_error(std::string("cannot open ") + path + " for writing");
    return OUU_ERR_INVALID_ARG;
  }
  bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof(h), 1, f) == 1 &&
            std::fwrite(prm.data(), 4, np, f) == np && std::fwrite(am.data(), 4, np, f) == np &&
            std::fwrite(av.data(), 4, np, f) == np && std::fwrite(sc.data(), 4, ru, f) == ru &&
            std::fwrite(phi.data(), 8, phi.size(), f) == phi.size() && std::fwrite(ub.data(), 8, ub.size(), f) == ub.size();
  ok = std::fclose(f) == 0 && ok;
  if (!ok) {
    ouu_set_error(std::string("writing ") + path + " failed");
    return OUU_ERR_INVALID_ARG;
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_load(ouu_dino_t d, const char* path) {
  OUU_CHECK_ARG(d && path, "null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    ouu_set_error(std::string("cannot open ") + path);
    return OUU_ERR_INVALID_ARG;
  }
  char magic[8];
  CkptHead h;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            std::fread(&h, sizeof(h), 1, f) == 1 && h.version == 1;
  if (!ok) {
    std::fclose(f);
    ouu_set_error(std::string(path) + " is not a network checkpoint");
    return OUU_ERR_INVALID_ARG;
  }
  if (h.n != d->n || h.lattice_L != d->desc.lattice_L || h.r_m != d->rm || h.r_u != d->ru || h.width != d->wd ||
      h.gamma != d->desc.gamma || h.delta != d->desc.delta || h.m_mean != d->desc.m_mean ||
      h.n_params != (uint64_t)d->n_params || h.adam_t < 0 || (h.bases_ready != 0 && h.bases_ready != 1)) {
    std::fclose(f);
    ouu_set_error(std::string(path) + " holds a network of other sizes or another prior");
    return OUU_ERR_INVALID_ARG;
  }
  const size_t np = d->n_params, ru = (size_t)d->ru, nn = (size_t)d->nn;
  std::vector<float> prm(np), am(np), av(np), sc(ru);
  std::vector<double> phi(h.bases_ready ? ru * nn : 0), ub(h.bases_ready ? nn : 0);
  ok = std::fread(prm.data(), 4, np, f) == np && std::fread(am.data(), 4, np, f) == np &&
       std::fread(av.data(), 4, np, f) == np && std::fread(sc.data(), 4, ru, f) == ru &&
       std::fread(phi.data(), 8, phi.size(), f) == phi.size() && std::fread(ub.data(), 8, ub.size(), f) == ub.size() &&
       std::fgetc(f) == EOF;   // nothing after the last array
  std::fclose(f);
  if (!ok) {
    ouu_set_error(std::string(path) + " is truncated or longer than its header says");
    return OUU_ERR_INVALID_ARG;
  }
  for (size_t r = 0; r < ru; ++r) OUU_CHECK_ARG(sc[r] > 0 && std::isfinite(sc[r]), "checkpoint: output scale not positive");
  d->val_ok = 0;
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_params, prm.data(), np * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_adam_m, am.data(), np * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_adam_v, av.data(), np * 4, cudaMemcpyHostToDevice, d->stream));
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_oscale, sc.data(), ru * 4, cudaMemcpyHostToDevice, d->stream));
  d->adam_t = h.adam_t;
  refresh_bf16_weights(d);
  OUU_CUDA_TRY(cudaGetLastError());
  if (h.bases_ready) {
    OUU_CUDA_TRY(cudaMemcpyAsync(d->d_phi64, phi.data(), ru * nn * 8, cudaMemcpyHostToDevice, d->stream));
    OUU_CUDA_TRY(cudaMemcpyAsync(d->d_ubar, ub.data(), nn * 8, cudaMemcpyHostToDevice, d->stream));
    return dino_install_bases(d);   // synchronises before the host buffers go
  }
  d->bases_ready = 0;   // the checkpoint was taken before the bases existed
  OUU_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_set_fused_network(ouu_dino_t d, int mode) {
  OUU_CHECK_ARG(d != nullptr, "null argument");
  OUU_CHECK_ARG(mode >= 0 && mode <= 2, "network mode: 0 per-layer kernels, 1 one kernel, 2 clusters");
  d->fused_mlp = mode;
  if (d->gexec) {   // a captured evaluation holds the other path's kernels
    cudaGraphExecDestroy(d->gexec);
    d->gexec = nullptr;
  }
  return OUU_OK;
}

extern "C" ouu_status ouu_dino_set_graphs(ouu_dino_t d, int enable) {
  OUU_CHECK_ARG(d != nullptr, "null argument");
  d->use_graphs = enable ? 1 : 0;
  if (!enable && d->gexec) {
    cudaGraphExecDestroy(d->gexec);
    d->gexec = nullptr;
  }
  return OUU_OK;
}
