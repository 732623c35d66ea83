// Risk weights over the sample average (Sec. 2.1-2.2): one CTA reduces the N
// per-sample QoIs, finds the CVaR minimiser t* when asked, and writes the weight
// w_i of every sample, so that grad rho = sum_i w_i grad Q_i.
//   mean + kappa var:  w_i = (1 + 2 kappa (Q_i - Qbar)) / N
//   smoothed CVaR:     w_i = s'_eps(Q_i - t) / (N (1 - beta))
#include "ouu_internal.cuh"

struct BlockRed {
  double* red;
  __device__ double sum(double v) const {
    CtaCtx c{red};
    return c.sum_d(v);
  }
  __device__ double minv(double v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
      double s = l < (int)(blockDim.x >> 5) ? red[l] : INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = fmin(s, __shfl_xor_sync(0xffffffffu, s, o));
      if (l == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
  }
};

static __device__ __forceinline__ double splus(double x, double eps) {
  if (x <= 0.0) return 0.0;
  if (x < eps) return x * x * x / (eps * eps) - x * x * x * x / (2.0 * eps * eps * eps);
  return x - 0.5 * eps;
}

static __device__ __forceinline__ double splus_d1(double x, double eps) {
  if (x <= 0.0) return 0.0;
  if (x < eps) return 3.0 * x * x / (eps * eps) - 2.0 * x * x * x / (eps * eps * eps);
  return 1.0;
}

static __device__ double cvar_dt(const BlockRed& br, const double* q, int N, double t, double beta, double eps) {
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += splus_d1(q[i] - t, eps);
  return 1.0 - br.sum(s) / ((double)N * (1.0 - beta));
}

__global__ void k_risk_weights(const double* q, int N, const RiskDev* risks, int n_risks, double* w, double* out) {
  __shared__ double red[40];
  BlockRed br{red};
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += q[i];
  const double qbar = br.sum(s) / N;
  double v = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) v += (q[i] - qbar) * (q[i] - qbar);
  const double var = br.sum(v) / N;
  for (int r = 0; r < n_risks; ++r) {
    const RiskDev R = risks[r];
    double* wr = w + (int64_t)r * N;
    if (R.kind == OUU_RISK_MEAN_VAR) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) wr[i] = (1.0 + 2.0 * R.kappa * (q[i] - qbar)) / N;
      if (threadIdx.x == 0) {
        out[3 * r + 0] = qbar + R.kappa * var;
        out[3 * r + 1] = 0.0;
        out[3 * r + 2] = 0.0;
      }
    } else {
      double t = R.t;
      const double scale = 1.0 / ((double)N * (1.0 - R.beta));
      if (R.t_optimal) {
        double mn = INFINITY, mx = -INFINITY;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          mn = fmin(mn, q[i]);
          mx = fmax(mx, q[i]);
        }
        double lo = br.minv(mn) - R.eps;
        double hi = -br.minv(-mx);
        for (int it = 0; it < 200; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          if (cvar_dt(br, q, N, mid, R.beta, R.eps) < 0.0) lo = mid;
          else hi = mid;
        }
        t = cvar_dt(br, q, N, lo, R.beta, R.eps) >= 0.0 ? lo : hi;
      }
      double sv = 0.0, sd = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double d1 = splus_d1(q[i] - t, R.eps);
        wr[i] = d1 * scale;
        sv += splus(q[i] - t, R.eps);
        sd += d1;
      }
      const double tv = br.sum(sv);
      const double td = br.sum(sd);
      if (threadIdx.x == 0) {
        out[3 * r + 0] = t + tv * scale;
        out[3 * r + 1] = 1.0 - td * scale;
        out[3 * r + 2] = t;
      }
    }
    __syncthreads();
  }
}

void launch_risk_weights(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* out,
                         cudaStream_t s) {
  k_risk_weights<<<1, 1024, 0, s>>>(q, N, risks_dev, n_risks, w, out);
}
