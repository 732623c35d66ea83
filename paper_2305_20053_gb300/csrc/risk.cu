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

// Smoothed plus function (Sec. 2.1) and its derivative, written with y = x / eps:
// s = eps (y^3 - y^4 / 2), s' = 3 y^2 - 2 y^3 on (0, eps); no division per sample.
static __device__ __forceinline__ double splus(double x, double eps, double inv_eps) {
  if (x <= 0.0) return 0.0;
  if (x < eps) {
    const double y = x * inv_eps;
    return eps * y * y * y * (1.0 - 0.5 * y);
  }
  return x - 0.5 * eps;
}

static __device__ __forceinline__ double splus_d1(double x, double eps, double inv_eps) {
  if (x <= 0.0) return 0.0;
  if (x < eps) {
    const double y = x * inv_eps;
    return y * y * (3.0 - 2.0 * y);
  }
  return 1.0;
}

static __device__ double cvar_dt(const BlockRed& br, const double* q, int N, double t, double beta, double eps) {
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += splus_d1(q[i] - t, eps, 1.0 / eps);
  return 1.0 - br.sum(s) / ((double)N * (1.0 - beta));
}

// Order-preserving map of a double to an unsigned 64-bit key, and back.
static __device__ __forceinline__ uint64_t dkey(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
static __device__ __forceinline__ double dval(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

// k-th largest (1-based) of q[0, N) by block-wide 8-bit radix select on the keys.  With
// N <= KPT * blockDim.x the keys stay in registers across the eight passes.
template <int KPT>
static __device__ double kth_largest(const double* q, int N, int k, unsigned* hist, unsigned* sel) {
  uint64_t prefix = 0, mask = 0;
  unsigned kk = (unsigned)k;
  const int lane = threadIdx.x & 31;
  const bool regs = N <= KPT * (int)blockDim.x;
  uint64_t kr[KPT];
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int i = j * blockDim.x + threadIdx.x;
    kr[j] = (regs && i < N) ? dkey(q[i]) : 0ull;
  }
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    for (int i0 = 0, j = 0; i0 < N; i0 += blockDim.x, ++j) {   // warp-uniform trip count for __match_any_sync
      const int i = i0 + threadIdx.x;
      uint64_t key = 0;
      bool in = false;
      if (i < N) {
        if (regs) {
#pragma unroll
          for (int jj = 0; jj < KPT; ++jj)
            if (jj == j) key = kr[jj];
        } else {
          key = dkey(q[i]);
        }
        in = (key & mask) == prefix;
      }
      const unsigned bin = in ? (unsigned)((key >> shift) & 255u) : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, bin);   // lanes sharing a bin add once
      if (in && (threadIdx.x & 31) == (__ffs(peers) - 1)) atomicAdd(&hist[bin], (unsigned)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // lane L owns buckets 255-8L .. 248-8L (descending); prefix sums from the top
      unsigned loc[8], s = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        loc[j] = hist[255 - 8 * lane - j];
        s += loc[j];
      }
      unsigned incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const unsigned excl = incl - s;
      if (excl < kk && kk <= incl) {
        unsigned cum = excl;
        for (int j = 0; j < 8; ++j) {
          if (cum + loc[j] >= kk) {
            sel[0] = 255u - 8u * lane - j;
            sel[1] = kk - cum;
            break;
          }
          cum += loc[j];
        }
      }
    }
    __syncthreads();
    prefix |= (uint64_t)sel[0] << shift;
    mask |= (uint64_t)0xFF << shift;
    kk = sel[1];
    __syncthreads();
  }
  return dval(prefix);
}

#define RISK_WINDOW_MAX 2048
#define RISK_BLOCKS 148

// Pass 1 (many CTAs): per-block partial sums of Q and Q^2 (deterministic order).
__global__ void k_risk_moments(const double* __restrict__ q, int N, double* __restrict__ part) {
  __shared__ double red[40];
  BlockRed br{red};
  double s = 0.0, s2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double v = q[i];
    s += v;
    s2 += v * v;
  }
  const double ts = br.sum(s);
  const double ts2 = br.sum(s2);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ts;
    part[2 * blockIdx.x + 1] = ts2;
  }
}

// Pass 2 (one CTA): moments and, per CVaR risk, t* = argmin_t rho(z, t).
// With K = N (1 - beta), k0 = floor(K) and v the (k0 + 1)-th largest QoI (the N-th
// when k0 = N), the root of d rho/dt = 1 - S(t)/K, S(t) = sum_i s'_eps(Q_i - t), lies
// in [v - eps, v]: there every Q_i >= v + eps contributes exactly 1 and every
// Q_i <= v - eps exactly 0, so S(t) = C + sum over the window v - eps < Q_i < v + eps
// (v itself is in it).  The window test runs on order-preserving integer keys.  In the
// window coordinates y_i = (Q_i - v)/eps and t = v - eps theta, S = C + sum s'(y_i + theta)
// with s'(y) = y^2 (3 - 2y) on (0, 1): an FP32 bisection on theta in [0, 1] brackets the
// root, and an FP64 Illinois regula falsi (bracketing, so safe where S is flat) takes the
// bracket down to adjacent doubles; the end rule is that of a plain bisection over
// [min Q - eps, max Q]: lo if d rho/dt(lo) >= 0, else hi.  (Every FP64 instruction
// occupies GB300's narrow FP64 pipe for a whole warp, so most of the search runs in FP32
// and the window is spread over the lanes of one warp.)  params[r] = {t, mean, var}.
__global__ void k_risk_select(const double* __restrict__ q, int N, const double* __restrict__ part, int nparts,
                              const RiskDev* __restrict__ risks, int n_risks, double* __restrict__ params) {
  __shared__ double red[40];
  __shared__ unsigned hist[256];
  __shared__ unsigned sel[2];
  __shared__ double win[RISK_WINDOW_MAX];
  __shared__ int nwin;
  __shared__ double s_t;
  BlockRed br{red};
  double s = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    s += part[2 * i];
    s2 += part[2 * i + 1];
  }
  const double qbar = br.sum(s) / N;
  const double var = fmax(br.sum(s2) / N - qbar * qbar, 0.0);
  const int lane = threadIdx.x & 31;
  for (int r = 0; r < n_risks; ++r) {
    const RiskDev R = risks[r];
    double t = R.t;
    if (R.kind == OUU_RISK_CVAR_SMOOTH && R.t_optimal) {
      const double eps = R.eps, ie = 1.0 / eps;
      const double K = (double)N * (1.0 - R.beta);
      int kq = (int)floor(K) + 1;
      if (kq > N) kq = N;
      if (kq < 1) kq = 1;
      const double v = kth_largest<8>(q, N, kq, hist, sel);
      const uint64_t khi = dkey(v + eps), klo = dkey(v - eps);
      if (threadIdx.x == 0) nwin = 0;
      __syncthreads();
      unsigned cnt = 0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const uint64_t k = dkey(q[i]);
        if (k >= khi) cnt += 1u;
        else if (k > klo) {
          const int slot = atomicAdd(&nwin, 1);
          if (slot < RISK_WINDOW_MAX) win[slot] = q[i];
        }
      }
      const double C = br.sum((double)cnt);
      const int W = nwin;
      if (W <= RISK_WINDOW_MAX) {
        if (threadIdx.x < 32) {
          // FP32 bisection on theta (S(theta) = C + sum s'(y_i + theta) is non-decreasing):
          // compares the window sum against K - C so that tiny targets keep their precision.
          const float Tf = (float)(K - C);
          float th_lo = 0.f, th_hi = 1.f;
          for (int it = 0; it < 40; ++it) {
            const float mid = 0.5f * (th_lo + th_hi);
            if (mid <= th_lo || mid >= th_hi) break;
            float sp = 0.f;
            for (int i = lane; i < W; i += 32) {
              const float y = (float)((win[i] - v) * ie) + mid;
              sp += y <= 0.f ? 0.f : (y >= 1.f ? 1.f : y * y * (3.f - 2.f * y));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
            if (sp < Tf) th_lo = mid;
            else th_hi = mid;
          }
          // FP64 on G(t) = (K - C) - S_window(t), which has the sign of d rho/dt = 1 - S(t)/K
          // without a division: bracket check, then Illinois regula falsi (secant ratio in
          // FP32) until the bracket (lo: G < 0, hi: G >= 0) is a few ulps wide.
          const double KC = K - C;
          auto G = [&](double tt) {
            double S = 0.0;
            for (int i = lane; i < W; i += 32) S += splus_d1(win[i] - tt, eps, ie);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
            return KC - S;
          };
          double lo = v - eps * (double)th_hi, hi = v - eps * (double)th_lo;
          double glo = G(lo), ghi = G(hi);
          if (!(glo < 0.0)) {
            lo = v - eps;
            glo = G(lo);
          }
          if (!(ghi >= 0.0)) {
            hi = v;
            ghi = G(hi);
          }
          int side = 0;
          for (int it = 0; it < 60 && glo < 0.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi || hi - lo <= 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi))) break;
            const float ratio = (float)ghi / ((float)ghi - (float)glo);
            double c = hi - (double)ratio * (hi - lo);
            if (!(c > lo && c < hi)) c = mid;
            const double gc = G(c);
            if (gc < 0.0) {
              lo = c;
              glo = gc;
              if (side == -1) ghi *= 0.5;
              side = -1;
            } else {
              hi = c;
              ghi = gc;
              if (side == 1) glo *= 0.5;
              side = 1;
            }
          }
          const double tt = glo >= 0.0 ? lo : hi;
          if (threadIdx.x == 0) s_t = tt;
        }
        __syncthreads();
        t = s_t;
      } else {
        double lo = v - eps, hi = v;
        for (int it = 0; it < 200; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          if (cvar_dt(br, q, N, mid, R.beta, eps) < 0.0) lo = mid;
          else hi = mid;
        }
        t = cvar_dt(br, q, N, lo, R.beta, eps) >= 0.0 ? lo : hi;
      }
    }
    if (threadIdx.x == 0) {
      params[3 * r + 0] = t;
      params[3 * r + 1] = qbar;
      params[3 * r + 2] = var;
    }
    __syncthreads();
  }
}

// Pass 3 (many CTAs): weights w[r][i] and per-block partial sums of s_eps and s'_eps.
__global__ void k_risk_apply(const double* __restrict__ q, int N, const RiskDev* __restrict__ risks, int n_risks,
                             const double* __restrict__ params, double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[40];
  BlockRed br{red};
  for (int r = 0; r < n_risks; ++r) {
    const RiskDev R = risks[r];
    const double t = params[3 * r], qbar = params[3 * r + 1];
    double* wr = w + (int64_t)r * N;
    double sv = 0.0, sd = 0.0;
    if (R.kind == OUU_RISK_MEAN_VAR) {
      const double invN = 1.0 / N, k2 = 2.0 * R.kappa;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        wr[i] = (1.0 + k2 * (q[i] - qbar)) * invN;
    } else {
      const double scale = 1.0 / ((double)N * (1.0 - R.beta)), ie = 1.0 / R.eps;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double x = q[i] - t;
        const double d1 = splus_d1(x, R.eps, ie);
        wr[i] = d1 * scale;
        sv += splus(x, R.eps, ie);
        sd += d1;
      }
    }
    const double tv = br.sum(sv);
    const double td = br.sum(sd);
    if (threadIdx.x == 0) {
      part[(2 * r) * gridDim.x + blockIdx.x] = tv;
      part[(2 * r + 1) * gridDim.x + blockIdx.x] = td;
    }
  }
}

// Pass 4 (one CTA): risk values and d rho / dt.  out[3r..3r+2] = value, dt, t.
__global__ void k_risk_finish(int N, const RiskDev* __restrict__ risks, int n_risks, const double* __restrict__ params,
                              const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double red[40];
  BlockRed br{red};
  for (int r = 0; r < n_risks; ++r) {
    const RiskDev R = risks[r];
    double sv = 0.0, sd = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
      sv += part[(2 * r) * nparts + i];
      sd += part[(2 * r + 1) * nparts + i];
    }
    const double tv = br.sum(sv), td = br.sum(sd);
    if (threadIdx.x == 0) {
      const double t = params[3 * r], qbar = params[3 * r + 1], var = params[3 * r + 2];
      if (R.kind == OUU_RISK_MEAN_VAR) {
        out[3 * r + 0] = qbar + R.kappa * var;
        out[3 * r + 1] = 0.0;
        out[3 * r + 2] = 0.0;
      } else {
        const double scale = 1.0 / ((double)N * (1.0 - R.beta));
        out[3 * r + 0] = t + tv * scale;
        out[3 * r + 1] = 1.0 - td * scale;
        out[3 * r + 2] = t;
      }
    }
    __syncthreads();
  }
}

void launch_risk_weights(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* out,
                         double* scratch, cudaStream_t s) {
  static_assert(OUU_RISK_SCRATCH >= 3 * OUU_MAX_RISKS + 2 * OUU_MAX_RISKS * RISK_BLOCKS, "risk scratch size");
  double* params = scratch;
  double* part = scratch + 3 * OUU_MAX_RISKS;
  k_risk_moments<<<RISK_BLOCKS, 256, 0, s>>>(q, N, part);
  k_risk_select<<<1, 1024, 0, s>>>(q, N, part, RISK_BLOCKS, risks_dev, n_risks, params);
  k_risk_apply<<<RISK_BLOCKS, 256, 0, s>>>(q, N, risks_dev, n_risks, params, w, part);
  k_risk_finish<<<1, 256, 0, s>>>(N, risks_dev, n_risks, params, part, RISK_BLOCKS, out);
}
