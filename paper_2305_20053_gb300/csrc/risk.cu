// Risk values and weights over the sample average (Sec. 2.1-2.2), in three passes: the
// moments of the N per-sample QoIs (many CTAs; or sums a caller already has), then one CTA
// that finds the CVaR minimiser t* when asked and computes the risk values, then the weight
// w_i of every sample (many CTAs), with sum_i w_i grad Q_i when per-sample gradients are
// given, so that grad rho = sum_i w_i grad Q_i.
//   mean + kappa var:  w_i = (1 + 2 kappa (Q_i - Qbar)) / N
//   smoothed CVaR:     w_i = s'_eps(Q_i - t) / (N (1 - beta))
#include "ouu_internal.cuh"
#include "ouu_kernels.h"

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

// Warp sum of v over lanes [0, 2^k) where 2^k >= active (active <= 32): the butterfly runs only
// as deep as the data, then lane 0's total is broadcast.  (FP64 adds are expensive on
// GB300's narrow FP64 pipe; a window of one sample needs none.)
static __device__ __forceinline__ double warp_sum_active(double v, int active) {
  for (int o = 1; o < active && o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}
static __device__ __forceinline__ float warp_sum_active_f(float v, int active) {
  for (int o = 1; o < active && o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Block sums of a and b over threads [0, nact) (the other threads' values are not read):
// the values pass through shared memory and warp 0 adds them, nact/32 + 5 FP64 adds per
// lane of one warp instead of a shuffle tree on every warp (each FP64 warp instruction
// holds GB300's narrow FP64 pipe for many cycles).  buf holds 2 blockDim.x + 2 doubles.
// Every thread gets both sums.
static __device__ void block_sum2(double& a, double& b, double* buf, int nact) {
  const int n = blockDim.x;
  if ((int)threadIdx.x < nact) {
    buf[threadIdx.x] = a;
    buf[n + threadIdx.x] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < nact; i += 32) {
      sa += buf[i];
      sb += buf[n + i];
    }
    sa = warp_sum_active(sa, nact < 32 ? nact : 32);
    sb = warp_sum_active(sb, nact < 32 ? nact : 32);
    if (threadIdx.x == 0) {
      buf[2 * n] = sa;
      buf[2 * n + 1] = sb;
    }
  }
  __syncthreads();
  a = buf[2 * n];
  b = buf[2 * n + 1];
  __syncthreads();   // buf may be reused at once
}

// Pass 1 (many CTAs): per-block partial sums of Q and Q^2 (deterministic order).
__global__ void k_risk_moments(const double* __restrict__ q, int N, double* __restrict__ part) {
  __shared__ double buf[2 * 256 + 2];
  pdl_wait();
  double s = 0.0, s2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double v = q[i];
    s += v;
    s2 += v * v;
  }
  // threads that hold samples: all when N covers the grid, else those below N in the first pass
  const long long first = (long long)blockIdx.x * blockDim.x;
  const int nact = N >= (long long)gridDim.x * blockDim.x ? (int)blockDim.x
                                                          : (int)max(0ll, min((long long)blockDim.x, N - first));
  if (nact > 0) block_sum2(s, s2, buf, nact);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = nact > 0 ? s : 0.0;
    part[2 * blockIdx.x + 1] = nact > 0 ? s2 : 0.0;
  }
}

// Top 32 bits of the order-preserving keys of q[0, N), N <= KEYS_PER_THREAD * blockDim.x.
#define KEYS_PER_THREAD 16
static __device__ __forceinline__ void load_key_prefixes(const double* q, int N, uint32_t (&kr)[KEYS_PER_THREAD]) {
#pragma unroll
  for (int j = 0; j < KEYS_PER_THREAD; ++j) {
    const int i = j * blockDim.x + threadIdx.x;
    kr[j] = i < N ? (uint32_t)(dkey(q[i]) >> 32) : 0u;
  }
}

// k-th largest (1-based) of q[0, N) for N <= 16 * blockDim.x (blockDim.x = 1024), on the
// top 32 bits of the order-preserving keys (held in registers).  The bits above the keys'
// highest difference are common to all; radix digits of at most 11 bits follow from there
// down, each narrowing the prefix to the bin that holds rank k, until at most 32 keys share
// it; the answer is then chosen exactly among those samples by their full 64-bit keys.
// *ok = false when more than 32 samples share all 32 bits (the caller falls back).
static __device__ double kth_largest_prefix(const double* q, int N, int k, const uint32_t (&kr)[KEYS_PER_THREAD],
                                            unsigned* hist, unsigned* sel, double* cand, int* ncand, bool* ok) {
  constexpr int KPT = KEYS_PER_THREAD;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t ka = 0xFFFFFFFFu, ko = 0u;
#pragma unroll
  for (int j = 0; j < KPT; ++j)
    if (j * (int)blockDim.x + (int)threadIdx.x < N) {
      ka &= kr[j];
      ko |= kr[j];
    }
  ka = __reduce_and_sync(0xffffffffu, ka);
  ko = __reduce_or_sync(0xffffffffu, ko);
  if (threadIdx.x == 0) {
    sel[0] = 0xFFFFFFFFu;
    sel[1] = 0u;
  }
  __syncthreads();
  if (lane == 0) {
    atomicAnd(&sel[0], ka);
    atomicOr(&sel[1], ko);
  }
  __syncthreads();
  const uint32_t diff = sel[0] ^ sel[1];
  int top = diff ? 31 - __clz(diff) : -1;   // highest bit in which keys differ
  uint32_t mask = top >= 0 ? ~(0xFFFFFFFFu >> (31 - top)) : 0xFFFFFFFFu;
  uint32_t prefix = sel[0] & mask;
  unsigned kk = (unsigned)k, count = (unsigned)N;
  __syncthreads();
  while (count > 32u && top >= 0) {
    const int width = top + 1 < 11 ? top + 1 : 11, shift = top + 1 - width;
    const uint32_t dmask = (1u << width) - 1u;
    for (int b = threadIdx.x; b < 2048; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int i = j * blockDim.x + threadIdx.x;
      if (i < N && (kr[j] & mask) == prefix) atomicAdd(&hist[(kr[j] >> shift) & dmask], 1u);
    }
    __syncthreads();
    // descending bins: thread t owns bins 2047 - 2t and 2046 - 2t; block-wide exclusive scan
    unsigned h0 = 0, h1 = 0;
    if (2 * threadIdx.x < 2048) {
      h0 = hist[2047 - 2 * threadIdx.x];
      h1 = hist[2046 - 2 * threadIdx.x];
    }
    const unsigned c = h0 + h1;
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sel[2 + warp] = incl;   // warp totals
    __syncthreads();
    if (warp == 0) {
      unsigned wt = lane < nw ? sel[2 + lane] : 0u, wi = wt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      if (lane < nw) sel[2 + 32 + lane] = wi - wt;   // exclusive warp offsets
    }
    __syncthreads();
    const unsigned excl = sel[2 + 32 + warp] + incl - c;
    if (2 * threadIdx.x < 2048 && excl < kk && kk <= excl + c) {
      if (excl + h0 >= kk) {
        sel[0] = 2047u - 2u * threadIdx.x;
        sel[1] = kk - excl;
        sel[66] = h0;
      } else {
        sel[0] = 2046u - 2u * threadIdx.x;
        sel[1] = kk - excl - h0;
        sel[66] = h1;
      }
    }
    __syncthreads();
    prefix |= sel[0] << shift;
    mask |= dmask << shift;
    kk = sel[1];
    count = sel[66];
    top = shift - 1;
    __syncthreads();
  }
  *ok = count <= 32u;
  if (count > 32u) return 0.0;
  // the samples under the selected prefix; the answer is the kk-th largest of them
  if (threadIdx.x == 0) *ncand = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int i = j * blockDim.x + threadIdx.x;
    if (i < N && (kr[j] & mask) == prefix) {
      const int slot = atomicAdd(ncand, 1);
      if (slot < 32) cand[slot] = q[i];
    }
  }
  __syncthreads();
  const int nc = *ncand;
  if (warp == 0) {
    const uint64_t mine = lane < nc ? dkey(cand[lane]) : 0ull;
    unsigned rank = 0;
    for (int i = 0; i < nc; ++i) {
      const uint64_t o = dkey(cand[i]);
      rank += (o > mine || (o == mine && i < lane)) ? 1u : 0u;
    }
    if (lane < nc && rank == kk - 1) sel[0] = (unsigned)lane;
  }
  __syncthreads();
  return cand[sel[0]];
}

// sum_i s_eps(Q_i - t) and sum_i s'_eps(Q_i - t) over the N samples; every thread gets both.
// Only samples above t contribute.  With the key prefixes in registers (N <= 16 blockDim.x),
// the samples whose prefix is not below t's (the contributors and a few more) are gathered
// into list (in thread order, through a block-wide scan of their counts) and warp 0 alone
// does the FP64 arithmetic: a warp instruction holds GB300's narrow FP64 pipe whatever its
// number of active lanes, so FP64 work spread thinly over every warp would cost a pass of
// the pipe per warp.  More than lmax of them, or no prefixes: every thread takes its own
// samples and the sums go to warp 0 through list (2 blockDim.x + 2 doubles).  Fixed
// summation order either way.
static __device__ void cvar_sums(const double* q, int N, bool prefix_path, const uint32_t (&kr)[KEYS_PER_THREAD],
                                 double t, double eps, double inv_eps, double* list, int lmax, int* wtot,
                                 double* res, double& s, double& d) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  s = 0.0;
  d = 0.0;
  if (prefix_path) {
    const uint32_t tp = (uint32_t)(dkey(t) >> 32);
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < KEYS_PER_THREAD; ++j) {
      const int i = j * blockDim.x + threadIdx.x;
      if (i < N && kr[j] >= tp) mask |= 1u << j;
    }
    const int c = __popc(mask);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      const int v = wtot[w];
      base += w < warp ? v : 0;
      total += v;
    }
    if (total <= lmax) {
      int pos = base + inc - c;
#pragma unroll
      for (int j = 0; j < KEYS_PER_THREAD; ++j)
        if ((mask >> j) & 1u) list[pos++] = q[j * blockDim.x + threadIdx.x];
      __syncthreads();
      if (warp == 0) {
        for (int k = lane; k < total; k += 32) {
          const double x = list[k] - t;
          s += splus(x, eps, inv_eps);
          d += splus_d1(x, eps, inv_eps);
        }
        const int act = total < 32 ? total : 32;
        s = warp_sum_active(s, act);
        d = warp_sum_active(d, act);
        if (lane == 0) {
          res[0] = s;
          res[1] = d;
        }
      }
      __syncthreads();
      s = res[0];
      d = res[1];
      __syncthreads();   // list, wtot and res may be reused at once
      return;
    }
#pragma unroll
    for (int j = 0; j < KEYS_PER_THREAD; ++j)
      if ((mask >> j) & 1u) {
        const double x = q[j * blockDim.x + threadIdx.x] - t;
        s += splus(x, eps, inv_eps);
        d += splus_d1(x, eps, inv_eps);
      }
  } else {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double x = q[i] - t;
      if (x > 0.0) {
        s += splus(x, eps, inv_eps);
        d += splus_d1(x, eps, inv_eps);
      }
    }
  }
  block_sum2(s, d, list, blockDim.x);
}

// Pass 2 (one CTA): moments and, per CVaR risk, t* = argmin_t rho(z, t).
// With K = N (1 - beta), k0 = floor(K) and v the (k0 + 1)-th largest QoI (the N-th
// when k0 = N), the root of d rho/dt = 1 - S(t)/K, S(t) = sum_i s'_eps(Q_i - t), lies
// in [v - eps, v]: there every Q_i >= v + eps contributes exactly 1 and every
// Q_i <= v - eps exactly 0, so S(t) = C + sum over the window v - eps < Q_i < v + eps
// (v itself is in it).  The window test runs on order-preserving integer keys.  In the
// window coordinates y_i = (Q_i - v)/eps and t = v - eps theta, S = C + sum s'(y_i + theta)
// with s'(y) = y^2 (3 - 2y) on (0, 1), non-decreasing in theta: an FP32 Illinois regula
// falsi on theta in [0, 1] narrows the bracket, and an FP64 one (bracketing, so safe where
// S is flat) takes it to a few ulps; the end rule is that of a plain bisection over
// [min Q - eps, max Q]: lo if d rho/dt(lo) >= 0, else hi.  Every FP64 instruction occupies
// GB300's narrow FP64 pipe for a whole warp, so the FP64 work stays on one warp and the
// block-wide parts are integer.  params[r] = {t, mean, var}.
// Then the risk values from all N samples: out[3r..3r+2] = value, d rho / dt, t (mean +
// variance: Qbar + kappa var, 0, 0; CVaR: t + sum s_eps / K, 1 - sum s'_eps / K, t).
__global__ void __launch_bounds__(1024, 1) k_risk_select(const double* __restrict__ q, int N, const double* __restrict__ part, int nparts,
                              const RiskDev* __restrict__ risks, int n_risks, double* __restrict__ params,
                              double* __restrict__ out, double* __restrict__ zero_out, int n_zero) {
  __shared__ unsigned hist[2048];
  __shared__ unsigned sel[2 + 64 + 1];
  __shared__ double cand[32];
  __shared__ int ncand;
  __shared__ double win[RISK_WINDOW_MAX + 2];   // also the buffer of the value sums (2 x 1024 + 2)
  __shared__ float winf[RISK_WINDOW_MAX];
  __shared__ int nwin, s_above;
  __shared__ double s_par[6];   // qbar, var, -, v + eps, v - eps, t
  __shared__ bool s_ok;
  __shared__ double red[40];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pdl_wait();
  if (zero_out)   // the weighted-gradient sums of the next pass start from 0
    for (int i = threadIdx.x; i < n_zero; i += blockDim.x) zero_out[i] = 0.0;
  // key prefixes first (whether or not a t* is asked for): their loads are in flight while
  // the risk descriptors are read and warp 0 combines the moments
  const bool prefix_path = N <= KEYS_PER_THREAD * (int)blockDim.x;
  uint32_t kr[KEYS_PER_THREAD];
  if (prefix_path) load_key_prefixes(q, N, kr);
  if (warp == 0) {   // moments from the per-block partial sums
    double s = 0.0, s2 = 0.0;
    for (int i = lane; i < nparts; i += 32) {
      s += part[2 * i];
      s2 += part[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      const double invN = risks[0].inv_N;   // 1/N from the host (an FP64 division is long on the narrow pipe)
      s_par[0] = s * invN;
      s_par[1] = fmax(s2 * invN - s_par[0] * s_par[0], 0.0);
    }
  }
  __syncthreads();
  const double qbar = s_par[0], var = s_par[1];
  for (int r = 0; r < n_risks; ++r) {
    const RiskDev R = risks[r];
    double t = R.t;
    if (R.kind == OUU_RISK_CVAR_SMOOTH && R.t_optimal) {
      const double eps = R.eps, ie = R.inv_eps;
      const int kq = R.kq;
      double v = 0.0;
      bool okp = false;
      if (prefix_path) {
        v = kth_largest_prefix(q, N, kq, kr, hist, sel, cand, &ncand, &s_ok);
        okp = s_ok;
      }
      if (!okp) v = kth_largest<8>(q, N, kq, hist, sel);
      if (threadIdx.x == 0) {
        s_par[3] = v + eps;
        s_par[4] = v - eps;
        nwin = 0;
        s_above = 0;
      }
      __syncthreads();
      const uint64_t khi = dkey(s_par[3]), klo = dkey(s_par[4]);
      int C = 0;   // samples at or above v + eps (each contributes exactly 1)
      if (prefix_path) {
        // from the register-held prefixes: a prefix above that of v + eps is above it, one
        // below that of v - eps is below the window; the rest (the window and the two
        // boundary prefixes) are tested on their full keys
        const uint32_t hp = (uint32_t)(khi >> 32), lp = (uint32_t)(klo >> 32);
        unsigned above = 0;
#pragma unroll
        for (int j = 0; j < KEYS_PER_THREAD; ++j) {
          const int i = j * blockDim.x + threadIdx.x;
          if (i < N) {
            if (kr[j] > hp) {
              ++above;
            } else if (kr[j] >= lp) {
              const double qi = q[i];
              const uint64_t kf = dkey(qi);
              if (kf >= khi) {
                ++above;
              } else if (kf > klo) {
                const int slot = atomicAdd(&nwin, 1);
                if (slot < RISK_WINDOW_MAX) win[slot] = qi;
              }
            }
          }
        }
        above = __reduce_add_sync(0xffffffffu, above);
        if (lane == 0) atomicAdd(&s_above, (int)above);
        __syncthreads();
        C = s_above;
      } else {
        for (int i0 = 0; i0 < N; i0 += blockDim.x) {   // uniform trip count for __syncthreads_count
          const int i = i0 + threadIdx.x;
          bool above = false;
          if (i < N) {
            const double qi = q[i];
            const uint64_t k = dkey(qi);
            above = k >= khi;
            if (!above && k > klo) {
              const int slot = atomicAdd(&nwin, 1);
              if (slot < RISK_WINDOW_MAX) win[slot] = qi;
            }
          }
          C += __syncthreads_count(above);
        }
      }
      const int W = nwin;
      const double K = R.K;
      if (W <= RISK_WINDOW_MAX) {
        if (warp == 0) {
          for (int i = lane; i < W; i += 32) winf[i] = (float)((win[i] - v) * ie);
          __syncwarp();
          // Safeguarded Newton, first in FP32 on theta in [0, 1] (F(theta) = sum_window
          // s'(y_i + theta) - (K - C), non-decreasing, F' = sum 6 y (1 - y)), then in FP64 on
          // G(t) = (K - C) - S_window(t) (the sign of d rho/dt = 1 - S(t)/K without a
          // division; G' = sum 6 y (1 - y) / eps): a step that leaves the bracket, or meets
          // G' = 0, bisects instead.  The end rule then walks to adjacent doubles.
          const int act = W < 32 ? W : 32;
          const float Tf = (float)(K - (double)C);
          float th = 0.5f, tlo = 0.f, thi = 1.f;
          for (int it = 0; it < 4; ++it) {
            float f = 0.f, fp = 0.f;
            for (int i = lane; i < W; i += 32) {
              const float y = winf[i] + th;
              if (y >= 1.f) f += 1.f;
              else if (y > 0.f) {
                f += y * y * (3.f - 2.f * y);
                fp += 6.f * y * (1.f - y);
              }
            }
            f = warp_sum_active_f(f, act) - Tf;
            fp = warp_sum_active_f(fp, act);
            if (f < 0.f) tlo = th;
            else thi = th;
            float nt = fp > 0.f ? th - f / fp : 0.5f * (tlo + thi);
            if (!(nt > tlo && nt < thi)) nt = 0.5f * (tlo + thi);
            th = nt;
          }
          const double KC = K - (double)C;
          // the bracket [lo, hi] and the iterate in order-preserving keys: the bookkeeping (bracket
          // width in ulps, membership, neighbours, bisection) is integer arithmetic, and the FP64
          // instructions (each holding the narrow FP64 pipe) are those of G and of the step
          uint64_t klo = dkey(v - eps), khi = dkey(v);
          double t = v - eps * (double)th;
          bool lo_neg = false;   // G(lo) < 0 was evaluated
          auto G = [&](double tt, double* dG) {
            double S = 0.0, Sp = 0.0;
            for (int i = lane; i < W; i += 32) {
              const double x = win[i] - tt;
              if (x >= eps) S += 1.0;
              else if (x > 0.0) {
                const double y = x * ie;
                S += y * y * (3.0 - 2.0 * y);
                Sp += 6.0 * y * (1.0 - y);
              }
            }
            if (dG) *dG = warp_sum_active(Sp, act) * ie;
            return KC - warp_sum_active(S, act);
          };
          for (int it = 0; it < 64; ++it) {
            double dg;
            const double g = G(t, &dg);
            const uint64_t kt = dkey(t);
            if (g < 0.0) {
              klo = kt;
              lo_neg = true;
            } else {
              khi = kt;
            }
            if ((int64_t)(khi - klo) <= 4) break;   // a few ulps wide (or crossed by rounding noise)
            // the Newton step needs a few correct bits only: an FP32 reciprocal of G' (an
            // FP64 division is a long sequence on the narrow FP64 pipe)
            double step = INFINITY;
            if (dg > 0.0) {
              const float df = (float)dg;
              step = (df > 1e-30f && df < 1e30f) ? g * (double)(1.0f / df) : g / dg;
            }
            // converged when |step| < 2^-52 |t|: from the exponent fields
            const int es = (__double2hiint(step) >> 20) & 0x7FF, et = (__double2hiint(t) >> 20) & 0x7FF;
            uint64_t kn;
            if (((uint64_t)__double_as_longlong(step) << 1) == 0 || es + 53 <= et) {
              // converged: t bounds the root on the side its sign says; walk to adjacent doubles
              // on the other side until the sign changes (usually the first one)
              const bool tneg = g < 0.0;
              uint64_t kx = kt;
              for (int w = 0; w < 8; ++w) {
                kx = tneg ? kx + 1 : kx - 1;
                const bool neg = G(dval(kx), nullptr) < 0.0;
                if (neg) {
                  klo = kx > klo ? kx : klo;
                  lo_neg = true;
                } else {
                  khi = kx < khi ? kx : khi;
                }
                if (neg != tneg) break;
              }
              if ((int64_t)(khi - klo) <= 4) break;
              kn = klo + (khi - klo) / 2;
            } else {
              const uint64_t k1 = dkey(t - step);
              kn = (k1 > klo && k1 < khi && !(it >= 8 && it % 2 == 0)) ? k1 : klo + (khi - klo) / 2;   // bisect when slow
            }
            t = dval(kn);
          }
          const double lo = dval(klo), hi = dval(khi);
          // bisection end rule: lo if G(lo) >= 0 (possible only for the unevaluated v - eps), else hi
          const bool take_lo = !lo_neg && G(lo, nullptr) >= 0.0;
          if (lane == 0) s_par[5] = take_lo ? lo : hi;
        }
        __syncthreads();
        t = s_par[5];
      } else {
        BlockRed br{red};
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
    double val = qbar + R.kappa * var, dt = 0.0, tout = 0.0;
    if (R.kind == OUU_RISK_CVAR_SMOOTH) {
      double ssum, dsum;
      cvar_sums(q, N, prefix_path, kr, t, R.eps, R.inv_eps, win, RISK_WINDOW_MAX, (int*)sel, red, ssum, dsum);
      val = t + ssum * R.inv_K;
      dt = 1.0 - dsum * R.inv_K;
      tout = t;
    }
    if (threadIdx.x == 0) {
      params[3 * r + 0] = t;
      params[3 * r + 1] = qbar;
      params[3 * r + 2] = var;
      out[3 * r + 0] = val;
      out[3 * r + 1] = dt;
      out[3 * r + 2] = tout;
    }
    __syncthreads();
  }
}

// Pass 3 (many CTAs, each a contiguous range of samples): weights w[r][i]; with per-sample
// gradients gq [N][ldg] (FP32), also grad_out[r][j] += sum_i w[r][i] gq[i][j] (per-block
// FP64 sums added atomically; the select pass zeroed grad_out).  The products and the
// per-thread sums run in float-float arithmetic: w = wh + wl (two FP32), wh g split exactly
// by an FMA, sums by the error-free two-sum, so each thread's total carries about 44 bits
// and only the totals are FP64.
#define APPLY_W 256   // samples of a block whose weights sit in shared memory at a time
static __device__ __forceinline__ void ff_add_prod(float& sh, float& sl, float wh, float wl, float g) {
  const float p = wh * g;
  float e = fmaf(wh, g, -p);   // wh g = p + e exactly
  e = fmaf(wl, g, e);
  const float t = sh + p;      // two-sum: sh + p = t + err exactly
  const float bp = t - sh;
  const float err = (sh - (t - bp)) + (p - bp);
  sh = t;
  sl += err + e;
}

// Thread (g, jl) of the gradient sum: column j of samples s0 + kg + g + 2k, k < 16 (one batch of
// loads in flight instead of one round trip per sample).
// Rows of gq are the samples of the window [wlo, whi); samples outside it load 0.
static __device__ __forceinline__ void load_grad_group(float (&gv)[16], const float* __restrict__ gq, int ldg, int dz,
                                                       int s0, int s1, int kg, int g, int j, int wlo, int whi) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int i = s0 + kg + g + 2 * k;
    gv[k] = (i < s1 && i >= wlo && i < whi && j < dz) ? __ldg(gq + (int64_t)(i - wlo) * ldg + j) : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_risk_apply(const double* __restrict__ q, int N,
                                                    const RiskDev* __restrict__ risks, int n_risks,
                                                    const double* __restrict__ params, double* __restrict__ w,
                                                    const float* __restrict__ gq, int ldg, int dz,
                                                    double* __restrict__ grad_out, int wlo, int whi,
                                                    const int* __restrict__ flag_src, double* __restrict__ flag_dst) {
  __shared__ float wsh[OUU_MAX_RISKS][APPLY_W], wsl[OUU_MAX_RISKS][APPLY_W];
  __shared__ double gsum[OUU_MAX_RISKS][128];
  pdl_wait();
  if (flag_src && blockIdx.x == 0 && threadIdx.x == 0) *flag_dst = (double)__ldcg(flag_src);
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int i0 = min(N, (int)blockIdx.x * chunk), i1 = min(N, i0 + chunk);
  const int g = threadIdx.x >> 7, jl = threadIdx.x & 127;   // two sample parities x 128 columns
  for (int s0 = i0; s0 < i1; s0 += APPLY_W) {
    const int s1 = min(i1, s0 + APPLY_W), ns = s1 - s0;
    const bool gsub = gq && s1 > wlo && s0 < whi;   // uniform over the block
    float gv[16];
    if (gsub) load_grad_group(gv, gq, ldg, dz, s0, s1, 0, g, jl, wlo, whi);   // in flight during the weights
    const int i = s0 + threadIdx.x;
    if (i < s1) {
      const double qi = q[i];
#pragma unroll
      for (int r = 0; r < OUU_MAX_RISKS; ++r) {
        if (r >= n_risks) break;
        const RiskDev& R = risks[r];
        const double t = params[3 * r], qbar = params[3 * r + 1];
        double wi;
        if (R.kind == OUU_RISK_MEAN_VAR) {
          wi = (1.0 + 2.0 * R.kappa * (qi - qbar)) * R.inv_N;
        } else {
          wi = splus_d1(qi - t, R.eps, R.inv_eps) * R.inv_K;
        }
        if (i >= wlo && i < whi) w[(int64_t)r * (whi - wlo) + (i - wlo)] = wi;
        if (gsub) {
          const float wh = (float)wi;
          wsh[r][threadIdx.x] = wh;
          wsl[r][threadIdx.x] = (float)(wi - (double)wh);
        }
      }
    }
    if (gsub) {
      __syncthreads();   // the weights of the sub-range are in shared memory
      for (int jb = 0; jb < dz; jb += 128) {
        const int j = jb + jl;
        float sh[OUU_MAX_RISKS], sl[OUU_MAX_RISKS];
#pragma unroll
        for (int r = 0; r < OUU_MAX_RISKS; ++r) sh[r] = sl[r] = 0.f;
        for (int kg = 0; kg < ns; kg += 32) {
          if (jb > 0 || kg > 0) load_grad_group(gv, gq, ldg, dz, s0, s1, kg, g, j, wlo, whi);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int ii = kg + g + 2 * k;
            if (ii < ns)
#pragma unroll
              for (int r = 0; r < OUU_MAX_RISKS; ++r)
                if (r < n_risks) ff_add_prod(sh[r], sl[r], wsh[r][ii], wsl[r][ii], gv[k]);
          }
        }
        if (g == 1)
#pragma unroll
          for (int r = 0; r < OUU_MAX_RISKS; ++r)
            if (r < n_risks) gsum[r][jl] = (double)sh[r] + (double)sl[r];
        __syncthreads();
        if (g == 0 && j < dz)
#pragma unroll
          for (int r = 0; r < OUU_MAX_RISKS; ++r)
            if (r < n_risks) atomicAdd(&grad_out[r * dz + j], ((double)sh[r] + (double)sl[r]) + gsum[r][jl]);
        __syncthreads();
      }
    }
  }
}

void launch_risk_select(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* out,
                        double* scratch, cudaStream_t s, double* grad_out, int n_grad, const double* mom_part,
                        int mom_n) {
  static_assert(OUU_RISK_SCRATCH >= 3 * OUU_MAX_RISKS + 2 * RISK_BLOCKS, "risk scratch size");
  double* params = scratch;
  const double* part = mom_part;
  int nparts = mom_n;
  if (!mom_part) {
    double* p = scratch + 3 * OUU_MAX_RISKS;
    launch_pdl(k_risk_moments, dim3(RISK_BLOCKS), dim3(256), 0, s, q, N, p);
    part = p;
    nparts = RISK_BLOCKS;
  }
  launch_pdl(k_risk_select, dim3(1), dim3(1024), 0, s, q, N, part, nparts, risks_dev, n_risks, params, out, grad_out,
             grad_out ? n_grad : 0);
}

void launch_risk_apply(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* scratch,
                       cudaStream_t s, const float* gq, int ldg, int dz, double* grad_out, int wfirst, int wcount,
                       const int* flag_src, double* flag_dst) {
  const int wlo = wcount < 0 ? 0 : wfirst, whi = wcount < 0 ? N : wfirst + wcount;
  const double* params = scratch;
  launch_pdl(k_risk_apply, dim3(RISK_BLOCKS), dim3(256), 0, s, q, N, risks_dev, n_risks, params, w, gq, ldg, dz,
             grad_out, wlo, whi, flag_dst ? flag_src : nullptr, flag_dst);
}

void launch_risk_weights(const double* q, int N, const RiskDev* risks_dev, int n_risks, double* w, double* out,
                         double* scratch, cudaStream_t s, const float* gq, int ldg, int dz, double* grad_out,
                         int wfirst, int wcount, const int* flag_src, double* flag_dst) {
  launch_risk_select(q, N, risks_dev, n_risks, out, scratch, s, gq ? grad_out : nullptr, n_risks * dz);
  launch_risk_apply(q, N, risks_dev, n_risks, w, scratch, s, gq, ldg, dz, grad_out, wfirst, wcount, flag_src,
                    flag_dst);
}

// Kernel-level entry used by the risk-weight numerics test (declared in include/ouu_kernels.h).
extern "C" ouu_status ouu_kernel_risk_weights(const double* q_dev, int N, const ouu_risk_desc* risks, int n_risks,
                                              double* w_dev, double* out_host, const float* gq_dev, int ldg, int dz,
                                              double* grad_host, void* stream) {
  OUU_CHECK_ARG(q_dev && risks && w_dev && out_host, "null argument");
  OUU_CHECK_ARG(!gq_dev || (grad_host && dz >= 1 && ldg >= dz), "gradients: grad_host, dz >= 1, ldg >= dz");
  OUU_CHECK_ARG(N >= 1 && n_risks >= 1 && n_risks <= OUU_MAX_RISKS, "N >= 1 and 1 <= n_risks <= 4");
  for (int r = 0; r < n_risks; ++r)
    OUU_CHECK_ARG(risks[r].kind == OUU_RISK_MEAN_VAR ||
                      (risks[r].kind == OUU_RISK_CVAR_SMOOTH && risks[r].eps > 0 && risks[r].beta >= 0 && risks[r].beta < 1),
                  "risk descriptor: kind, and for CVaR eps > 0 and beta in [0, 1)");
  RiskDev rd[OUU_MAX_RISKS];
  for (int r = 0; r < n_risks; ++r) {
    rd[r].kind = risks[r].kind;
    rd[r].kappa = risks[r].kappa;
    rd[r].beta = risks[r].beta;
    rd[r].eps = risks[r].eps;
    rd[r].t = risks[r].t;
    rd[r].t_optimal = risks[r].t_optimal;
    risk_dev_finish(rd[r], N);
  }
  cudaStream_t s = (cudaStream_t)stream;
  RiskDev* d_r = nullptr;
  double* scr = nullptr;
  double* d_out = nullptr;
  double* d_grad = nullptr;
  ouu_status st = OUU_OK;
  const size_t gbytes = gq_dev ? (size_t)n_risks * dz * 8 : 8;
  if (cudaMalloc((void**)&d_r, sizeof(rd)) != cudaSuccess || cudaMalloc((void**)&scr, OUU_RISK_SCRATCH * 8) != cudaSuccess ||
      cudaMalloc((void**)&d_out, 3 * OUU_MAX_RISKS * 8) != cudaSuccess || cudaMalloc((void**)&d_grad, gbytes) != cudaSuccess) {
    ouu_set_error("cudaMalloc failed");
    st = OUU_ERR_OOM;
  } else if (cudaMemcpy(d_r, rd, sizeof(RiskDev) * n_risks, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(scr, 0, OUU_RISK_SCRATCH * 8) != cudaSuccess) {
    ouu_set_error("risk set-up copy failed");
    st = OUU_ERR_CUDA;
  } else {
    launch_risk_weights(q_dev, N, d_r, n_risks, w_dev, d_out, scr, s, gq_dev, ldg, dz, gq_dev ? d_grad : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, d_out, (size_t)3 * n_risks * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && gq_dev) e = cudaMemcpyAsync(grad_host, d_grad, gbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      ouu_set_error(std::string("risk weights: ") + cudaGetErrorString(e));
      st = OUU_ERR_CUDA;
    }
  }
  cudaFree(d_r);
  cudaFree(scr);
  cudaFree(d_out);
  cudaFree(d_grad);
  return st;
}
