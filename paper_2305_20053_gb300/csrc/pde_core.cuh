// Per-sample semilinear elliptic solver: geometric multigrid-preconditioned CG
// inside an inexact Newton iteration with an FP64 residual.
//
// State equation (Sec. 4.2 of arXiv 2305.20053): -div(e^m grad u) + r u^3 = sum_j z_j f_j
// on (0,1)^2 with u = 0 on the boundary, discretised by the 5-point stencil on the
// vertex grid x_i = i h (h = 1/(n-1)) with face coefficient exp((m_a + m_b)/2).
//
// Every routine here is *collective* over one cooperating group (one CTA on the
// GPU): each member calls it with the same arguments, and the context `C`
// supplies the member's share of the iteration space, barriers and sums.
// Arrays are full n x n grids, row-major [iy * n + ix]; only interior entries are
// ever written, so boundary entries keep the zeros they were initialised with.
#pragma once
#include <stdint.h>
#include <math.h>

#ifndef __CUDACC__
#define __device__
#define __host__
#define __forceinline__ inline
#endif

#define OUU_MAX_LEVELS 11

struct MgLevel {
  int n;          // nodes per side
  float inv_h2;   // 1 / h_l^2
  float* kx;      // face (ix,iy)-(ix+1,iy)
  float* ky;      // face (ix,iy)-(ix,iy+1)
  float* D;       // diagonal: (sum of the four faces) / h^2 + reaction
  float* x;       // iterate
  float* b;       // right-hand side
  float* r;       // residual / scratch
};

struct Hierarchy {
  int nlev;
  MgLevel lev[OUU_MAX_LEVELS];
};

// ------------------------------------------------------------------ loops
// Interior loop: rows are dealt to row groups (warps), columns to lanes, so that a
// warp touches consecutive addresses of one row.
#define OUU_FOR_RANGE(c, j, j0, j1, i, i0, i1)                         \
  for (int j = (j0) + (c).row0(); j <= (j1); j += (c).rowstep())       \
    for (int i = (i0) + (c).col0(); i <= (i1); i += (c).colstep())

#define OUU_FOR_INTERIOR(c, n, iy, ix) OUU_FOR_RANGE(c, iy, 1, (n) - 2, ix, 1, (n) - 2)

// ------------------------------------------------------------------ multigrid set-up
// Coarse face coefficients: the two fine faces that make one coarse face are in
// series (harmonic mean); the three fine rows across it are averaged 1/4,1/2,1/4.
template <class C>
__device__ void mg_coarsen_coeffs(const C& c, const MgLevel& F, MgLevel& K) {
  const int nf = F.n, nk = K.n;
  OUU_FOR_RANGE(c, J, 1, nk - 2, I, 0, nk - 2) {
    float acc = 0.f;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      const int y = 2 * J + d;
      const float a = F.kx[y * nf + 2 * I], b = F.kx[y * nf + 2 * I + 1];
      acc += (d == 0 ? 0.5f : 0.25f) * (2.f * a * b / (a + b));
    }
    K.kx[J * nk + I] = acc;
  }
  OUU_FOR_RANGE(c, J, 0, nk - 2, I, 1, nk - 2) {
    float acc = 0.f;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      const int x = 2 * I + d;
      const float a = F.ky[(2 * J) * nf + x], b = F.ky[(2 * J + 1) * nf + x];
      acc += (d == 0 ? 0.5f : 0.25f) * (2.f * a * b / (a + b));
    }
    K.ky[J * nk + I] = acc;
  }
}

// Full-weighting restriction of the interior of `src` (fine) into `dst` (coarse).
template <class C>
__device__ void mg_restrict(const C& c, int nf, const float* src, int nk, float* dst) {
  OUU_FOR_INTERIOR(c, nk, J, I) {
    const float* s = src + (2 * J) * nf + 2 * I;
    const float v = 4.f * s[0] + 2.f * (s[-1] + s[1] + s[-nf] + s[nf]) +
                    (s[-nf - 1] + s[-nf + 1] + s[nf - 1] + s[nf + 1]);
    dst[J * nk + I] = 0.0625f * v;
  }
}

// D = (kxW + kxE + kyS + kyN) / h^2 + react (react may be null).
template <class C>
__device__ void mg_set_diag(const C& c, MgLevel& L, const float* react) {
  const int n = L.n;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const float s = L.kx[p] + L.kx[p - 1] + L.ky[p] + L.ky[p - n];
    L.D[p] = s * L.inv_h2 + (react ? react[p] : 0.f);
  }
}

// ------------------------------------------------------------------ smoothing / transfer
// One red-black Gauss-Seidel half sweep over the points with (ix + iy) % 2 == color.
// from_zero: the other colour is taken as zero (first sweep of a cycle), so the
// stale iterate is never read.
template <class C>
__device__ void mg_rbgs(const C& c, MgLevel& L, int color, bool from_zero) {
  const int n = L.n;
  const float ih2 = L.inv_h2;
  const int half = (n - 2 + 1) / 2;      // points of one colour per row (upper bound)
  for (int iy = 1 + c.row0(); iy <= n - 2; iy += c.rowstep()) {
    const int ix0 = 1 + ((iy + 1 + color) & 1);   // first ix >= 1 with (ix+iy)&1 == color
    for (int k = c.col0(); k < half; k += c.colstep()) {
      const int ix = ix0 + 2 * k;
      if (ix > n - 2) break;
      const int p = iy * n + ix;
      float v = L.b[p];
      if (!from_zero)
        v += ih2 * (L.kx[p] * L.x[p + 1] + L.kx[p - 1] * L.x[p - 1] + L.ky[p] * L.x[p + n] +
                    L.ky[p - n] * L.x[p - n]);
      L.x[p] = v / L.D[p];
    }
  }
}

// r = b - A x.
template <class C>
__device__ void mg_residual(const C& c, MgLevel& L) {
  const int n = L.n;
  const float ih2 = L.inv_h2;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const float ax = L.D[p] * L.x[p] - ih2 * (L.kx[p] * L.x[p + 1] + L.kx[p - 1] * L.x[p - 1] +
                                              L.ky[p] * L.x[p + n] + L.ky[p - n] * L.x[p - n]);
    L.r[p] = L.b[p] - ax;
  }
}

// F.x += P K.x (bilinear interpolation; coarse boundary values are zero).
template <class C>
__device__ void mg_prolong_add(const C& c, const MgLevel& K, MgLevel& F) {
  const int nf = F.n, nk = K.n;
  OUU_FOR_INTERIOR(c, nf, iy, ix) {
    const int I = ix >> 1, J = iy >> 1;
    const float* xc = K.x + J * nk + I;
    float v;
    if (!(ix & 1) && !(iy & 1)) v = xc[0];
    else if (ix & 1 && !(iy & 1)) v = 0.5f * (xc[0] + xc[1]);
    else if (!(ix & 1)) v = 0.5f * (xc[0] + xc[nk]);
    else v = 0.25f * (xc[0] + xc[1] + xc[nk] + xc[nk + 1]);
    F.x[iy * nf + ix] += v;
  }
}

// Symmetric V(1,1) cycle: red-black pre-smoothing, black-red post-smoothing, so the
// preconditioner is symmetric (restriction = P^T / 4) as CG requires.  Solves the
// coarsest (3 x 3, one unknown) level exactly in FP64.  Starts from x = 0.
template <class C>
__device__ void mg_vcycle(const C& c, Hierarchy& H) {
  const int nl = H.nlev;
  for (int l = 0; l < nl - 1; ++l) {
    MgLevel& L = H.lev[l];
    mg_rbgs(c, L, 0, true);
    c.sync();
    mg_rbgs(c, L, 1, false);
    c.sync();
    mg_residual(c, L);
    c.sync();
    mg_restrict(c, L.n, L.r, H.lev[l + 1].n, H.lev[l + 1].b);
    c.sync();
  }
  {
    MgLevel& L = H.lev[nl - 1];   // n == 3
    if (c.row0() == 0 && c.col0() == 0) L.x[4] = (float)((double)L.b[4] / (double)L.D[4]);
    c.sync();
  }
  for (int l = nl - 2; l >= 0; --l) {
    MgLevel& L = H.lev[l];
    mg_prolong_add(c, H.lev[l + 1], L);
    c.sync();
    mg_rbgs(c, L, 1, false);
    c.sync();
    mg_rbgs(c, L, 0, false);
    c.sync();
  }
}

// ------------------------------------------------------------------ CG on level 0
// q = J p and returns (p, q).  Inner products of the CG iteration are FP64 sums of the
// FP32 entries' products (a product of two FP32 numbers is exact in FP64).
template <class C>
__device__ double op_apply_dot(const C& c, const MgLevel& L, const float* p, float* q) {
  const int n = L.n;
  const float ih2 = L.inv_h2;
  double acc = 0.0;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int k = iy * n + ix;
    const float v = L.D[k] * p[k] - ih2 * (L.kx[k] * p[k + 1] + L.kx[k - 1] * p[k - 1] +
                                           L.ky[k] * p[k + n] + L.ky[k - n] * p[k - n]);
    q[k] = v;
    acc = fma((double)p[k], (double)v, acc);
  }
  return c.sum_d(acc);
}

struct CgResult {
  int iters;
  double rel;       // final ||r|| / ||b||
  double scale;     // the solution of J x = b is scale * x (b is normalised to unit norm)
};

// Solves J x = b for x (x overwritten) with the V-cycle as preconditioner.  On entry
// H.lev[0].b holds b (it becomes the CG residual); H.lev[0].x and H.lev[0].r are the
// preconditioner's output and scratch; p, q are work vectors.  FP32 vectors; the inner
// products are accumulated in FP64 (per member and across members).
template <class C>
__device__ CgResult pcg_solve(const C& c, Hierarchy& H, float* x, float* p, float* q,
                              double bnorm, double rtol, int maxit) {
  MgLevel& L = H.lev[0];
  const int n = L.n;
  float* r = L.b;
  float* z = L.x;
  CgResult res{0, 1.0, 0.0};
  // Normalise b to unit norm (keeps FP32 dot products far from underflow when b is
  // a late refinement residual) and start from x = 0.
  const float inv = bnorm > 0.0 ? (float)(1.0 / bnorm) : 0.f;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int k = iy * n + ix;
    r[k] *= inv;
    x[k] = 0.f;
  }
  c.sync();
  if (!(bnorm > 0.0) || !(bnorm < INFINITY)) {
    res.rel = bnorm > 0.0 ? 1.0 : 0.0;
    return res;
  }
  res.scale = bnorm;
  bnorm = 1.0;
  mg_vcycle(c, H);
  double acc = 0.0;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int k = iy * n + ix;
    p[k] = z[k];
    acc = fma((double)r[k], (double)z[k], acc);
  }
  double rz = c.sum_d(acc);
  for (int it = 1; it <= maxit; ++it) {
    const double pq = op_apply_dot(c, L, p, q);
    if (!(pq > 0.0)) break;   // breakdown (exact solution reached, or not SPD): keep x
    const double alpha = rz / pq;
    const float af = (float)alpha;
    double rr = 0.0;
    OUU_FOR_INTERIOR(c, n, iy, ix) {
      const int k = iy * n + ix;
      x[k] += af * p[k];
      const float rv = r[k] - af * q[k];
      r[k] = rv;
      rr = fma((double)rv, (double)rv, rr);
    }
    const double rnorm = sqrt(c.sum_d(rr));
    res.iters = it;
    res.rel = rnorm / bnorm;
    if (!(res.rel > rtol) || it == maxit) break;   // also stops on NaN
    mg_vcycle(c, H);
    acc = 0.0;
    OUU_FOR_INTERIOR(c, n, iy, ix) {
      const int k = iy * n + ix;
      acc = fma((double)r[k], (double)z[k], acc);
    }
    const double rz_new = c.sum_d(acc);
    const float beta = (float)(rz_new / rz);
    rz = rz_new;
    OUU_FOR_INTERIOR(c, n, iy, ix) {
      const int k = iy * n + ix;
      p[k] = z[k] + beta * p[k];
    }
    c.sync();
  }
  return res;
}

// ------------------------------------------------------------------ FP64 Newton pieces
// E = exp(m/2) at every node; level-0 FP32 faces k = E_a E_b.
template <class C>
__device__ void build_fine_coeffs(const C& c, int n, const double* m, double* E, MgLevel& L0) {
  for (int iy = c.row0(); iy < n; iy += c.rowstep())
    for (int ix = c.col0(); ix < n; ix += c.colstep()) E[iy * n + ix] = exp(0.5 * m[iy * n + ix]);
  c.sync();
  for (int iy = c.row0(); iy < n; iy += c.rowstep())
    for (int ix = c.col0(); ix < n; ix += c.colstep()) {
      const int p = iy * n + ix;
      const double e = E[p];
      L0.kx[p] = ix < n - 1 ? (float)(e * E[p + 1]) : 0.f;
      L0.ky[p] = iy < n - 1 ? (float)(e * E[p + n]) : 0.f;
    }
}

// R = A_h u + r u^3 - f in FP64 (A_h from E); writes rhs = -R (FP32) and returns ||R||^2.
template <class C>
__device__ double newton_residual(const C& c, int n, double inv_h2, double rr, const double* E,
                                  const double* f, const double* u, float* rhs) {
  double acc = 0.0;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const double uc = u[p];
    const double s = E[p + 1] * (uc - u[p + 1]) + E[p - 1] * (uc - u[p - 1]) +
                     E[p + n] * (uc - u[p + n]) + E[p - n] * (uc - u[p - n]);
    const double R = E[p] * s * inv_h2 + rr * uc * uc * uc - f[p];
    rhs[p] = (float)(-R);
    acc += R * R;
  }
  return c.sum_d(acc);
}

// Same residual with a given right-hand side b (FP64) and the linear operator J(u0)
// applied to lam: R = b - J lam, J = A_h + 3 r u0^2 (adjoint refinement).
template <class C>
__device__ double linear_residual(const C& c, int n, double inv_h2, double rr, const double* E,
                                  const double* u0, const double* b, const double* lam, float* rhs) {
  double acc = 0.0;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const double lc = lam[p];
    const double s = E[p + 1] * (lc - lam[p + 1]) + E[p - 1] * (lc - lam[p - 1]) +
                     E[p + n] * (lc - lam[p + n]) + E[p - n] * (lc - lam[p - n]);
    const double u = u0[p];
    const double R = b[p] - (E[p] * s * inv_h2 + 3.0 * rr * u * u * lc);
    rhs[p] = (float)R;
    acc += R * R;
  }
  return c.sum_d(acc);
}

// u += step * dx on the interior.
template <class C>
__device__ void axpy_interior(const C& c, int n, double step, const float* dx, double* u) {
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    u[p] += step * (double)dx[p];
  }
}

// Level-0 reaction 3 r u^2 into `react` and the level-0 diagonal; then the coarse
// reactions (full weighting) and diagonals.
template <class C>
__device__ void setup_jacobian(const C& c, Hierarchy& H, double rr, const double* u) {
  MgLevel& L0 = H.lev[0];
  const int n = L0.n;
  float* react = L0.r;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const double uv = u[p];
    const float cr = (float)(3.0 * rr * uv * uv);
    react[p] = cr;
    const float s = L0.kx[p] + L0.kx[p - 1] + L0.ky[p] + L0.ky[p - n];
    L0.D[p] = s * L0.inv_h2 + cr;
  }
  c.sync();
  for (int l = 1; l < H.nlev; ++l) {
    MgLevel& F = H.lev[l - 1];
    MgLevel& K = H.lev[l];
    mg_restrict(c, F.n, F.r, K.n, K.r);
    c.sync();
    mg_set_diag(c, K, K.r);
    c.sync();
  }
}

// Coefficients of every coarse level (do once per sample, after build_fine_coeffs).
template <class C>
__device__ void setup_coarse_coeffs(const C& c, Hierarchy& H) {
  for (int l = 1; l < H.nlev; ++l) {
    mg_coarsen_coeffs(c, H.lev[l - 1], H.lev[l]);
    c.sync();
  }
}

// f = sum_j z_j g_j with separable sources g_j(x, y) = gx[jx](x) gy[jy](y) / (w sqrt(2 pi)):
// tmp[jy][ix] = sum_jx z[jy L + jx] gx[jx][ix], f[iy][ix] = s sum_jy gy[jy][iy] tmp[jy][ix].
template <class C>
__device__ void build_forcing(const C& c, int n, int L, const double* gx, const double* gy, double scale,
                              const double* z, double* tmp, double* f) {
  for (int jy = c.row0(); jy < L; jy += c.rowstep())
    for (int ix = c.col0(); ix < n; ix += c.colstep()) {
      double a = 0.0;
      for (int jx = 0; jx < L; ++jx) a += z[jy * L + jx] * gx[jx * n + ix];
      tmp[jy * n + ix] = a;
    }
  c.sync();
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    double a = 0.0;
    for (int jy = 0; jy < L; ++jy) a += gy[jy * n + iy] * tmp[jy * n + ix];
    f[iy * n + ix] = scale * a;
  }
}

// Newton solve of A_h u + r u^3 = f from u = 0 (u's interior must be zero on entry).
// Stops once ||R|| <= rtol ||f||, then takes one more step; backtracks (halving, at
// most 10 times) when a step increases ||R||.  Returns 0 on success, 1 when not
// converged within maxit steps, 2 on a non-finite residual.
struct NewtonResult {
  int status;
  int newton_iters;
  int cg_iters;
};

template <class C>
__device__ NewtonResult newton_solve(const C& c, Hierarchy& H, double rr, const double* E,
                                     const double* f, double* u, float* x, float* p, float* q,
                                     double rtol, int maxit, double cg_rtol, int cg_maxit) {
  MgLevel& L0 = H.lev[0];
  const int n = L0.n;
  const double ih2 = (double)(n - 1) * (double)(n - 1);
  NewtonResult res{0, 0, 0};
  double rn = sqrt(newton_residual(c, n, ih2, rr, E, f, u, L0.b));
  const double fnorm = rn;   // u = 0: R = -f
  c.sync();
  if (!(rn == rn) || isinf(rn)) {   // non-finite coefficients or forcing
    res.status = 2;
    return res;
  }
  if (!(fnorm > 0.0)) return res;
  bool extra = false;
  for (int it = 0;; ++it) {
    if (!(rn == rn) || isinf(rn)) { res.status = 2; break; }
    if (rn <= rtol * fnorm) {
      if (extra) break;
      extra = true;
    } else if (it >= maxit) {
      res.status = 1;
      break;
    }
    setup_jacobian(c, H, rr, u);
    CgResult cg = pcg_solve(c, H, x, p, q, rn, cg_rtol, cg_maxit);
    res.cg_iters += cg.iters;
    double step = cg.scale;
    axpy_interior(c, n, step, x, u);
    c.sync();
    double rn_new = sqrt(newton_residual(c, n, ih2, rr, E, f, u, L0.b));
    c.sync();
    for (int bt = 0; bt < 10 && rn_new > rn; ++bt) {
      axpy_interior(c, n, -0.5 * step, x, u);
      step *= 0.5;
      c.sync();
      rn_new = sqrt(newton_residual(c, n, ih2, rr, E, f, u, L0.b));
      c.sync();
    }
    rn = rn_new;
    res.newton_iters = it + 1;
    if (extra) break;
  }
  return res;
}

// Adjoint (or any linear) solve J(u) lam = b by FP32 MG-PCG inside FP64 iterative
// refinement: lam += J^-1 (b - J lam) until ||b - J lam|| <= rtol ||b||, or, once below
// 1e-9 ||b||, until a refinement step no longer halves the residual: the FP64 residual
// has then reached its rounding floor (eps times the stencil terms, which on fine grids
// and high-contrast fields exceeds 1e-12 ||b||).
// lam's interior must be zero on entry.  J's levels must already be set up for u.
template <class C>
__device__ NewtonResult refine_solve(const C& c, Hierarchy& H, double rr, const double* E,
                                     const double* u, const double* b, double* lam, float* x,
                                     float* p, float* q, double rtol, int maxit, double cg_rtol,
                                     int cg_maxit) {
  MgLevel& L0 = H.lev[0];
  const int n = L0.n;
  const double ih2 = (double)(n - 1) * (double)(n - 1);
  NewtonResult res{0, 0, 0};
  double rn = sqrt(linear_residual(c, n, ih2, rr, E, u, b, lam, L0.b));
  c.sync();
  const double bnorm = rn;
  if (!(rn == rn) || isinf(rn)) {
    res.status = 2;
    return res;
  }
  if (!(bnorm > 0.0)) return res;
  double prev = INFINITY;
  for (int it = 0;; ++it) {
    if (!(rn == rn) || isinf(rn)) { res.status = 2; break; }
    if (rn <= rtol * bnorm) break;
    if (rn <= 1e-9 * bnorm && rn > 0.5 * prev) break;   // rounding floor
    if (it >= maxit) { res.status = 1; break; }
    CgResult cg = pcg_solve(c, H, x, p, q, rn, cg_rtol, cg_maxit);
    res.cg_iters += cg.iters;
    axpy_interior(c, n, cg.scale, x, lam);
    c.sync();
    prev = rn;
    rn = sqrt(linear_residual(c, n, ih2, rr, E, u, b, lam, L0.b));
    c.sync();
    res.newton_iters = it + 1;
  }
  return res;
}

// Q = 1/2 h^2 sum (u - ut)^2 and (optionally) dq = h^2 (u - ut) on the interior.
template <class C>
__device__ double qoi_and_grad(const C& c, int n, const double* u, const double* ut, double* dq) {
  const double h2 = 1.0 / ((double)(n - 1) * (double)(n - 1));
  double acc = 0.0;
  OUU_FOR_INTERIOR(c, n, iy, ix) {
    const int p = iy * n + ix;
    const double d = u[p] - ut[p];
    acc += d * d;
    if (dq) dq[p] = h2 * d;
  }
  return 0.5 * h2 * c.sum_d(acc);
}
