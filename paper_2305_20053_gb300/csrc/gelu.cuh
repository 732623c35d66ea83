// GELU of the reduced-basis network (Sec. 3.3) and its derivatives:
//   gelu(a) = a Phi(a),  gelu'(a) = Phi(a) + a phi(a),  gelu''(a) = phi(a) (2 - a^2),
// phi and Phi the standard normal density and distribution function.  Phi by the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions, 26.2.17 (after
// Hastings): for x >= 0, 1 - Phi(x) = phi(x) (b1 t + b2 t^2 + b3 t^3 + b4 t^4 + b5 t^5) with
// t = 1 / (1 + p x), absolute error below 7.5e-8; Phi(-x) = 1 - Phi(x).  One exponential
// serves phi, Phi and both derivatives (the fast exponential and reciprocal add an absolute
// error of order 1e-7 to Phi), about a fifth of the instructions of an erf evaluation.
#pragma once

static __device__ __forceinline__ void norm_pdf_cdf(float a, float& pdf, float& cdf) {
  const float x = fabsf(a);
  pdf = 0.3989422804014327f * __expf(-0.5f * a * a);
  const float t = __fdividef(1.f, fmaf(0.2316419f, x, 1.f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.330274429f, -1.821255978f), 1.781477937f), -0.356563782f), 0.319381530f);
  const float upper = pdf * poly;   // 1 - Phi(|a|)
  cdf = a >= 0.f ? 1.f - upper : upper;
}

static __device__ __forceinline__ float gelu_fwd(float a) {
  float pdf, cdf;
  norm_pdf_cdf(a, pdf, cdf);
  return a * cdf;
}

static __device__ __forceinline__ float gelu_d1(float a) {
  float pdf, cdf;
  norm_pdf_cdf(a, pdf, cdf);
  return fmaf(a, pdf, cdf);
}

static __device__ __forceinline__ float gelu_d2(float a) {
  return 0.3989422804014327f * __expf(-0.5f * a * a) * (2.f - a * a);
}

// gelu(a) and gelu'(a) together.
static __device__ __forceinline__ void gelu_and_d1(float a, float& g, float& d) {
  float pdf, cdf;
  norm_pdf_cdf(a, pdf, cdf);
  g = a * cdf;
  d = fmaf(a, pdf, cdf);
}
