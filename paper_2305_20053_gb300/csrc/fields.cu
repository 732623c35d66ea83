// Random-field synthesis (Sec. 2 prior, Karhunen-Loeve expansion of Sec. 3.3):
//   m[iy][ix] = mbar + n sum_{k2,k1} V[k2][iy] (xi[k2][k1] / lambda[k2][k1]) V[k1][ix],
// V the orthonormal DCT-II matrix (eigenvectors of the Neumann second difference).
// Standard normals xi: Philox4x32-10 (Salmon et al., SC'11), counter
// (q/2, sample_lo, sample_hi, tag), key (seed_lo, seed_hi); two 52-bit uniforms
// per output block, Box-Muller gives the normals of modes q = 2c and 2c+1.
// Two passes, both FP64: rows C'[k2][:] = C[k2][:] V (C generated on the fly),
// then columns m[:, ix] = mbar + n V^T C'[:, ix] in place.
#include "ouu_internal.cuh"

#define OUU_PHILOX_TAG 0x4B4C5158u

static __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

static __device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  const uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
  return ((double)k + 0.5) * 0x1p-52;
}

static __device__ double field_normal(uint64_t seed, uint64_t sample, uint32_t q) {
  uint32_t c[4] = {q >> 1, (uint32_t)sample, (uint32_t)(sample >> 32), OUU_PHILOX_TAG};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = uniform52(c[0], c[1]);
  const double u2 = uniform52(c[2], c[3]);
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return (q & 1) ? r * sn : r * cs;
}

#define OUU_FIELD_ROWS 8

__global__ void k_fields_rows(int n, uint64_t seed, int64_t first, const double* invlam, const double* V,
                              double* m) {
  extern __shared__ double crow[];   // [OUU_FIELD_ROWS][n]
  const int s = blockIdx.y;
  const int r0 = blockIdx.x * OUU_FIELD_ROWS;
  const uint64_t gs = (uint64_t)(first + s);
  for (int e = threadIdx.x; e < OUU_FIELD_ROWS * n; e += blockDim.x) {
    const int k2 = r0 + e / n, k1 = e % n;
    double v = 0.0;
    if (k2 < n) v = field_normal(seed, gs, (uint32_t)(k2 * n + k1)) * invlam[k2 * n + k1];
    crow[e] = v;
  }
  __syncthreads();
  double* ms = m + (int64_t)s * n * n;
  for (int e = threadIdx.x; e < OUU_FIELD_ROWS * n; e += blockDim.x) {
    const int rr = e / n, ix = e % n, k2 = r0 + rr;
    if (k2 >= n) continue;
    double a = 0.0;
    for (int k1 = 0; k1 < n; ++k1) a += crow[rr * n + k1] * V[k1 * n + ix];
    ms[(int64_t)k2 * n + ix] = a;
  }
}

__global__ void k_fields_cols(int n, const double* V, double m_mean, double* m) {
  extern __shared__ double tile[];   // [n][32]
  const int s = blockIdx.y;
  const int ix0 = blockIdx.x * 32;
  double* ms = m + (int64_t)s * n * n;
  const int j = threadIdx.x & 31;
  for (int k2 = threadIdx.x >> 5; k2 < n; k2 += blockDim.x >> 5)
    tile[k2 * 32 + j] = ix0 + j < n ? ms[(int64_t)k2 * n + ix0 + j] : 0.0;
  __syncthreads();
  if (ix0 + j >= n) return;
  for (int iy = threadIdx.x >> 5; iy < n; iy += blockDim.x >> 5) {
    double a = 0.0;
    for (int k2 = 0; k2 < n; ++k2) a += V[k2 * n + iy] * tile[k2 * 32 + j];
    ms[(int64_t)iy * n + ix0 + j] = m_mean + (double)n * a;
  }
}

void launch_sample_fields(int n, uint64_t seed, int64_t first, int count, const double* invlam, const double* V,
                          double m_mean, double* m, cudaStream_t s) {
  if (count <= 0) return;
  const size_t sm1 = (size_t)OUU_FIELD_ROWS * n * sizeof(double);
  const size_t sm2 = (size_t)n * 32 * sizeof(double);
  if (sm2 > 48 * 1024) ouu_smem_limit((const void*)k_fields_cols, sm2);
  if (sm1 > 48 * 1024) ouu_smem_limit((const void*)k_fields_rows, sm1);
  dim3 g1((n + OUU_FIELD_ROWS - 1) / OUU_FIELD_ROWS, count);
  k_fields_rows<<<g1, 256, sm1, s>>>(n, seed, first, invlam, V, m);
  dim3 g2((n + 31) / 32, count);
  k_fields_cols<<<g2, 256, sm2, s>>>(n, V, m_mean, m);
}
