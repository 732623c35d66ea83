// Mass-weighted POD basis of training states (Sec. 3.3), all in FP64 on the GPU:
// snapshot Gram C = h^2 D D^T (D = centred interior states), its eigenpairs by
// the cyclic two-sided Jacobi method with a round-robin ("tournament") ordering
// so that the n/2 rotations of one step are independent, then
// Phi = D^T V Lambda^-1/2 on the r_u largest eigenvalues.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dino.cuh"

#define GRID_STRIDE(e, total) \
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (total); e += (int64_t)gridDim.x * blockDim.x)

static int grid_for(int64_t total, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 152 * 16));
}

__global__ void k_mean_states(const double* __restrict__ u, int Ns, int64_t nn, double* __restrict__ ubar) {
  GRID_STRIDE(p, nn) {
    double s = 0.0;
    for (int i = 0; i < Ns; ++i) s += u[(int64_t)i * nn + p];
    ubar[p] = s / Ns;
  }
}

// D[i][p] = u_i[p] - ubar[p] on interior nodes, 0 on the boundary.
__global__ void k_center(const double* __restrict__ u, const double* __restrict__ ubar, int Ns, int n,
                         double* __restrict__ D) {
  const int64_t nn = (int64_t)n * n;
  GRID_STRIDE(e, (int64_t)Ns * nn) {
    const int64_t p = e % nn;
    const int iy = (int)(p / n), ix = (int)(p % n);
    const bool in = iy > 0 && ix > 0 && iy < n - 1 && ix < n - 1;
    D[e] = in ? u[e] - ubar[p] : 0.0;
  }
}

// C[i][j] = alpha sum_k A(i, k) B(j, k), A(i, k) = A[i*sa0 + k*sa1], B(j, k) = B[j*sb0 + k*sb1].
// 32 x 32 output tiles, 256 threads (4 outputs each), K in chunks of 32.
__global__ void k_dgemm(int M, int N, int K, const double* __restrict__ A, int64_t sa0, int64_t sa1,
                        const double* __restrict__ B, int64_t sb0, int64_t sb1, double* __restrict__ C, int64_t ldc,
                        double alpha) {
  __shared__ double ta[32][33], tb[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const bool a_kfast = sa1 == 1, b_kfast = sb1 == 1;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int q = ty; q < 32; q += 8) {
      // tile element (row, k): pick the lane index along the contiguous direction
      {
        const int r = a_kfast ? q : tx, k = a_kfast ? tx : q;
        const int gi = i0 + r, gk = k0 + k;
        ta[r][k] = (gi < M && gk < K) ? A[gi * sa0 + gk * sa1] : 0.0;
      }
      {
        const int r = b_kfast ? q : tx, k = b_kfast ? tx : q;
        const int gj = j0 + r, gk = k0 + k;
        tb[r][k] = (gj < N && gk < K) ? B[gj * sb0 + gk * sb1] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double b = tb[tx][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += ta[ty + 8 * q][k] * b;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < M && j < N) C[i * ldc + j] = alpha * acc[q];
  }
}

static void dgemm(int M, int N, int K, const double* A, int64_t sa0, int64_t sa1, const double* B, int64_t sb0,
                  int64_t sb1, double* C, int64_t ldc, double alpha, cudaStream_t s) {
  dim3 g((N + 31) / 32, (M + 31) / 32);
  k_dgemm<<<g, 256, 0, s>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, alpha);
}

// Round-robin pairing for step s of n (even) indices: (s, n-1) and ((s+k) mod (n-1), (s-k) mod (n-1)).
__global__ void k_jacobi_params(const double* __restrict__ A, int n, int step, double* __restrict__ cs,
                                int* __restrict__ pq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n / 2) return;
  const int m = n - 1;
  int p, q;
  if (k == 0) {
    p = step;
    q = m;
  } else {
    p = (step + k) % m;
    q = (step - k + m) % m;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q], apq = A[(int64_t)p * n + q];
  double c = 1.0, s = 0.0;
  if (apq != 0.0) {
    // zero A[p][q] of J^T A J with J = [[c, s], [-s, c]] (symmetric Schur decomposition)
    const double tau = (aqq - app) / (2.0 * apq);
    const double t = fabs(tau) > 1e150 ? 0.5 / tau : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  cs[2 * k] = c;
  cs[2 * k + 1] = s;
  pq[2 * k] = p;
  pq[2 * k + 1] = q;
}

// A <- J^T A (rows p, q of every pair).
__global__ void k_jacobi_rows(double* __restrict__ A, int n, const double* __restrict__ cs, const int* __restrict__ pq) {
  GRID_STRIDE(e, (int64_t)(n / 2) * n) {
    const int k = (int)(e / n), j = (int)(e % n);
    const int p = pq[2 * k], q = pq[2 * k + 1];
    const double c = cs[2 * k], s = cs[2 * k + 1];
    const double ap = A[(int64_t)p * n + j], aq = A[(int64_t)q * n + j];
    A[(int64_t)p * n + j] = c * ap - s * aq;
    A[(int64_t)q * n + j] = s * ap + c * aq;
  }
}

// A <- A J and V <- V J (columns p, q of every pair).
__global__ void k_jacobi_cols(double* __restrict__ A, double* __restrict__ V, int n, const double* __restrict__ cs,
                              const int* __restrict__ pq) {
  GRID_STRIDE(e, (int64_t)n * (n / 2)) {
    const int i = (int)(e / (n / 2)), k = (int)(e % (n / 2));
    const int p = pq[2 * k], q = pq[2 * k + 1];
    const double c = cs[2 * k], s = cs[2 * k + 1];
    double* a = A + (int64_t)i * n;
    const double ap = a[p], aq = a[q];
    a[p] = c * ap - s * aq;
    a[q] = s * ap + c * aq;
    double* v = V + (int64_t)i * n;
    const double vp = v[p], vq = v[q];
    v[p] = c * vp - s * vq;
    v[q] = s * vp + c * vq;
  }
}

// out[0] = sum_{i != j} A_ij^2, out[1] = sum_i A_ii^2.
__global__ void k_offdiag(const double* __restrict__ A, int n, double* __restrict__ out) {
  __shared__ double red[40];
  double off = 0.0, dia = 0.0;
  GRID_STRIDE(e, (int64_t)n * n) {
    const double v = A[e];
    if (e / n == e % n) dia += v * v;
    else off += v * v;
  }
  CtaCtx c{red};
  const double so = c.sum_d(off);
  const double sd = c.sum_d(dia);
  if (threadIdx.x == 0) {
    atomicAdd(out, so);
    atomicAdd(out + 1, sd);
  }
}

__global__ void k_identity(double* V, int n) {
  GRID_STRIDE(e, (int64_t)n * n) V[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void k_pad_gram(const double* __restrict__ C, int Ns, int n, double* __restrict__ A) {
  GRID_STRIDE(e, (int64_t)n * n) {
    const int i = (int)(e / n), j = (int)(e % n);
    A[e] = (i < Ns && j < Ns) ? C[(int64_t)i * Ns + j] : 0.0;
  }
}

// VselT[k][s] = V[s][order[k]] / sqrt(lambda_k)
__global__ void k_select_modes(const double* __restrict__ V, int n, int Ns, const int* __restrict__ order,
                               const double* __restrict__ inv_sqrt, int ru, double* __restrict__ VselT) {
  GRID_STRIDE(e, (int64_t)ru * Ns) {
    const int k = (int)(e / Ns), s = (int)(e % Ns);
    VselT[e] = V[(int64_t)s * n + order[k]] * inv_sqrt[k];
  }
}

// Flip each mode so that its largest-magnitude entry (first one on ties) is positive.
__global__ void k_pod_sign(double* __restrict__ phi, int64_t nn) {
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  double* row = phi + (int64_t)blockIdx.x * nn;
  double best = -1.0;
  int64_t bidx = 0;
  for (int64_t p = threadIdx.x; p < nn; p += blockDim.x) {
    const double a = fabs(row[p]);
    if (a > best) {
      best = a;
      bidx = p;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = bv[threadIdx.x + o];
      const int64_t ai = bi[threadIdx.x + o];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ai < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const bool flip = row[bi[0]] < 0.0;
  __syncthreads();
  if (flip)
    for (int64_t p = threadIdx.x; p < nn; p += blockDim.x) row[p] = -row[p];
}

extern "C" ouu_status ouu_dino_build_bases(ouu_dino_t d, const double* u_dev, int n_states, double* eig_host) {
  OUU_CHECK_ARG(d && u_dev, "null argument");
  OUU_CHECK_ARG(n_states >= d->ru && n_states <= 16384, "need r_u <= n_states <= 16384 snapshots");
  cudaStream_t st = d->stream;
  const int Ns = n_states, n = d->n;
  const int64_t nn = d->nn;
  const int np = Ns + (Ns & 1);   // Jacobi needs an even order: pad with a zero row/column
  double *D = nullptr, *C = nullptr, *A = nullptr, *V = nullptr, *cs = nullptr, *aux = nullptr, *VselT = nullptr;
  int *pq = nullptr, *ord = nullptr;
  auto cleanup = [&]() {
    cudaFree(D); cudaFree(C); cudaFree(A); cudaFree(V); cudaFree(cs); cudaFree(aux); cudaFree(VselT);
    cudaFree(pq); cudaFree(ord);
  };
  // Set-up call: temporary work arrays are allocated here and freed before returning.
  if (cudaMalloc(&D, (size_t)Ns * nn * 8) || cudaMalloc(&C, (size_t)Ns * Ns * 8) ||
      cudaMalloc(&A, (size_t)np * np * 8) || cudaMalloc(&V, (size_t)np * np * 8) || cudaMalloc(&cs, (size_t)np * 8) ||
      cudaMalloc(&pq, (size_t)np * 4) || cudaMalloc(&aux, 64) || cudaMalloc(&VselT, (size_t)d->ru * Ns * 8) ||
      cudaMalloc(&ord, (size_t)d->ru * 4)) {
    cudaGetLastError();
    cleanup();
    ouu_set_error("allocation failed in ouu_dino_build_bases");
    return OUU_ERR_OOM;
  }
  k_mean_states<<<grid_for(nn), 256, 0, st>>>(u_dev, Ns, nn, d->d_ubar);
  k_center<<<grid_for((int64_t)Ns * nn), 256, 0, st>>>(u_dev, d->d_ubar, Ns, n, D);
  dgemm(Ns, Ns, (int)nn, D, nn, 1, D, nn, 1, C, Ns, d->h * d->h, st);
  k_pad_gram<<<grid_for((int64_t)np * np), 256, 0, st>>>(C, Ns, np, A);
  k_identity<<<grid_for((int64_t)np * np), 256, 0, st>>>(V, np);
  double h_aux[2];
  int sweeps = 0;
  for (; sweeps < 30; ++sweeps) {
    for (int s = 0; s < np - 1; ++s) {
      k_jacobi_params<<<(np / 2 + 127) / 128, 128, 0, st>>>(A, np, s, cs, pq);
      k_jacobi_rows<<<grid_for((int64_t)(np / 2) * np), 256, 0, st>>>(A, np, cs, pq);
      k_jacobi_cols<<<grid_for((int64_t)np * (np / 2)), 256, 0, st>>>(A, V, np, cs, pq);
    }
    OUU_CUDA_TRY(cudaMemsetAsync(aux, 0, 16, st));
    k_offdiag<<<256, 256, 0, st>>>(A, np, aux);
    OUU_CUDA_TRY(cudaMemcpyAsync(h_aux, aux, 16, cudaMemcpyDeviceToHost, st));
    OUU_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(h_aux[0] > 1e-30 * h_aux[1])) break;
  }
  // eigenvalues: diagonal of A, sorted descending
  std::vector<double> Ah((size_t)np * np);
  OUU_CUDA_TRY(cudaMemcpyAsync(Ah.data(), A, (size_t)np * np * 8, cudaMemcpyDeviceToHost, st));
  OUU_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> lam(Ns);
  for (int i = 0; i < Ns; ++i) lam[i] = Ah[(size_t)i * np + i];
  std::vector<int> order(Ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
  if (eig_host)
    for (int i = 0; i < Ns; ++i) eig_host[i] = lam[order[i]];
  std::vector<double> isq(d->ru);
  for (int k = 0; k < d->ru; ++k) {
    if (!(lam[order[k]] > 0.0)) {
      cleanup();
      ouu_set_error("snapshot set has rank < r_u");
      return OUU_ERR_INVALID_ARG;
    }
    isq[k] = 1.0 / std::sqrt(lam[order[k]]);
  }
  std::vector<int> ordk(order.begin(), order.begin() + d->ru);
  OUU_CUDA_TRY(cudaMemcpyAsync(ord, ordk.data(), (size_t)d->ru * 4, cudaMemcpyHostToDevice, st));
  double* d_is = nullptr;
  if (cudaMalloc(&d_is, (size_t)d->ru * 8) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    ouu_set_error("allocation failed in ouu_dino_build_bases");
    return OUU_ERR_OOM;
  }
  OUU_CUDA_TRY(cudaMemcpyAsync(d_is, isq.data(), (size_t)d->ru * 8, cudaMemcpyHostToDevice, st));
  k_select_modes<<<grid_for((int64_t)d->ru * Ns), 256, 0, st>>>(V, np, Ns, ord, d_is, d->ru, VselT);
  // Phi[k][p] = sum_s VselT[k][s] D[s][p]
  dgemm(d->ru, (int)nn, Ns, VselT, Ns, 1, D, 1, nn, d->d_phi64, nn, 1.0, st);
  k_pod_sign<<<d->ru, 256, 0, st>>>(d->d_phi64, nn);
  OUU_CUDA_TRY(cudaGetLastError());
  OUU_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(d_is);
  cleanup();
  // output scale of the network: RMS of each kept mode over the snapshots, sqrt(lambda_k / Ns)
  std::vector<float> sc(d->ru);
  for (int k = 0; k < d->ru; ++k) sc[k] = (float)std::sqrt(lam[order[k]] / Ns);
  OUU_CUDA_TRY(cudaMemcpyAsync(d->d_oscale, sc.data(), (size_t)d->ru * 4, cudaMemcpyHostToDevice, st));
  return dino_install_bases(d);
}
