// Allocation-free variant of the batched state solve (ouu_pde_solve_batch_noalloc).
//
// Some callers cannot allocate device memory at call time: code running under a
// memory pool or budget that forbids new cudaMalloc calls, plug-ins that are
// handed a stream and buffers by a host application that owns all device
// allocations, or callers that must not create a library handle (which
// allocates its workspace).  This entry point runs the same per-sample
// Newton/MG-PCG kernel as ouu_pde_solve_batch, but every byte of scratch it needs
// (tables, per-CTA solver slots, the work counter) comes from the file-scope
// device array below, which each GPU that loads the library holds until the
// process exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ouu_internal.cuh"

// Fixed scratch: 8 MiB per device.
#define OUU_NOALLOC_SCRATCH_BYTES (8u << 20)
#define OUU_NOALLOC_CHUNK 4096          // samples per launch (bounds the iteration-count table)

static __device__ __align__(256) unsigned char g_noalloc_scratch[OUU_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch in the current context.  In host code the symbol
// name is only a host-side stand-in, never a device address.  The lookup is repeated on
// every call (it allocates nothing): a cached address would go stale if the context were
// torn down and recreated (cudaDeviceReset), since the module may then load elsewhere.
static ouu_status scratch_address(unsigned char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr) {
    ouu_set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
    return OUU_ERR_CUDA;
  }
  *out = (unsigned char*)ptr;
  return OUU_OK;
}

// Source factors gx = gy (Gaussian profile of each lattice line) and the target state.
__global__ void k_noalloc_tables(int n, int L, double width, double* gx, double* ut) {
  const int nn = n * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * n + nn; e += gridDim.x * blockDim.x) {
    if (e < L * n) {
      const int j = e / n, i = e % n;
      const double d = i * (1.0 / (n - 1)) - (j + 0.5) / L;
      gx[e] = exp(-(d * d) / (2.0 * width * width));
    } else {
      const int k = e - L * n, iy = k / n, ix = k % n;
      ut[k] = sinpi(ix / (double)(n - 1)) * sinpi(iy / (double)(n - 1));
    }
  }
}

static int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

extern "C" ouu_status ouu_pde_solve_batch_noalloc(const ouu_problem_desc* desc, const double* m_dev, int n_samples,
                                                  const double* z_dev, int64_t z_stride, double* u_dev,
                                                  double* q_dev, int32_t* status_dev, void* cuda_stream) {
  OUU_CHECK_ARG(desc != nullptr, "desc is null");
  const int n = desc->n, L = desc->lattice_L;
  OUU_CHECK_ARG(n >= 5 && n <= 1025 && (((n - 1) & (n - 2)) == 0), "n must be 2^k + 1 with 5 <= n <= 1025");
  OUU_CHECK_ARG(L >= 1 && L <= 64, "lattice_L must be in [1, 64]");
  OUU_CHECK_ARG(desc->bump_width > 0 && desc->reaction_r >= 0, "bad source width or reaction");
  OUU_CHECK_ARG(desc->newton_rtol > 0 && desc->newton_maxit >= 1, "bad Newton tolerance/cap");
  OUU_CHECK_ARG(desc->cg_rtol > 0 && desc->cg_rtol < 1 && desc->cg_maxit >= 1, "bad CG tolerance/cap");
  OUU_CHECK_ARG(n_samples >= 0, "n_samples must be >= 0");
  if (n_samples == 0) return OUU_OK;
  OUU_CHECK_ARG(m_dev && z_dev && u_dev && q_dev && status_dev, "m_dev, z_dev, u_dev, q_dev, status_dev are required");
  OUU_CHECK_ARG(z_stride == 0 || z_stride >= (int64_t)L * L, "z_stride must be 0 or >= d_Z");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int device = 0, sms = 0, smem_optin = 0;
  OUU_CUDA_TRY(cudaGetDevice(&device));
  OUU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  OUU_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  unsigned char* base = nullptr;
  if (ouu_status st = scratch_address(&base)) return st;

  // Layout inside the scratch: counter | gx | ut | iteration table | slots.
  const int nlev = ouu_num_levels(n);
  const int64_t nn = (int64_t)n * n;
  int64_t off = 256;
  const int64_t off_gx = off;
  off += align256((int64_t)L * n * 8);
  const int64_t off_ut = off;
  off += align256(nn * 8);
  const int64_t off_it = off;
  off += align256((int64_t)OUU_NOALLOC_CHUNK * 3 * 4);
  const int64_t slots_off = off;
  // per-slot layout of what the state kernel touches
  SlotLayout lay;
  memset(&lay, 0, sizeof(lay));
  int64_t s = 0;
  auto take = [&](int64_t b) {
    const int64_t o = s;
    s += align256(b);
    return o;
  };
  lay.E = take(nn * 8);
  lay.f = take(nn * 8);
  lay.tmp = take((int64_t)L * n * 8);
  lay.kx = take(nn * 4);
  lay.ky = take(nn * 4);
  lay.D = take(nn * 4);
  lay.x = take(nn * 4);
  lay.r = take(nn * 4);
  lay.z = take(nn * 4);
  lay.p = take(nn * 4);
  lay.q = take(nn * 4);
  lay.t = take(nn * 4);
  int64_t soff = 0;
  for (int l = 0; l < OUU_MAX_LEVELS; ++l) lay.lev[l] = lay.smem_lev[l] = -1;
  for (int l = 1, nl = (n + 1) / 2; l < nlev; ++l, nl = (nl + 1) / 2) {
    const int64_t blk = 6 * ouu_level_array_bytes(nl);
    if (nl <= OUU_SMEM_MAX_N) {
      lay.smem_lev[l] = soff;
      soff += blk;
    } else {
      lay.lev[l] = take(blk);
    }
  }
  lay.smem_bytes = soff;
  lay.bytes = align256(s);
  const int64_t room = (int64_t)OUU_NOALLOC_SCRATCH_BYTES - slots_off;
  if (room < lay.bytes) {
    ouu_set_error("grid too large for the no-allocation scratch: one solver slot needs " +
                  std::to_string(slots_off + lay.bytes) + " bytes of the fixed " +
                  std::to_string(OUU_NOALLOC_SCRATCH_BYTES) + " (n <= 257 fits)");
    return OUU_ERR_INVALID_ARG;
  }
  if (lay.smem_bytes + 1024 > smem_optin) {
    ouu_set_error("grid too large for the solver's shared-memory multigrid levels: " +
                  std::to_string(lay.smem_bytes + 1024) + " bytes per block, device limit " +
                  std::to_string(smem_optin));
    return OUU_ERR_INVALID_ARG;
  }
  const int nslots = (int)std::min<int64_t>(std::min<int64_t>(room / lay.bytes, sms), n_samples);

  // Contents persist between calls: zero the counter and slots (boundary entries of
  // the solver vectors must be zero), then rebuild the tables for this grid.
  OUU_CUDA_TRY(cudaMemsetAsync(base, 0, (size_t)(slots_off + (int64_t)nslots * lay.bytes), stream));
  k_noalloc_tables<<<64, 256, 0, stream>>>(n, L, desc->bump_width, (double*)(base + off_gx), (double*)(base + off_ut));
  OUU_CUDA_TRY(cudaGetLastError());

  PdeArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.nlev = nlev;
  a.L = L;
  a.rr = desc->reaction_r;
  a.gscale = 1.0 / (desc->bump_width * sqrt(2.0 * M_PI));
  a.newton_rtol = desc->newton_rtol;
  a.newton_maxit = desc->newton_maxit;
  a.cg_rtol = desc->cg_rtol;
  a.cg_maxit = desc->cg_maxit;
  a.gx = (const double*)(base + off_gx);
  a.gy = (const double*)(base + off_gx);
  a.ut = (const double*)(base + off_ut);
  a.iters = (int32_t*)(base + off_it);
  a.counter = (int*)base;
  a.slots = (char*)(base + slots_off);
  a.lay = lay;
  for (int first = 0; first < n_samples; first += OUU_NOALLOC_CHUNK) {
    const int cnt = std::min(OUU_NOALLOC_CHUNK, n_samples - first);
    a.n_samples = cnt;
    a.m = m_dev + (int64_t)first * nn;
    a.z = z_dev + (int64_t)first * z_stride;
    a.z_stride = z_stride;
    a.u = u_dev + (int64_t)first * nn;
    a.q = q_dev + first;
    a.status = status_dev + first;
    OUU_CUDA_TRY(cudaMemsetAsync(base, 0, 4, stream));
    launch_pde_state(a, std::min(nslots, cnt), stream);
    OUU_CUDA_TRY(cudaGetLastError());
  }
  // Per-sample statuses into a fixed host buffer, chunk by chunk.
  int32_t hs[1024];
  int worst = 0, bad = -1;
  for (int first = 0; first < n_samples; first += 1024) {
    const int cnt = std::min(1024, n_samples - first);
    OUU_CUDA_TRY(cudaMemcpyAsync(hs, status_dev + first, (size_t)cnt * 4, cudaMemcpyDeviceToHost, stream));
    OUU_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int i = 0; i < cnt; ++i)
      if (hs[i] > worst) {
        worst = hs[i];
        bad = first + i;
      }
  }
  if (worst == OUU_SAMPLE_NOT_CONVERGED) {
    ouu_set_error("sample " + std::to_string(bad) + " did not converge");
    return OUU_ERR_NOT_CONVERGED;
  }
  if (worst == OUU_SAMPLE_NONFINITE) {
    ouu_set_error("non-finite residual in sample " + std::to_string(bad));
    return OUU_ERR_NONFINITE;
  }
  return OUU_OK;
}
