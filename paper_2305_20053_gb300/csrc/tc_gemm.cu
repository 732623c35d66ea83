// tcgen05 + TMA BF16 GEMM with fused epilogues (see tc_gemm.cuh).
//
// CTA = 12 warps (384 threads), one 128 x BN output tile:
//   warp 0 (one lane): TMA producer, 4- or 5-stage ring of 64-wide K blocks (SWIZZLE_128B)
//   warp 1 (one lane): tcgen05.mma issuer (kind::f16, BF16 x BF16 -> FP32 in TMEM);
//                      warp 1 also allocates / frees the tensor memory
//   warps 2..5       : TMEM -> shared staging tile, one accumulator row (TMEM lane) per thread
//   all 12 warps     : the fused epilogue over the staged tile, and the global stores
// Every mbarrier wait is bounded (about 2 s of SM clock); on a timeout the CTA
// drains its own TMA copies (bounded), frees its tensor memory and raises *err.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "gelu.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#define GEMM_BM 128
#define GEMM_BK 64
#define GEMM_THREADS 384

static __device__ __forceinline__ float gelu_f(float x) { return gelu_fwd(x); }
static __device__ __forceinline__ float gelu_d1f(float x) { return gelu_d1(x); }

// Pipeline depth: four stages; five for the wide tiles of long-K projections (one CTA per
// SM) where five still fit in 227 KB of shared memory (BN = 208: 210 KB; BN = 256 would need 240).
template <int BN>
struct GemmStages {
  static constexpr int value = (BN > 128 && 5 * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) <= 216 * 1024) ? 5 : 4;
};

// Epilogue B: one pass over the staged tile in quads of four consecutive columns,
// consecutive threads on consecutive quads of a row (16-byte shared loads, 16-byte FP32
// and 8-byte BF16 global stores when ep.vec).  One compact loop per mode keeps the code
// that every CTA runs once small.  MODE 7 = split-K partial sums, added atomically.
template <int BN, int MODE>
static __device__ __forceinline__ void epi_quads(float* stage, const float* sbias, const float* sscale,
                                                 const float* sadd, float* rowsum, int m0, int n0, int M, int N,
                                                 const EpiParams& ep, bool keep) {
  constexpr int SROW = BN + 4, QPR = BN / 4;
  const bool vec = ep.vec != 0;
  const float alpha = ep.alpha;
  if (MODE == EPI_DECODE) {
    // whole rows per warp, lanes over consecutive columns (coalesced rows of any length or
    // alignment); the row's squared differences summed per lane, then once per row by a warp
    // reduction
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int tr = warp; tr < GEMM_BM; tr += GEMM_THREADS / 32) {
      const int r = m0 + tr;
      if (r >= M) break;
      float* orow = ep.out_f32 + (size_t)r * ep.ld_f32;
      const float* srow = stage + tr * SROW;
      float sq = 0.f;
#pragma unroll 4
      for (int cc = lane; cc < BN; cc += 32) {
        const int c = n0 + cc;
        if (c < N) {
          const float v = srow[cc] + sadd[cc];
          orow[c] = v;
          const float d = v - sscale[cc];   // sscale holds col_ref in this mode
          sq = fmaf(d, d, sq);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) rowsum[tr] = sq;
    }
    return;
  }
  if (MODE == EPI_QOI) {
    // whole rows per warp, lanes over quads, the row's quadratic by a warp reduction
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int tr = warp; tr < GEMM_BM; tr += GEMM_THREADS / 32) {
      const int r = m0 + tr;
      if (r >= M) break;
      float sq = 0.f;
      for (int qd = lane; qd < QPR; qd += 32) {
        const int cc = 4 * qd, c = n0 + cc;
        if (c >= N) break;
        const int nv = min(4, N - c);
        const float4 a4 = *reinterpret_cast<const float4*>(stage + tr * SROW + cc);
        const float acc[4] = {a4.x, a4.y, a4.z, a4.w};
        float y[4], o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          y[j] = (acc[j] + sbias[cc + j]) * sscale[cc + j];
          const float v = j < nv ? y[j] + sadd[cc + j] : 0.f;
          o[j] = v * sscale[cc + j];
          sq += v * v;
        }
        float* of = ep.out_f32 ? ep.out_f32 + (size_t)r * ep.ld_f32 + c : nullptr;
        __nv_bfloat16* ob = ep.out_bf16 ? ep.out_bf16 + (size_t)r * ep.ld_bf16 + c : nullptr;
        if (vec && nv == 4) {
          if (of) *reinterpret_cast<float4*>(of) = make_float4(y[0], y[1], y[2], y[3]);
          if (ob) {
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
            *reinterpret_cast<uint2*>(ob) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
          }
        } else {
          for (int j = 0; j < nv; ++j) {
            if (of) of[j] = y[j];
            if (ob) ob[j] = __float2bfloat16(o[j]);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) rowsum[tr] = sq;
    }
    return;
  }
#pragma unroll 2
  for (int e = threadIdx.x; e < GEMM_BM * QPR; e += GEMM_THREADS) {
    const int tr = e / QPR, cc = (e - tr * QPR) * 4, r = m0 + tr, c = n0 + cc;
    if (r >= M || c >= N) continue;
    const int nv = min(4, N - c);
    const bool full = vec && nv == 4;
    float* sp = stage + tr * SROW + cc;
    const float4 a4 = *reinterpret_cast<const float4*>(sp);
    const float acc[4] = {a4.x, a4.y, a4.z, a4.w};
    float y[4], o[4];
    if (MODE == EPI_DGELU_SCALE || MODE == EPI_SCALE) {
      const float* ap = ep.aux + (size_t)(r / ep.aux_rdiv) * ep.ld_aux + c;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      if (full) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(ap));
        x[0] = t.x, x[1] = t.y, x[2] = t.z, x[3] = t.w;
      } else {
        for (int j = 0; j < nv; ++j) x[j] = ap[j];
      }
      if (MODE == EPI_SCALE) {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = y[j] = acc[j] * x[j];
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = y[j] = acc[j] * gelu_d1f(x[j]);
      }
    } else if (MODE == EPI_GELU_D) {
#pragma unroll
      for (int j = 0; j < 4; ++j) gelu_and_d1(acc[j] + sbias[cc + j], o[j], y[j]);   // one exp for both
    } else if (MODE == EPI_GELU) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        y[j] = acc[j] + sbias[cc + j];
        o[j] = gelu_f(y[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = y[j] = (alpha * acc[j] + sbias[cc + j]) * sscale[cc + j];
    }
    float* of = ep.out_f32 ? ep.out_f32 + (size_t)r * ep.ld_f32 + c : nullptr;
    if (MODE == 7) {
      if (full) {
        atomicAdd(reinterpret_cast<float4*>(of), make_float4(y[0], y[1], y[2], y[3]));
      } else {
        for (int j = 0; j < nv; ++j) atomicAdd(of + j, y[j]);
      }
      continue;
    }
    __nv_bfloat16* ob = ep.out_bf16 ? ep.out_bf16 + (size_t)r * ep.ld_bf16 + c : nullptr;
    __nv_bfloat16* o2 = ep.out2_bf16 ? ep.out2_bf16 + (size_t)r * ep.ld2 + c : nullptr;
    if (full) {
      if (of) {
        float4 v = make_float4(y[0], y[1], y[2], y[3]);
        if (ep.accumulate) {
          const float4 old = *reinterpret_cast<const float4*>(of);
          v.x += old.x, v.y += old.y, v.z += old.z, v.w += old.w;
        }
        *reinterpret_cast<float4*>(of) = v;
      }
      if (ob) {
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
        *reinterpret_cast<uint2*>(ob) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
      }
      if (o2) {
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(acc[0], acc[1]), p1 = __floats2bfloat162_rn(acc[2], acc[3]);
        *reinterpret_cast<uint2*>(o2) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
      }
    } else {
      for (int j = 0; j < nv; ++j) {
        if (of) of[j] = ep.accumulate ? of[j] + y[j] : y[j];
        if (ob) ob[j] = __float2bfloat16(o[j]);
        if (o2) o2[j] = __float2bfloat16(acc[j]);
      }
    }
    if (keep) *reinterpret_cast<float4*>(sp) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                EpiParams ep, int* err) {
  constexpr int GEMM_STAGES = GemmStages<BN>::value;
  constexpr uint32_t A_BYTES = GEMM_BM * GEMM_BK * 2;
  constexpr uint32_t B_BYTES = BN * GEMM_BK * 2;
  constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
  static_assert(B_BYTES % 1024 == 0, "stage buffers must stay 1024-byte aligned");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sa = smem;
  uint8_t* sb = smem + GEMM_STAGES * A_BYTES;
  uint64_t* full = (uint64_t*)(sb + GEMM_STAGES * B_BYTES);
  uint64_t* empty = full + GEMM_STAGES;
  uint64_t* tfull = empty + GEMM_STAGES;
  uint32_t* tslot = (uint32_t*)(tfull + 1);
  __shared__ volatile int s_fail;
  __shared__ __align__(16) float s_bias[BN], s_scale[BN], s_add[BN];
  __shared__ float s_rowsum[GEMM_BM];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * GEMM_BM, n0 = blockIdx.x * BN;
  // split-K: CTA z owns K blocks [kb_lo, kb_lo + KB)
  const int KB_all = (K + GEMM_BK - 1) / GEMM_BK;
  const int per = (KB_all + gridDim.z - 1) / gridDim.z;
  const int kb_lo = blockIdx.z * per;
  const int KB = max(0, min(KB_all, kb_lo + per) - kb_lo);
  const bool splitk = gridDim.z > 1;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < GEMM_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, TMEM_COLS);
  if (warp == 0 && lane < 2) tmap_prefetch(lane == 0 ? &ta : &tb);
  pdl_wait();   // everything below reads or writes what earlier kernels produce or consume
  for (int i = threadIdx.x; i < BN; i += GEMM_THREADS) {   // per-column epilogue constants
    const int c = n0 + i;
    s_bias[i] = (c < N && ep.bias && blockIdx.z == 0) ? ep.bias[c] : 0.f;
    s_scale[i] = ep.mode == EPI_DECODE ? (c < N ? ep.col_ref[c] : 0.f) : (c < N && ep.col_scale) ? ep.col_scale[c] : 1.f;
    s_add[i] = (c < N && ep.col_add) ? ep.col_add[c] : 0.f;
  }
  for (int i = threadIdx.x; i < GEMM_BM; i += GEMM_THREADS) s_rowsum[i] = 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % GEMM_STAGES;
        const uint32_t ph = (uint32_t)(kb / GEMM_STAGES) & 1u;
        if (kb >= GEMM_STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
          s_fail = 1;
          break;
        }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sa + s * A_BYTES, &ta, (kb_lo + kb) * GEMM_BK, m0, &full[s]);
        tma_load_2d(sb + s * B_BYTES, &tb, (kb_lo + kb) * GEMM_BK, n0, &full[s]);
        issued = kb + 1;
      }
      // Drain: the last copy issued into every stage must have landed before exit.
      for (int kb = std::max(0, issued - GEMM_STAGES); kb < issued; ++kb)
        if (!mbar_wait(&full[kb % GEMM_STAGES], (uint32_t)(kb / GEMM_STAGES) & 1u)) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(GEMM_BM >> 4) << 24);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % GEMM_STAGES;
        const uint32_t ph = (uint32_t)(kb / GEMM_STAGES) & 1u;
        if (!mbar_wait(&full[s], ph)) {
          s_fail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sa + s * A_BYTES), b0 = smem_u32(sb + s * B_BYTES);
#pragma unroll
        for (int k = 0; k < GEMM_BK / 16; ++k)
          tc_mma(tmem, smem_desc_sw128(a0 + k * 32), smem_desc_sw128(b0 + k * 32), idesc, (kb | k) != 0);
        tc_commit(&empty[s]);
      }
      tc_commit(tfull);   // completes once every MMA issued above has finished
    }
  } else if (warp < 6) {
    // Epilogue A (warps 2..5): TMEM -> shared staging tile, one accumulator row per thread
    // (warp w may read TMEM lanes 32 (w % 4) .. +31).  The pipeline buffers are free once
    // every MMA has completed.
    const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull, 0) ? 1 : 0);
    tc_fence_after();
    const int q = warp & 3;
    // Row stride BN + 4 floats (4 x an odd number): the 16-byte stores of eight
    // consecutive rows fall in distinct bank groups.
    float* stage = (float*)smem;
    constexpr int SROW = BN + 4;
    float4* srow = reinterpret_cast<float4*>(stage + (q * 32 + lane) * SROW);
    if (!ok && lane == 0) s_fail = 1;
    if (ok && KB > 0) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          srow[(c0 + j) >> 2] = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
      }
    } else if (ok) {   // empty K range (split-K remainder): contributes zero
      for (int c = 0; c < BN; c += 4) srow[c >> 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  tc_fence_before();
  __syncthreads();   // staging tile complete; producer and MMA roles are done
  {
    constexpr int SROW = BN + 4;
    float* stage = (float*)smem;
    const bool run = !s_fail;
    const bool keep = ep.out_t_bf16 != nullptr && !splitk;
    if (run) {
      if (splitk)
        epi_quads<BN, 7>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, false);
      else if (ep.mode == EPI_LINEAR)
        epi_quads<BN, EPI_LINEAR>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
      else if (ep.mode == EPI_GELU)
        epi_quads<BN, EPI_GELU>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
      else if (ep.mode == EPI_GELU_D)
        epi_quads<BN, EPI_GELU_D>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
      else if (ep.mode == EPI_SCALE)
        epi_quads<BN, EPI_SCALE>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
      else if (ep.mode == EPI_QOI)
        epi_quads<BN, EPI_QOI>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
      else if (ep.mode == EPI_DECODE)
        epi_quads<BN, EPI_DECODE>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, false);
      else
        epi_quads<BN, EPI_DGELU_SCALE>(stage, s_bias, s_scale, s_add, s_rowsum, m0, n0, M, N, ep, keep);
    }
    if (ep.mode == EPI_QOI && run) {   // the tile holds whole rows: finish the per-row quadratic
      __syncthreads();
      for (int tr = threadIdx.x; tr < GEMM_BM; tr += GEMM_THREADS)
        if (m0 + tr < M) ep.out_q[m0 + tr] = ep.qconst + 0.5 * (double)s_rowsum[tr];
    }
    if (ep.mode == EPI_DECODE && run) {   // this tile's columns of each row's sum
      __syncthreads();
      for (int tr = threadIdx.x; tr < GEMM_BM; tr += GEMM_THREADS)
        if (m0 + tr < M) atomicAdd(&ep.out_q[m0 + tr], ep.qconst * (double)s_rowsum[tr]);
    }
    if (ep.out_t_bf16 && !splitk) {
      // Epilogue C (all warps): transposed output, consecutive threads on consecutive rows.
      __syncthreads();
      if (run)
        for (int e = threadIdx.x; e < GEMM_BM * BN; e += GEMM_THREADS) {
          const int tr = e % GEMM_BM, cc = e / GEMM_BM, r = m0 + tr, c = n0 + cc;
          if (r < M && c < N) ep.out_t_bf16[(size_t)c * ep.ld_t + r] = __float2bfloat16(stage[tr * SROW + cc]);
        }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool ouu_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, uint32_t esize, const void* base, uint64_t d0, uint64_t d1,
                 uint64_t stride1_bytes, uint32_t box0, uint32_t box1, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || ((uintptr_t)base & 15) || (stride1_bytes % 16) || ((uint64_t)box0 * esize) % 16) return false;
  cuuint64_t dims[2] = {d0, d1};
  cuuint64_t strides[1] = {stride1_bytes};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool ouu_tmap_bf16(CUtensorMap* map, const void* base, uint64_t k, uint64_t rows, uint64_t ld, uint32_t box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || ((uintptr_t)base & 15) || (ld % 8) || k > ld) return false;
  cuuint64_t dims[2] = {k, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {GEMM_BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
static ouu_status launch_bn(const CUtensorMap& ta, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                            const EpiParams& ep, int* err, cudaStream_t s, int splits) {
  constexpr int GEMM_STAGES = GemmStages<BN>::value;
  static_assert((size_t)GEMM_STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) >= (size_t)GEMM_BM * (BN + 4) * 4,
                "the pipeline buffers must hold the epilogue staging tile");
  CUtensorMap tb;
  if (!ouu_tmap_bf16(&tb, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, BN)) {
    ouu_set_error("tensor map for GEMM operand B failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  const size_t smem = 1024 + (size_t)GEMM_STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) +
                      (2 * GEMM_STAGES + 1) * 8 + 16;
  OUU_CUDA_TRY(ouu_smem_limit((const void*)k_gemm_bf16<BN>, smem));
  dim3 grid((N + BN - 1) / BN, (M + GEMM_BM - 1) / GEMM_BM, splits);
  OUU_CUDA_TRY(launch_pdl(k_gemm_bf16<BN>, grid, dim3(GEMM_THREADS), smem, s, ta, tb, M, N, K, ep, err));
  return OUU_OK;
}

static ouu_status launch_by_bn(int bn, const CUtensorMap& ta, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                               const EpiParams& e2, int* err, cudaStream_t s, int splits) {
  switch (bn) {
    case 256: return launch_bn<256>(ta, B, ldb, M, N, K, e2, err, s, splits);
    case 208: return launch_bn<208>(ta, B, ldb, M, N, K, e2, err, s, splits);
    case 128: return launch_bn<128>(ta, B, ldb, M, N, K, e2, err, s, splits);
    case 112: return launch_bn<112>(ta, B, ldb, M, N, K, e2, err, s, splits);
    case 80: return launch_bn<80>(ta, B, ldb, M, N, K, e2, err, s, splits);
    default: return launch_bn<64>(ta, B, ldb, M, N, K, e2, err, s, splits);
  }
}

// Autotuner state: the measured best N tile per (M, N, K, epilogue mode, split) shape.
struct GemmKey {
  int M, N, K, mode, splits;
  bool operator<(const GemmKey& o) const {
    return std::tie(M, N, K, mode, splits) < std::tie(o.M, o.N, o.K, o.mode, o.splits);
  }
};
static std::map<GemmKey, int> g_tuned;
static std::mutex g_tune_mu;
static std::atomic<int> g_autotune{0};

ouu_status ouu_gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                         const EpiParams& ep, int* err, cudaStream_t s, int splits) {
  OUU_CHECK_ARG(M >= 1 && N >= 1 && K >= 1, "GEMM sizes must be positive");
  OUU_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0, "GEMM operands must be 16-byte aligned");
  OUU_CHECK_ARG(lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K, "GEMM leading dimensions: multiple of 8, >= K");
  OUU_CHECK_ARG(ep.mode >= EPI_LINEAR && ep.mode <= EPI_DECODE, "unknown epilogue mode");
  OUU_CHECK_ARG(ep.mode != EPI_DECODE || (ep.out_f32 && ep.out_q && ep.col_add && ep.col_ref && splits == 1 &&
                                          !ep.accumulate && !ep.out_bf16 && !ep.out_t_bf16 && !ep.out2_bf16),
                "EPI_DECODE needs out_f32, out_q, col_add and col_ref, one FP32 output and no split-K");
  OUU_CHECK_ARG(ep.mode != EPI_QOI || (N <= 256 && ep.out_q && ep.col_scale && ep.col_add && splits == 1 &&
                                       !ep.accumulate && !ep.out_t_bf16),
                "EPI_QOI needs N <= 256, out_q, col_scale and col_add, and no split-K");
  OUU_CHECK_ARG((ep.mode != EPI_DGELU_SCALE && ep.mode != EPI_SCALE) || (ep.aux && ep.aux_rdiv >= 1),
                "EPI_DGELU_SCALE and EPI_SCALE need aux");
  OUU_CHECK_ARG(splits >= 1 && splits <= 64, "split-K factor in [1, 64]");
  {   // every K slice must own a K block: an empty slice would add an unwritten accumulator
    const int kb_all = (K + GEMM_BK - 1) / GEMM_BK, per = (kb_all + splits - 1) / splits;
    OUU_CHECK_ARG((splits - 1) * per < kb_all, "split-K factor leaves a slice without a K block");
  }
  OUU_CHECK_ARG(splits == 1 || (ep.mode == EPI_LINEAR && ep.out_f32 && !ep.out_bf16 && !ep.out_t_bf16 &&
                                !ep.out2_bf16 && !ep.col_scale && !ep.accumulate),
                "split-K supports one FP32 output of EPI_LINEAR, accumulated into a zeroed buffer");
  // 16-byte FP32 / 8-byte BF16 epilogue accesses need aligned bases and leading dimensions
  // that are multiples of four elements; otherwise every element is stored on its own.
  auto al = [](const void* q, uintptr_t a, int ld) { return q == nullptr || (((uintptr_t)q % a) == 0 && ld % 4 == 0); };
  EpiParams e2 = ep;
  e2.vec = al(ep.out_f32, 16, ep.ld_f32) && al(ep.out_bf16, 8, ep.ld_bf16) && al(ep.out2_bf16, 8, ep.ld2) &&
           ((ep.mode != EPI_DGELU_SCALE && ep.mode != EPI_SCALE) || al(ep.aux, 16, ep.ld_aux));
  CUtensorMap ta;
  if (!ouu_tmap_bf16(&ta, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, GEMM_BM)) {
    ouu_set_error("tensor map for GEMM operand A failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  // Autotuned tile for this shape, if the tuner has timed it (see ouu_gemm_set_autotune).
  const GemmKey key{M, N, K, ep.mode, splits};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return launch_by_bn(it->second, ta, B, ldb, M, N, K, e2, err, s, splits);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  // Timing runs would add into outputs that accumulate (accumulate flag, split-K atomics).
  if (g_autotune && cap == cudaStreamCaptureStatusNone && !ep.accumulate && splits == 1) {
    int best_bn = 0;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int bn : {256, 208, 128, 112, 80, 64}) {
      if (ep.mode == EPI_QOI && bn < N) continue;
      if (launch_by_bn(bn, ta, B, ldb, M, N, K, e2, err, s, splits) != OUU_OK) continue;   // warm-up
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch_by_bn(bn, ta, B, ldb, M, N, K, e2, err, s, splits);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best_bn = bn;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_bn) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = best_bn;
      return launch_by_bn(best_bn, ta, B, ldb, M, N, K, e2, err, s, splits);
    }
  }
  // N tile: a CTA's time is mostly fixed latency (TMA round trips, MMA commit, epilogue)
  // plus a part that grows with BN, and tiles beyond one per SM run in a further wave;
  // pick the tile that minimises waves x (BN + 64) (ties: the wider tile).
  static const int sms = [] {   // initialised once, thread-safe (one device per process)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  static const int cands[] = {256, 208, 128, 112, 80, 64};
  int best = 64;
  long best_cost = 1L << 60;
  const long mt = (long)((M + GEMM_BM - 1) / GEMM_BM) * splits;
  for (int bn : cands) {
    if (ep.mode == EPI_QOI && bn < N) continue;   // whole rows in one tile
    const long tiles = mt * ((N + bn - 1) / bn);
    const long cost = ((tiles + sms - 1) / sms) * (bn + 64);
    if (cost < best_cost) {
      best_cost = cost;
      best = bn;
    }
  }
  return launch_by_bn(best, ta, B, ldb, M, N, K, e2, err, s, splits);
}

void ouu_gemm_set_autotune(int on) { g_autotune = on; }

int ouu_gemm_tuned_count() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tuned.size();
}

// Kernel-level entry used by the GEMM numerics test (declared in include/ouu_kernels.h).
extern "C" ouu_status ouu_kernel_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                           int mode, float alpha, const float* bias, const float* aux, int ld_aux,
                                           int aux_rdiv, float* out_f32, int ld_f32, int accumulate, void* out_bf16,
                                           int ld_bf16, void* out_t_bf16, int ld_t, void* out2_bf16, int ld2,
                                           int* err_dev, void* stream) {
  EpiParams ep;
  std::memset(&ep, 0, sizeof(ep));
  ep.mode = mode;
  ep.alpha = alpha;
  ep.bias = bias;
  ep.col_scale = nullptr;
  ep.out_f32 = out_f32;
  ep.ld_f32 = ld_f32;
  ep.accumulate = accumulate;
  ep.out_bf16 = (__nv_bfloat16*)out_bf16;
  ep.ld_bf16 = ld_bf16;
  ep.out_t_bf16 = (__nv_bfloat16*)out_t_bf16;
  ep.ld_t = ld_t;
  ep.out2_bf16 = (__nv_bfloat16*)out2_bf16;
  ep.ld2 = ld2;
  ep.aux = aux;
  ep.ld_aux = ld_aux;
  ep.aux_rdiv = aux_rdiv;
  OUU_CHECK_ARG(err_dev != nullptr, "err_dev is required");
  return ouu_gemm_bf16((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, M, N, K, ep, err_dev,
                       (cudaStream_t)stream, 1);
}

// Kernel-level entry of the reduced-QoI epilogue (declared in include/ouu_kernels.h).
extern "C" ouu_status ouu_kernel_gemm_qoi_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                               const float* bias, const float* col_scale, const float* col_add,
                                               double qconst, float* out_f32, int ld_f32, void* out_bf16, int ld_bf16,
                                               double* out_q, int* err_dev, void* stream) {
  EpiParams ep;
  std::memset(&ep, 0, sizeof(ep));
  ep.mode = EPI_QOI;
  ep.alpha = 1.f;
  ep.bias = bias;
  ep.col_scale = col_scale;
  ep.col_add = col_add;
  ep.qconst = qconst;
  ep.out_f32 = out_f32;
  ep.ld_f32 = ld_f32;
  ep.out_bf16 = (__nv_bfloat16*)out_bf16;
  ep.ld_bf16 = ld_bf16;
  ep.out_q = out_q;
  ep.aux_rdiv = 1;
  OUU_CHECK_ARG(err_dev != nullptr, "err_dev is required");
  return ouu_gemm_bf16((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, M, N, K, ep, err_dev,
                       (cudaStream_t)stream, 1);
}

extern "C" int ouu_kernel_gemm_tuned_shapes(void) { return ouu_gemm_tuned_count(); }
