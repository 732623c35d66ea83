// tcgen05 + TMA BF16 GEMM with fused epilogues (see tc_gemm.cuh).
//
// CTA = 6 warps, one 128 x BN output tile:
//   warp 0 (one lane): TMA producer, 4-stage ring of 64-wide K blocks (SWIZZLE_128B)
//   warp 1 (one lane): tcgen05.mma issuer (kind::f16, BF16 x BF16 -> FP32 in TMEM);
//                      warp 1 also allocates / frees the tensor memory
//   warps 2..5       : epilogue, one accumulator row (TMEM lane) per thread
// Every mbarrier wait is bounded (about 2 s of SM clock); on a timeout the CTA
// drains its own TMA copies (bounded), frees its tensor memory and raises *err.
#include <math.h>

#include <algorithm>

#include "tc_gemm.cuh"

#define GEMM_BM 128
#define GEMM_BK 64
#define GEMM_THREADS 192
#define GEMM_WAIT_CYCLES (1ll << 32)

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Wait until the phase with the given parity has completed; false after the limit.
// The suspend-time hint lets the waiting thread sleep until the phase completes instead
// of spinning (spinning warps would take issue slots from the MMA-issuing thread).
static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(1000000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > GEMM_WAIT_CYCLES) return false;
  }
}

static __device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

static __device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

static __device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

static __device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

static __device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                              uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accum)
      : "memory");
}

static __device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle layout
// (8 rows x 128 B atoms, atoms 1024 B apart), as written by a SWIZZLE_128B TMA box.
static __device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                     // leading-dimension byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride-dimension byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
  return d;
}

static __device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
static __device__ __forceinline__ float gelu_d1f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

// Pipeline depth: four stages, five for the widest tiles (long-K projections, one CTA per SM).
template <int BN>
struct GemmStages {
  static constexpr int value = BN > 128 ? 5 : 4;
};

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
  } else {
    // Epilogue A (warps 2..5): TMEM -> shared staging tile, one accumulator row per thread
    // (warp w may read TMEM lanes 32 (w % 4) .. +31).  The pipeline buffers are free once
    // every MMA has completed.
    const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull, 0) ? 1 : 0);
    tc_fence_after();
    const int q = warp & 3;
    float* stage = (float*)smem;
    constexpr int SROW = BN + 1;
    if (!ok && lane == 0) s_fail = 1;
    if (ok && KB > 0) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) stage[(q * 32 + lane) * SROW + c0 + j] = __uint_as_float(v[j]);
      }
    } else if (ok) {   // empty K range (split-K remainder): contributes zero
      for (int c = 0; c < BN; ++c) stage[(q * 32 + lane) * SROW + c] = 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();   // staging tile complete; producer and MMA roles are done
  {
    // Epilogue B (all 6 warps): lanes over columns, rows dealt to warps, four rows per step
    // so that their loads are in flight together; row-major outputs are written coalesced.
    constexpr int SROW = BN + 1;
    constexpr int NC = (BN + 31) / 32;
    constexpr int NW = GEMM_THREADS / 32;
    float* stage = (float*)smem;
    const bool run = !s_fail;
    const float* __restrict__ bias = ep.bias;
    const float* __restrict__ cscale = ep.col_scale;
    const float* __restrict__ aux = ep.aux;
    float* __restrict__ of = ep.out_f32;
    __nv_bfloat16* __restrict__ ob16 = ep.out_bf16;
    __nv_bfloat16* __restrict__ o2 = ep.out2_bf16;
    const int mode = ep.mode;
    float bcol[NC], scol[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const int cc = lane + 32 * k, c = n0 + cc;
      const bool in = cc < BN && c < N;
      bcol[k] = (in && bias && (!splitk || blockIdx.z == 0)) ? bias[c] : 0.f;
      scol[k] = (in && cscale) ? cscale[c] : 1.f;
    }
    if (run) {
      for (int t0 = warp; t0 < GEMM_BM; t0 += 4 * NW) {
        float accv[4][NC], auxv[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int tr = t0 + u * NW, r = m0 + tr;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int cc = lane + 32 * k, c = n0 + cc;
            const bool in = tr < GEMM_BM && cc < BN && c < N && r < M;
            accv[u][k] = in ? stage[tr * SROW + cc] : 0.f;
            auxv[u][k] = (in && mode == EPI_DGELU_SCALE) ? aux[(size_t)(r / ep.aux_rdiv) * ep.ld_aux + c] : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int tr = t0 + u * NW, r = m0 + tr;
          if (tr >= GEMM_BM || r >= M) break;
          float* orow = of ? of + (size_t)r * ep.ld_f32 : nullptr;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int cc = lane + 32 * k, c = n0 + cc;
            if (cc >= BN || c >= N) break;
            const float acc = accv[u][k];
            float y, obv;
            if (splitk) {
              atomicAdd(orow + c, ep.alpha * acc + bcol[k]);
              continue;
            }
            if (mode == EPI_LINEAR) {
              y = (ep.alpha * acc + bcol[k]) * scol[k];
              obv = y;
            } else if (mode == EPI_GELU) {
              y = acc + bcol[k];
              obv = gelu_f(y);
            } else {
              y = acc * gelu_d1f(auxv[u][k]);
              obv = y;
            }
            if (orow) orow[c] = ep.accumulate ? orow[c] + y : y;
            if (ob16) ob16[(size_t)r * ep.ld_bf16 + c] = __float2bfloat16(obv);
            if (o2) o2[(size_t)r * ep.ld2 + c] = __float2bfloat16(acc);
            if (ep.out_t_bf16) stage[tr * SROW + cc] = obv;
          }
        }
      }
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
  static_assert((size_t)GEMM_STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) >= (size_t)GEMM_BM * (BN + 1) * 4,
                "the pipeline buffers must hold the epilogue staging tile");
  CUtensorMap tb;
  if (!ouu_tmap_bf16(&tb, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, BN)) {
    ouu_set_error("tensor map for GEMM operand B failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  const size_t smem = 1024 + (size_t)GEMM_STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) +
                      (2 * GEMM_STAGES + 1) * 8 + 16;
  static bool attr_set = false;   // one device per process is the supported set-up
  if (!attr_set) {
    cudaFuncSetAttribute((const void*)k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  dim3 grid((N + BN - 1) / BN, (M + GEMM_BM - 1) / GEMM_BM, splits);
  k_gemm_bf16<BN><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, M, N, K, ep, err);
  OUU_CUDA_TRY(cudaGetLastError());
  return OUU_OK;
}

ouu_status ouu_gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                         const EpiParams& ep, int* err, cudaStream_t s, int splits) {
  OUU_CHECK_ARG(M >= 1 && N >= 1 && K >= 1, "GEMM sizes must be positive");
  OUU_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0, "GEMM operands must be 16-byte aligned");
  OUU_CHECK_ARG(lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K, "GEMM leading dimensions: multiple of 8, >= K");
  OUU_CHECK_ARG(ep.mode != EPI_DGELU_SCALE || (ep.aux && ep.aux_rdiv >= 1), "EPI_DGELU_SCALE needs aux");
  OUU_CHECK_ARG(splits >= 1 && splits <= 64, "split-K factor in [1, 64]");
  OUU_CHECK_ARG(splits == 1 || (ep.mode == EPI_LINEAR && ep.out_f32 && !ep.out_bf16 && !ep.out_t_bf16 &&
                                !ep.out2_bf16 && !ep.col_scale && !ep.accumulate),
                "split-K supports one FP32 output of EPI_LINEAR, accumulated into a zeroed buffer");
  CUtensorMap ta;
  if (!ouu_tmap_bf16(&ta, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, GEMM_BM)) {
    ouu_set_error("tensor map for GEMM operand A failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  // N tile with the least padding (ties: the wider tile).
  static const int cands[] = {256, 208, 128, 112, 80, 64};
  int best = 64;
  long best_pad = 1L << 40;
  for (int bn : cands) {
    const long pad = (long)((N + bn - 1) / bn) * bn - N;
    if (pad < best_pad) {
      best_pad = pad;
      best = bn;
    }
  }
  switch (best) {
    case 256: return launch_bn<256>(ta, B, ldb, M, N, K, ep, err, s, splits);
    case 208: return launch_bn<208>(ta, B, ldb, M, N, K, ep, err, s, splits);
    case 128: return launch_bn<128>(ta, B, ldb, M, N, K, ep, err, s, splits);
    case 112: return launch_bn<112>(ta, B, ldb, M, N, K, ep, err, s, splits);
    case 80: return launch_bn<80>(ta, B, ldb, M, N, K, ep, err, s, splits);
    default: return launch_bn<64>(ta, B, ldb, M, N, K, ep, err, s, splits);
  }
}

// Kernel-level entry used by the GEMM numerics test (declared in include/ouu_kernels.h).
extern "C" ouu_status ouu_kernel_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                           int mode, float alpha, const float* bias, const float* aux, int ld_aux,
                                           int aux_rdiv, float* out_f32, int ld_f32, int accumulate, void* out_bf16,
                                           int ld_bf16, void* out_t_bf16, int ld_t, void* out2_bf16, int ld2,
                                           int* err_dev, void* stream) {
  EpiParams ep;
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
