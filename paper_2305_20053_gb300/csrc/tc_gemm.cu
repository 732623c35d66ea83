// tcgen05 + TMA BF16 GEMM with fused epilogues (see tc_gemm.cuh): a persistent kernel, one CTA
// per SM, each taking (row tile, column tile, K slice) units in turn; two tensor-memory
// accumulators, so that the epilogue of one unit (read straight from tensor memory into
// registers) overlaps the MMAs of the next (warp roles at k_gemm_bf16).
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

// Pipeline depth: as many 64-wide K stages as fit in about 200 KB of shared memory (the
// epilogue reads the accumulator from tensor memory, so the ring holds nothing else).
template <int BN>
struct GemmStages {
  static constexpr int per = GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2;
  static constexpr int value = (200 * 1024 / per) > 8 ? 8 : (200 * 1024 / per);
};

// Tensor-memory columns of one accumulator buffer (a power of two >= BN); two buffers.
template <int BN>
struct GemmAcc {
  static constexpr uint32_t cols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

// Named barrier of the eight epilogue warps (warps 4..11).
static __device__ __forceinline__ void gemm_epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Row-major stores of a warp's 16-column chunk (32 rows, one per lane, rows r0 + lane)
// through the warp's shared tile (32 rows x 20 floats): after the transpose each store
// instruction covers 8 rows x 16 consecutive columns, full 64-byte (FP32) or 32-byte (BF16)
// segments, instead of 32 rows x one lane's part.  Warp-collective: every lane calls it;
// rows >= M and columns >= c0 + nv are not written.  vec: 16-byte FP32 / 8-byte BF16 stores
// are aligned (base and leading dimension).
#define GEMM_TROW 20
static __device__ __forceinline__ void store_rows_f32(float* tile, float* out, int ld, int r0, int M, int c0, int nv,
                                                      const float* v, bool vec, bool accumulate) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 16; k += 4)
    *reinterpret_cast<float4*>(tile + lane * GEMM_TROW + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
  __syncwarp();
  const int q = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = 8 * i + (lane >> 2), row = r0 + rr;
    const float4 w = *reinterpret_cast<const float4*>(tile + rr * GEMM_TROW + 4 * q);
    if (row < M) {
      float* p = out + (size_t)row * ld + c0 + 4 * q;
      if (vec && 4 * q + 3 < nv) {
        float4 x = w;
        if (accumulate) {
          const float4 o = *reinterpret_cast<const float4*>(p);
          x.x += o.x, x.y += o.y, x.z += o.z, x.w += o.w;
        }
        *reinterpret_cast<float4*>(p) = x;
      } else {
        const float e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < nv) p[j] = accumulate ? p[j] + e[j] : e[j];
      }
    }
  }
  __syncwarp();
}

static __device__ __forceinline__ void store_rows_bf16(float* tile, __nv_bfloat16* out, int ld, int r0, int M, int c0,
                                                       int nv, const float* v, bool vec) {
  const int lane = threadIdx.x & 31;
  uint32_t* t32 = reinterpret_cast<uint32_t*>(tile);
#pragma unroll
  for (int k = 0; k < 16; k += 2) {
    const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[k], v[k + 1]);
    t32[lane * GEMM_TROW + k / 2] = *reinterpret_cast<const uint32_t*>(&p2);
  }
  __syncwarp();
  const int q = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = 8 * i + (lane >> 2), row = r0 + rr;
    const uint2 w = *reinterpret_cast<const uint2*>(t32 + rr * GEMM_TROW + 2 * q);
    if (row < M) {
      __nv_bfloat16* p = out + (size_t)row * ld + c0 + 4 * q;
      if (vec && 4 * q + 3 < nv) {
        *reinterpret_cast<uint2*>(p) = w;
      } else {
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&w);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < nv) p[j] = e[j];
      }
    }
  }
  __syncwarp();
}

// The fused epilogue of one 16-column chunk of one accumulator row (row r, columns c0 ..
// c0 + nv - 1), straight from the registers the tensor-memory load filled.  rowsum: the
// row's running quadratic (EPI_QOI).  MODE 7: split-K partial sums, added
// atomically (the bias only from the first K slice).
template <int MODE>
static __device__ __forceinline__ void epi_chunk(const float (&acc)[16], int r, int M, int c0, int nv, const EpiParams& ep,
                                                 bool first_slice, float& rowsum, float* tile) {
  // warp-collective (the row stores go through the warp's shared tile): every lane of the warp
  // calls it, lanes of rows >= M with their values ignored
  const int r0 = r - (int)(threadIdx.x & 31);
  const bool live_row = r < M;
  float y[16], o[16];
  float cb[16], cs[16], ca[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {   // per-column constants (the same addresses in every lane: broadcast loads)
    const bool in = j < nv;
    cb[j] = (in && ep.bias && first_slice) ? __ldg(ep.bias + c0 + j) : 0.f;
    cs[j] = (in && ep.col_scale) ? __ldg(ep.col_scale + c0 + j) : 1.f;
    ca[j] = (in && ep.col_add) ? __ldg(ep.col_add + c0 + j) : 0.f;
  }
  if (MODE == EPI_DGELU_SCALE || MODE == EPI_SCALE) {
    const float* ap = ep.aux + (size_t)((live_row ? r : r0) / ep.aux_rdiv) * ep.ld_aux + c0;
    float x[16];
    if (ep.vec && nv == 16) {
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(ap + j));
        x[j] = t.x, x[j + 1] = t.y, x[j + 2] = t.z, x[j + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = j < nv ? ap[j] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = y[j] = MODE == EPI_SCALE ? acc[j] * x[j] : acc[j] * gelu_d1f(x[j]);
  } else if (MODE == EPI_GELU_D) {
#pragma unroll
    for (int j = 0; j < 16; ++j) gelu_and_d1(acc[j] + cb[j], o[j], y[j]);   // one exp for both
  } else if (MODE == EPI_GELU) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      y[j] = acc[j] + cb[j];
      o[j] = gelu_f(y[j]);
    }
  } else if (MODE == EPI_QOI) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      y[j] = (acc[j] + cb[j]) * cs[j];
      const float v = j < nv ? y[j] + ca[j] : 0.f;
      o[j] = v * cs[j];
      if (live_row) rowsum = fmaf(v, v, rowsum);
    }
  } else {   // EPI_LINEAR and the split-K partial sums
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = y[j] = (ep.alpha * acc[j] + cb[j]) * cs[j];
  }
  if (MODE == 7) {
    if (!live_row) return;
    float* of = ep.out_f32 + (size_t)r * ep.ld_f32 + c0;
    if (ep.vec && nv == 16) {
#pragma unroll
      for (int j = 0; j < 16; j += 4) atomicAdd(reinterpret_cast<float4*>(of + j), make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nv) atomicAdd(of + j, y[j]);
    }
    return;
  }
  if (ep.out_f32) store_rows_f32(tile, ep.out_f32, ep.ld_f32, r0, M, c0, nv, y, ep.vec != 0, ep.accumulate != 0);
  if (ep.out_bf16) store_rows_bf16(tile, ep.out_bf16, ep.ld_bf16, r0, M, c0, nv, o, ep.vec != 0);
  if (ep.out2_bf16) store_rows_bf16(tile, ep.out2_bf16, ep.ld2, r0, M, c0, nv, acc, ep.vec != 0);
  if (ep.out_t_bf16 && live_row)   // transposed: consecutive lanes (rows) write consecutive addresses of a column
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < nv) ep.out_t_bf16[(size_t)(c0 + j) * ep.ld_t + r] = __float2bfloat16(o[j]);
}

// Persistent GEMM: CTA b takes units b, b + gridDim.x, ... of the (row tile, column tile,
// K slice) grid, column tiles fastest.  Warp roles:
//   warp 0 (one lane): TMA producer; one ring of 64-wide K stages runs across the CTA's units
//   warp 1 (one lane): tcgen05.mma issuer into one of two tensor-memory accumulators
//                      (alternating per unit); warp 1 also allocates / frees the tensor memory
//   warps 4..11      : epilogue, straight from tensor memory: warp w reads the accumulator rows
//                      (TMEM lanes) 32 (w % 4) .. + 31, warps 4..7 the even and warps 8..11
//                      the odd 16-column chunks; a unit's epilogue overlaps the next unit's MMAs
// Every mbarrier wait is bounded (about 2 s of SM clock); on a timeout the CTA stops issuing,
// drains its own TMA copies and MMAs (bounded), frees its tensor memory and raises *err.
template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                int splits, EpiParams ep, int* err) {
  constexpr int STAGES = GemmStages<BN>::value;
  constexpr uint32_t A_BYTES = GEMM_BM * GEMM_BK * 2;
  constexpr uint32_t B_BYTES = BN * GEMM_BK * 2;
  constexpr uint32_t ACC = GemmAcc<BN>::cols;
  constexpr int NCH = (BN + 15) / 16;
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
  static_assert(B_BYTES % 1024 == 0, "stage buffers must stay 1024-byte aligned");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sa = smem;
  uint8_t* sb = smem + STAGES * A_BYTES;
  uint64_t* full = (uint64_t*)(sb + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;    // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;     // [2] epilogue -> MMA
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tslot = (uint32_t*)(mma_done + 1);
  __shared__ volatile int s_fail;
  __shared__ float s_part[2][GEMM_BM];    // row-sum halves (EPI_QOI)
  __shared__ float s_colsum[BN];          // column sums (EPI_DECODE)
  __shared__ __align__(16) float s_tile[8][32 * GEMM_TROW];   // per epilogue warp: the row-store transpose

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (M + GEMM_BM - 1) / GEMM_BM, nt = (N + BN - 1) / BN;
  const int units = mt * nt * splits;
  const int KB_all = (K + GEMM_BK - 1) / GEMM_BK;
  const int per = (KB_all + splits - 1) / splits;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 8);   // lane 0 of each epilogue warp
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, 2 * ACC);
  if (warp == 0 && lane < 2) tmap_prefetch(lane == 0 ? &ta : &tb);
  pdl_wait();   // everything below reads or writes what earlier kernels produce or consume
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int ntile = u % nt, rest = u / nt, mtile = rest % mt, z = rest / mt;
        const int kb_lo = z * per, KB = max(0, min(KB_all, kb_lo + per) - kb_lo);
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int st = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty[st], ((uint32_t)(g / STAGES) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], A_BYTES + B_BYTES);
          tma_load_2d(sa + st * A_BYTES, &ta, (kb_lo + kb) * GEMM_BK, mtile * GEMM_BM, &full[st]);
          tma_load_2d(sb + st * B_BYTES, &tb, (kb_lo + kb) * GEMM_BK, ntile * BN, &full[st]);
        }
      }
      if (!ok) s_fail = 1;
      // drain: the last copy issued into every stage has landed before exit
      for (int f = max(0, g - STAGES); f < g; ++f)
        if (!mbar_wait(&full[f % STAGES], (uint32_t)(f / STAGES) & 1u)) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(GEMM_BM >> 4) << 24);
      int g = 0, j = 0;
      bool ok = true, any = false;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++j) {
        const int z = u / (nt * mt);
        const int kb_lo = z * per, KB = max(0, min(KB_all, kb_lo + per) - kb_lo);
        const int b = j & 1;
        if (j >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((j >> 1) - 1) & 1u)) {   // the epilogue read buffer b
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)b * ACC;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int st = g % STAGES;
          if (!mbar_wait(&full[st], (uint32_t)(g / STAGES) & 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sa + st * A_BYTES), b0 = smem_u32(sb + st * B_BYTES);
#pragma unroll
          for (int k = 0; k < GEMM_BK / 16; ++k)
            tc_mma(d, smem_desc_sw128(a0 + k * 32), smem_desc_sw128(b0 + k * 32), idesc, (kb | k) != 0);
          tc_commit(&empty[st]);
          any = true;
        }
        if (ok) tc_commit(&acc_full[b]);   // completes once the unit's MMAs have finished
      }
      if (!ok) s_fail = 1;
      if (any) {
        tc_commit(mma_done);
        if (!mbar_wait(mma_done, 0)) s_fail = 1;
      }
    }
  } else if (warp >= 4) {
    const int q = warp & 3, half = (warp - 4) >> 2;
    int j = 0;
    bool live = true;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
      const int ntile = u % nt, rest = u / nt, mtile = rest % mt, z = rest / mt;
      const int kb_lo = z * per, KB = max(0, min(KB_all, kb_lo + per) - kb_lo);
      const int b = j & 1;
      // after a timed-out wait a warp stops reading and writing but keeps its place in the loop:
      // the named barriers below need all eight epilogue warps every time
      if (live) live = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)(j >> 1) & 1u) ? 1 : 0) != 0;
      if (!live && lane == 0) s_fail = 1;
      tc_fence_after();
      const int r = mtile * GEMM_BM + q * 32 + lane, n0 = ntile * BN;
      float rowsum = 0.f;
      if (ep.mode == EPI_DECODE) {   // rows are grid nodes, columns samples: out[c][r], column sums
        for (int i = threadIdx.x - 128; i < BN; i += 256) s_colsum[i] = 0.f;
        gemm_epi_sync();
        const float radd = (r < M && live) ? __ldg(ep.col_add + r) : 0.f;
        const float rref = (r < M && live) ? __ldg(ep.col_ref + r) : 0.f;
        for (int k = half; k < NCH && live; k += 2) {
          const int c0 = n0 + 16 * k;
          if (c0 >= N) break;   // the same in every lane
          uint32_t v[16];
          tmem_ld16(tmem + (uint32_t)b * ACC + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * k), v);
          const int nv = min(16, N - c0);
          float sq[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float val = __uint_as_float(v[i]) + radd;
            if (r < M && i < nv) ep.out_f32[(size_t)(c0 + i) * ep.ld_f32 + r] = val;   // coalesced over lanes
            const float dd = (r < M && i < nv) ? val - rref : 0.f;
            sq[i] = dd * dd;
          }
          // the 16 column sums over the warp's 32 rows by recursive halving: after the steps
          // over lane bits 4..1 lane L holds the sum over 16 lanes of column
          // 8 b4 + 4 b3 + 2 b2 + b1 (b_i the bits of L); the last step adds the lane pair
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const bool up = lane & 16;
            const float send = up ? sq[i] : sq[i + 8];
            const float got = __shfl_xor_sync(0xffffffffu, send, 16);
            sq[i] = (up ? sq[i + 8] : sq[i]) + got;
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool up = lane & 8;
            const float send = up ? sq[i] : sq[i + 4];
            const float got = __shfl_xor_sync(0xffffffffu, send, 8);
            sq[i] = (up ? sq[i + 4] : sq[i]) + got;
          }
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const bool up = lane & 4;
            const float send = up ? sq[i] : sq[i + 2];
            const float got = __shfl_xor_sync(0xffffffffu, send, 4);
            sq[i] = (up ? sq[i + 2] : sq[i]) + got;
          }
          {
            const bool up = lane & 2;
            const float send = up ? sq[0] : sq[1];
            const float got = __shfl_xor_sync(0xffffffffu, send, 2);
            sq[0] = (up ? sq[1] : sq[0]) + got;
          }
          sq[0] += __shfl_xor_sync(0xffffffffu, sq[0], 1);
          const int col = 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
          if (!(lane & 1) && col < nv) atomicAdd(&s_colsum[16 * k + col], sq[0]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
        gemm_epi_sync();
        for (int i = threadIdx.x - 128; i < BN; i += 256)
          if (n0 + i < N && live) atomicAdd(&ep.out_q[n0 + i], ep.qconst * (double)s_colsum[i]);
        gemm_epi_sync();   // read before the next unit clears it
        continue;
      }
      if (KB > 0 && live) {
        for (int k = half; k < NCH; k += 2) {
          const int c0 = n0 + 16 * k;
          if (c0 >= N) break;   // the same in every lane
          uint32_t v[16];
          tmem_ld16(tmem + (uint32_t)b * ACC + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * k), v);
          float acc[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] = __uint_as_float(v[i]);
          {   // every lane (the row stores are warp-collective); rows >= M are not written
            const int nv = min(16, N - c0);
            float* tile = s_tile[warp - 4];
            if (splits > 1)
              epi_chunk<7>(acc, r, M, c0, nv, ep, z == 0, rowsum, tile);
            else if (ep.mode == EPI_LINEAR)
              epi_chunk<EPI_LINEAR>(acc, r, M, c0, nv, ep, true, rowsum, tile);
            else if (ep.mode == EPI_GELU)
              epi_chunk<EPI_GELU>(acc, r, M, c0, nv, ep, true, rowsum, tile);
            else if (ep.mode == EPI_GELU_D)
              epi_chunk<EPI_GELU_D>(acc, r, M, c0, nv, ep, true, rowsum, tile);
            else if (ep.mode == EPI_SCALE)
              epi_chunk<EPI_SCALE>(acc, r, M, c0, nv, ep, true, rowsum, tile);
            else if (ep.mode == EPI_QOI)
              epi_chunk<EPI_QOI>(acc, r, M, c0, nv, ep, true, rowsum, tile);
            else
              epi_chunk<EPI_DGELU_SCALE>(acc, r, M, c0, nv, ep, true, rowsum, tile);
          }
        }
      }
      // the accumulator buffer is read: the MMA issuer may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      if (ep.mode == EPI_QOI) {   // the two halves of each row's quadratic
        s_part[half][q * 32 + lane] = rowsum;
        gemm_epi_sync();
        if (half == 0 && r < M && live)
          ep.out_q[r] = ep.qconst + 0.5 * ((double)s_part[0][q * 32 + lane] + (double)s_part[1][q * 32 + lane]);
        gemm_epi_sync();   // read before the next unit overwrites it
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * ACC);
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
  constexpr int STAGES = GemmStages<BN>::value;
  CUtensorMap tb;
  if (!ouu_tmap_bf16(&tb, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, BN)) {
    ouu_set_error("tensor map for GEMM operand B failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  const size_t smem = 1024 + (size_t)STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) + (2 * STAGES + 5) * 8 + 16;
  OUU_CUDA_TRY(ouu_smem_limit((const void*)k_gemm_bf16<BN>, smem));
  static const int sms = [] {   // initialised once, thread-safe (one device per process)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  const long units = (long)((N + BN - 1) / BN) * ((M + GEMM_BM - 1) / GEMM_BM) * splits;
  const int grid = (int)std::min<long>(units, sms);
  OUU_CUDA_TRY(launch_pdl(k_gemm_bf16<BN>, dim3(grid), dim3(GEMM_THREADS), smem, s, ta, tb, M, N, K, splits, ep, err));
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
