// Fused KL projection (Sec. 3.3, the input reduction of the reduced-basis network):
//   xi[s][c] = bias[c] + sum_k bf16(m[s][k]) * W[c][k],   s < N, c < r_m,
// reading the FP64 fields once.  One persistent CTA per SM over the units (128-sample tile,
// 64-wide K block).  The units are claimed at run time, one at a time, from a counter per
// tile: a CTA keeps claiming K blocks of its tile (accumulating them in one TMEM accumulator,
// flushed once per tile visit) and, when the tile runs out, moves to the tile with the most K
// blocks left; the CTAs start spread evenly over the tiles.  So every SM streams for as long
// as there is work, whatever its share of DRAM bandwidth, and all finish within about one
// unit of each other.  Per CTA:
//   warp 16      : field producer.  Claims the units (one ahead, to know where a tile visit
//                  ends), publishes each in a shared ring, and TMA-loads the FP64 slice
//                  m[tile rows][k0, k0+64).  With n^2 odd the row stride n^2 * 8 bytes is not a
//                  multiple of 16, which a tensor map needs; the fields are then read as rows
//                  of sample PAIRS (stride 2 n^2 * 8 bytes), even samples from x = k0 and odd
//                  samples from x = n^2 + k0 - 1 (one element early, so that x stays 16-byte
//                  aligned), 66 elements each: two copies per K block.  A last unpaired sample
//                  (N odd), and every sample when the base is not 16-byte aligned, is read with
//                  plain loads.
//   warps 0..15  : converters.  Each copies its 8 rows of the FP64 stage into registers and
//                  releases the stage at once (the next field copy then overlaps the
//                  arithmetic), then converts FP64 -> BF16 (round to FP32, then to BF16,
//                  both to nearest even; the first step in integer arithmetic, as the FP64
//                  pipe is narrow) straight into the swizzled K-major A tile that
//                  tcgen05.mma reads.  Warp 0 also loads the unit's BF16 basis block
//                  W[0, BN) x [k0, k0 + 64) (128-byte swizzle) once its stage is free.
//   warp 17      : tcgen05.mma issuer (M = 128, N = BN, K = 16 per instruction) into one of
//                  two TMEM accumulators (one per tile visit); allocates and frees the tensor
//                  memory; hands each visit's (tile, holds K block 0, final) to the epilogue.
//   warps 18..25 : epilogue, two groups of four (one per TMEM accumulator, so visits alternate
//                  between them and the final visit's flush need not wait for the previous
//                  visit's).  TMEM -> registers, + bias on the visit that holds K block 0 of
//                  its tile, 16-byte atomic adds into xi (zeroed beforehand); the CTA's final
//                  visit (when every CTA flushes at once) goes through the idle FP64 stages
//                  and TMA bulk reductions of whole rows instead.
// Every mbarrier wait is bounded; on a timeout the CTA publishes the end of its units, stops,
// drains its own copies and raises *err.
#include <cuda_bf16.h>

#include "dino.cuh"
#include "ouu_kernels.h"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#define KLP_CONV_WARPS 16
#define KLP_PROD_WARP 16
#define KLP_MMA_WARP 17
#define KLP_EPI_WARP0 18
#define KLP_EPI_GROUPS 2
#define KLP_THREADS ((KLP_EPI_WARP0 + 4 * KLP_EPI_GROUPS) * 32)
#define KLP_RING 16                          // published units (the MMA lags the producer by < 8)
#define KLP_ROWS_PER_WARP (128 / KLP_CONV_WARPS)
#define KLP_ROW_BYTES 528                    // pair mode: 66 doubles per sample row
#define KLP_F64_STAGE (128 * KLP_ROW_BYTES)
#define KLP_HALF (64 * KLP_ROW_BYTES)           // pair mode: even samples, then odd samples
#define KLP_A_STAGE (128 * 64 * 2)

struct KlpArgs {
  const double* m;
  int N, nn, KBt, BN, rm;
  int pair;        // 1: fields read as sample pairs (n^2 odd); 0: as rows (n^2 even)
  int n_tma;       // samples [0, n_tma) come by TMA, the rest (at most one) by plain loads
  int T;           // 128-sample tiles
  int bulk;        // 1: the final visit's rows are added by TMA bulk reductions (r_m % 4 == 0, xi 16-byte aligned)
  int* ctr;        // [T] next unclaimed K block of each tile, [T] CTAs finished; zero at launch and
                   // left zero by the last CTA
  const float* bias;
  float* xi;
  int* err;
  const float* zsrc;   // nz floats copied to zdst by block 0 (a rider for the work that follows)
  float* zdst;
  int nz;
};

// FP64 -> FP32, rounding to nearest even, in integer arithmetic on the two halves of the
// double (GB300's FP64 pipe is narrow).  Normal FP32 range on the fast path; otherwise
// a signed zero below it, an infinity above it, NaN kept.  The FP32 -> BF16 step (also to
// nearest even) is one packed hardware conversion of two values.
static __device__ __forceinline__ float f64_to_f32_slow(uint32_t hi, uint32_t lo) {
  const uint32_t e = (hi >> 20) & 0x7FFu, sign = hi & 0x80000000u;
  if (e == 0x7FFu) return __uint_as_float(sign | (((hi & 0xFFFFFu) | lo) ? 0x7FC00000u : 0x7F800000u));
  if (e > 1023u + 127u) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign);   // below the normal FP32 range
}

// (biased FP64 exponent - 897) << 20, wrapping below 897: under KLP_EXP_SPAN exactly when x
// rounds into FP32's normal range by the fast path below (exponent in [897, 1150]).  The
// maximum over many values tests them all with one comparison.
#define KLP_EXP_SPAN (254u << 20)
static __device__ __forceinline__ uint32_t f32_exp_offset(double x) {
  return ((uint32_t)__double2hiint(x) & 0x7FF00000u) - (897u << 20);
}

// Lane l's two values of one row of the FP64 stage: columns 2l and 2l + 1 of the K block.
// Row mode: rows of 512 bytes.  Pair mode: even samples in the first half, odd samples in
// the second, rows of 528 bytes; an odd sample's row starts one element early, so its
// 16-byte pair holds columns (2l - 1, 2l) and column 2l + 1 comes from the next lane (lane
// 31 reads column 63 itself, a broadcast load).
static __device__ __forceinline__ void stage_row(const uint8_t* fst, int pair, int rr, int lane, double& x0,
                                                 double& x1) {
  if (!pair) {
    const double2 v = reinterpret_cast<const double2*>(fst + rr * 512)[lane];
    x0 = v.x;
    x1 = v.y;
  } else if (!(rr & 1)) {
    const double2 v = reinterpret_cast<const double2*>(fst + (rr >> 1) * KLP_ROW_BYTES)[lane];
    x0 = v.x;
    x1 = v.y;
  } else {
    const uint8_t* row = fst + KLP_HALF + (rr >> 1) * KLP_ROW_BYTES;
    const double2 v = reinterpret_cast<const double2*>(row)[lane];
    const double c63 = reinterpret_cast<const double*>(row)[64];
    const double nx = __shfl_down_sync(0xffffffffu, v.x, 1);
    x0 = v.y;
    x1 = lane == 31 ? c63 : nx;
  }
}

// The fast path on its own: rounding the 64-bit pattern to nearest even at bit 29 carries
// through the mantissa into the exponent as it should; bits 23..31 of (bits >> 29) hold
// the low 9 exponent bits, and subtracting 896 mod 512 leaves the FP32 exponent.
static __device__ __forceinline__ float f64_to_f32_fast(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  b += 0x0FFFFFFFull + ((b >> 29) & 1ull);
  return __uint_as_float(((uint32_t)(b >> 29) - 0xC0000000u) | sign);
}

static __device__ __forceinline__ float f64_to_f32_rne(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e - 897u > 253u) return f64_to_f32_slow(hi, lo);   // e outside [897, 1150]
  // sign | (e - 896) << 23 | the top 23 mantissa bits
  uint32_t f = (hi & 0x80000000u) | ((((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29));
  // the remaining 29 bits: +1 exactly when they exceed half, or equal it with f odd
  f += ((lo & 0x1FFFFFFFu) + 0x0FFFFFFFu + (f & 1u)) >> 29;
  return __uint_as_float(f);
}

// A published unit: x = tile (< 0: no more units), y = K block | first << 16 | last << 17 |
// final << 18 (first / last unit of a tile visit; the last unit of the CTA).
__global__ void __launch_bounds__(KLP_THREADS, 1) k_kl_project(const __grid_constant__ CUtensorMap tw,
                                                                const __grid_constant__ CUtensorMap tm, KlpArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t B_BYTES = (uint32_t)a.BN * 128u;
  uint8_t* sA = smem;
  uint8_t* sB = sA + 2 * KLP_A_STAGE;
  uint8_t* sF = sB + 2 * B_BYTES;
  uint64_t* bars = (uint64_t*)(sF + 2 * KLP_F64_STAGE);
  uint64_t* f64_full = bars + 0;    // producer: unit published (and its field copies landed)
  uint64_t* f64_empty = bars + 2;   // converters: FP64 stage in registers
  uint64_t* b_full = bars + 4;      // converter warp 0: basis block landed
  uint64_t* a_full = bars + 6;      // converters: BF16 A tile written
  uint64_t* ab_empty = bars + 8;    // MMA: A and B stages consumed
  uint64_t* acc_full = bars + 10;   // MMA: accumulator complete
  uint64_t* acc_empty = bars + 12;  // epilogue: accumulator drained
  uint64_t* seg_full = bars + 14;   // MMA: tile-visit descriptor written
  uint64_t* mma_done = bars + 16;
  uint32_t* tslot = (uint32_t*)(bars + 17);
  __shared__ int2 s_unit[KLP_RING];
  __shared__ int2 s_seg[2];         // (tile, holds K block 0 | final visit << 1); tile < 0: no more visits
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nn = a.nn, KBt = a.KBt, N = a.N;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&f64_full[i], 1);
      mbar_init(&f64_empty[i], KLP_CONV_WARPS);
      mbar_init(&b_full[i], 1);
      mbar_init(&a_full[i], KLP_CONV_WARPS);
      mbar_init(&ab_empty[i], 1);
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
      mbar_init(&seg_full[i], 1);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == KLP_MMA_WARP) tmem_alloc(tslot, 512);
  if (warp == KLP_PROD_WARP && lane < 2) tmap_prefetch(lane == 0 ? &tm : &tw);
  pdl_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == KLP_PROD_WARP) {
    // ---------------------------------------------------------------- field producer
    int cur = (int)(((long long)blockIdx.x * a.T) / gridDim.x);   // the tile claimed from
    // The tile with the most K blocks left (the warp's lanes scan the counters; the lowest
    // index among equals); false when every tile is done.
    auto next_tile = [&]() -> bool {
      int best = 0x7FFFFFFF, left = 0;
      for (int t0 = 0; t0 < a.T; t0 += 32) {
        const int t = t0 + lane;
        const int l = t < a.T ? KBt - *(volatile int*)(a.ctr + t) : 0;
        if (l > left) {
          left = l;
          best = t;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int ol = __shfl_xor_sync(0xffffffffu, left, o), ob = __shfl_xor_sync(0xffffffffu, best, o);
        if (ol > left || (ol == left && ob < best)) {
          left = ol;
          best = ob;
        }
      }
      if (left <= 0) return false;
      cur = best;
      return true;
    };
    // A claimed K block kb of tile cur (kb from the counter, possibly past the end): true with
    // the unit if valid, else moves to another tile and claims there, synchronously.
    auto settle = [&](int kb, int& t_out, int& kb_out) -> bool {
      for (int tries = 0; tries < 4 * a.T + 8; ++tries) {
        if (kb < KBt) {
          t_out = cur;
          kb_out = kb;
          return true;
        }
        if (!next_tile()) return false;
        kb = 0;
        if (lane == 0) kb = atomicAdd(&a.ctr[cur], 1);
        kb = __shfl_sync(0xffffffffu, kb, 0);
      }
      return false;
    };
    // Claim pipeline: unit j (t_cur, kb_cur) and unit j + 1 (t_nxt, kb_nxt) resolved, the
    // counter increment for the one after in flight, so that its latency overlaps the wait
    // for a free stage.  The first claim takes two K blocks at once.
    int t_cur = 0, kb_cur = 0, t_nxt = -1, kb_nxt = 0, pend = 0, prev_t = -1, j = 0;
    bool have, have_nxt;
    {
      int k2 = 0;
      if (lane == 0) k2 = atomicAdd(&a.ctr[cur], 2);
      k2 = __shfl_sync(0xffffffffu, k2, 0);
      have = settle(k2, t_cur, kb_cur);
      if (have && t_cur == cur && k2 + 1 < KBt && kb_cur == k2) {
        t_nxt = cur;
        kb_nxt = k2 + 1;
        have_nxt = true;
      } else {
        int k1 = 0;
        if (have && lane == 0) k1 = atomicAdd(&a.ctr[cur], 1);
        k1 = __shfl_sync(0xffffffffu, k1, 0);
        have_nxt = have && settle(k1, t_nxt, kb_nxt);
      }
    }
    if (have_nxt && lane == 0) pend = atomicAdd(&a.ctr[cur], 1);
    bool ok = true;
    const uint32_t fbytes = a.pair ? 2u * KLP_HALF : 128u * 512u;
    for (;; ++j) {
      const int s = j & 1;
      if (j >= 2 && !__all_sync(0xffffffffu, mbar_wait(&f64_empty[s], (((uint32_t)j >> 1) & 1u) ^ 1u) ? 1 : 0))
        ok = false;
      const bool pub = have && ok;   // on a timeout the end is published instead
      if (lane == 0) {
        s_unit[j & (KLP_RING - 1)] =
            pub ? make_int2(t_cur, kb_cur | ((t_cur != prev_t) << 16) | ((!have_nxt || t_nxt != t_cur) << 17) |
                                       ((!have_nxt) << 18))
                : make_int2(-1, 0);
        uint8_t* dst = sF + s * KLP_F64_STAGE;
        if (!pub || a.n_tma == 0) {
          mbar_arrive(&f64_full[s]);   // the end, or plain loads only
        } else if (a.pair) {
          mbar_expect_tx(&f64_full[s], fbytes);
          tma_load_2d(dst, &tm, kb_cur * 64, t_cur * 64, &f64_full[s]);
          tma_load_2d(dst + KLP_HALF, &tm, nn + kb_cur * 64 - 1, t_cur * 64, &f64_full[s]);
        } else {
          mbar_expect_tx(&f64_full[s], fbytes);
          tma_load_2d(dst, &tm, kb_cur * 64, t_cur * 128, &f64_full[s]);
        }
      }
      if (!pub) break;
      prev_t = t_cur;
      t_cur = t_nxt;
      kb_cur = kb_nxt;
      have = have_nxt;
      if (have_nxt) {   // resolve the claim in flight, start the next
        have_nxt = settle(__shfl_sync(0xffffffffu, pend, 0), t_nxt, kb_nxt);
        if (have_nxt && lane == 0) pend = atomicAdd(&a.ctr[cur], 1);
      }
    }
    // drain: the copies of the last published units have landed before the CTA exits
    if (lane == 0) {
      if (!ok) s_fail = 1;
      for (int u = max(0, j - 1); u <= j; ++u)
        if (!mbar_wait(&f64_full[u & 1], ((uint32_t)u >> 1) & 1u)) s_fail = 1;
    }
  } else if (warp < KLP_CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    // Lane l owns columns 2l and 2l + 1 of the warp's 8 rows: one 16-byte shared load per
    // row, and its two BF16 values form one 32-bit word of the A tile.
    const int r0 = warp * KLP_ROWS_PER_WARP;
    for (int j = 0;; ++j) {
      const int s = j & 1;
      const uint32_t ph = (uint32_t)(j >> 1) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(&f64_full[s], ph) ? 1 : 0)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      const int2 e = s_unit[j & (KLP_RING - 1)];
      if (e.x < 0) {   // no more units: the MMA issuer learns it through a_full
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[s]);
        break;
      }
      const int t = e.x, k0 = (e.y & 0xFFFF) * 64;
      const uint8_t* fst = sF + s * KLP_F64_STAGE;
      const int rb = t * 128 + r0;   // the warp's first sample
      double x0[KLP_ROWS_PER_WARP], x1[KLP_ROWS_PER_WARP];
      if (rb + KLP_ROWS_PER_WARP <= a.n_tma) {
#pragma unroll
        for (int i = 0; i < KLP_ROWS_PER_WARP; ++i) stage_row(fst, a.pair, r0 + i, lane, x0[i], x1[i]);
      } else {   // the tile's end: rows by plain loads (r >= n_tma) or zero rows (r >= N)
#pragma unroll
        for (int i = 0; i < KLP_ROWS_PER_WARP; ++i) {
          const int r = rb + i, c = k0 + 2 * lane;
          x0[i] = 0.0;
          x1[i] = 0.0;
          if (r < a.n_tma) {
            stage_row(fst, a.pair, r0 + i, lane, x0[i], x1[i]);
          } else if (r < N) {
            const double* row = a.m + (size_t)r * nn;
            if (c < nn) x0[i] = row[c];
            if (c + 1 < nn) x1[i] = row[c + 1];
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&f64_empty[s]);   // the stage is in registers: refill it
      if (j >= 2 && !__all_sync(0xffffffffu, mbar_wait(&ab_empty[s], ph ^ 1u) ? 1 : 0)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      if (warp == 0 && lane == 0) {   // the unit's basis block into the freed stage
        mbar_expect_tx(&b_full[s], B_BYTES);
        tma_load_2d(sB + s * B_BYTES, &tw, k0, 0, &b_full[s]);
      }
      uint8_t* ast = sA + s * KLP_A_STAGE;
      // 128-byte swizzle: 16-byte chunk index XOR (row mod 8) within the 8-row atom;
      // r0 is a multiple of 8, so row r0 + i has (row mod 8) = i
      uint8_t* wp = ast + r0 * 128 + ((lane & 3) << 2);
      const uint32_t ch = (uint32_t)lane >> 2;
      uint32_t emax = 0;
#pragma unroll
      for (int i = 0; i < KLP_ROWS_PER_WARP; ++i) emax = max(emax, max(f32_exp_offset(x0[i]), f32_exp_offset(x1[i])));
      // the last K block (columns past n^2 zeroed) and values outside FP32's normal range
      // take the general rounding
      if (__all_sync(0xffffffffu, emax < KLP_EXP_SPAN) && k0 + 64 <= nn) {
#pragma unroll
        for (int i = 0; i < KLP_ROWS_PER_WARP; ++i) {
          const __nv_bfloat162 pk = __floats2bfloat162_rn(f64_to_f32_fast(x0[i]), f64_to_f32_fast(x1[i]));
          *(uint32_t*)(wp + i * 128 + ((ch ^ (uint32_t)i) << 4)) = *reinterpret_cast<const uint32_t*>(&pk);
        }
      } else {
        const int c = k0 + 2 * lane;
        const uint32_t keep = c + 1 < nn ? 0xFFFFFFFFu : (c < nn ? 0x0000FFFFu : 0u);
#pragma unroll
        for (int i = 0; i < KLP_ROWS_PER_WARP; ++i) {
          const __nv_bfloat162 pk = __floats2bfloat162_rn(f64_to_f32_rne(x0[i]), f64_to_f32_rne(x1[i]));
          *(uint32_t*)(wp + i * 128 + ((ch ^ (uint32_t)i) << 4)) = *reinterpret_cast<const uint32_t*>(&pk) & keep;
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full[s]);
    }
  } else if (warp == KLP_MMA_WARP) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.BN >> 3) << 17) | ((128u >> 4) << 24);
      int seg = 0, seg_t = -1, has0 = 0;
      bool ok = true, any = false;
      for (int j = 0;; ++j) {
        const int s = j & 1;
        const uint32_t ph = (uint32_t)(j >> 1) & 1u;
        if (!mbar_wait(&a_full[s], ph)) {
          ok = false;
          break;
        }
        const int2 e = s_unit[j & (KLP_RING - 1)];
        if (e.x < 0) break;
        const int kb = e.y & 0xFFFF;
        const bool first = (e.y >> 16) & 1, last = (e.y >> 17) & 1, fin = (e.y >> 18) & 1;
        const int acc = seg & 1;
        if (first) {
          if (seg >= 2 && !mbar_wait(&acc_empty[acc], (uint32_t)((seg >> 1) - 1) & 1u)) {
            ok = false;
            break;
          }
          seg_t = e.x;
          has0 = 0;
        }
        has0 |= kb == 0;
        if (!mbar_wait(&b_full[s], ph)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + s * KLP_A_STAGE), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          tc_mma(tmem + (uint32_t)acc * 256u, smem_desc_sw128(a0 + k * 32), smem_desc_sw128(b0 + k * 32), idesc,
                 (!first || k > 0) ? 1u : 0u);
        tc_commit(&ab_empty[s]);
        any = true;
        if (last) {
          tc_commit(&acc_full[acc]);
          s_seg[acc] = make_int2(seg_t, has0 | (fin ? 2 : 0));
          mbar_arrive(&seg_full[acc]);
          ++seg;
        }
      }
      if (!ok) s_fail = 1;
      // the end of the visits, in both slots (one per epilogue group), each once its group has
      // read the slot's last descriptor (visit k used slot k & 1; slot a holds (seg - a + 1) / 2)
      for (int sl = 0; sl < 2; ++sl) {
        const int acc = (seg + sl) & 1, na = (seg - acc + 1) / 2;
        if (na >= 1 && !mbar_wait(&acc_empty[acc], (uint32_t)(na - 1) & 1u)) s_fail = 1;
        s_seg[acc] = make_int2(-1, 0);
        mbar_arrive(&seg_full[acc]);
      }
      // every MMA issued above has completed before the tensor memory is freed
      if (any) {
        tc_commit(mma_done);
        if (!mbar_wait(mma_done, 0)) s_fail = 1;
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3, grp = (warp - KLP_EPI_WARP0) >> 2;
    if (blockIdx.x == 0)   // idle until the first tile visit completes
      for (int i = threadIdx.x - KLP_EPI_WARP0 * 32; i < a.nz; i += 4 * KLP_EPI_GROUPS * 32) a.zdst[i] = a.zsrc[i];
    for (int k = grp;; k += KLP_EPI_GROUPS) {   // this group's visits: accumulator grp
      const int acc = k & 1;
      const uint32_t ph = (uint32_t)(k >> 1) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(&seg_full[acc], ph) ? 1 : 0)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      const int2 d = s_seg[acc];
      if (d.x < 0) break;
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[acc], ph) ? 1 : 0)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      tc_fence_after();
      const int r = d.x * 128 + q * 32 + lane;
      float* orow = a.xi + (size_t)r * a.rm;
      // 16-byte vector atomics need every row start 16-byte aligned
      const bool vec4 = (a.rm & 3) == 0 && (reinterpret_cast<uintptr_t>(a.xi) & 15) == 0;
      if ((d.y & 2) && a.bulk) {
        // The CTA's final visit, when every CTA flushes at once: the rows go through the
        // (now idle) FP64 stages and are added into xi by the TMA engine, one bulk reduction
        // of r_m floats per row, in whole lines instead of 16-byte atomics.
        float* srow = reinterpret_cast<float*>(sF) + (size_t)(q * 32 + lane) * a.rm;
        for (int c0 = 0; c0 < a.BN; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * 256u + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const int c = c0 + i;
            if (c < a.rm) {   // r_m % 4 == 0
              float4 y = make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                                     __uint_as_float(v[i + 3]));
              if (d.y & 1) {
                y.x += a.bias[c];
                y.y += a.bias[c + 1];
                y.z += a.bias[c + 2];
                y.w += a.bias[c + 3];
              }
              *reinterpret_cast<float4*>(srow + c) = y;
            }
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          const int rw0 = d.x * 128 + q * 32;
          for (int i = 0; i < 32 && rw0 + i < N; ++i)
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(
                             a.xi + (size_t)(rw0 + i) * a.rm),
                         "r"(smem_u32(reinterpret_cast<float*>(sF) + (size_t)(q * 32 + i) * a.rm)), "r"(a.rm * 4)
                         : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // done before the CTA exits
        }
        __syncwarp();
      } else
      for (int c0 = 0; c0 < a.BN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * 256u + (uint32_t)c0, v);
        if (r < N) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const int c = c0 + i;
            if (c >= a.rm) break;
            float y[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
              y[jj] = __uint_as_float(v[i + jj]) + (((d.y & 1) && c + jj < a.rm) ? a.bias[c + jj] : 0.f);
            if (vec4) {
              atomicAdd(reinterpret_cast<float4*>(orow + c), make_float4(y[0], y[1], y[2], y[3]));
            } else {
              for (int jj = 0; jj < 4 && c + jj < a.rm; ++jj) atomicAdd(orow + c + jj, y[jj]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == KLP_MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0) {
    if (s_fail) atomicExch(a.err, 1);
    // the last CTA to finish (nobody claims any more) leaves the counters zero for the next launch
    if (atomicAdd(a.ctr + a.T, 1) == (int)gridDim.x - 1) {
      for (int t = 0; t <= a.T; ++t) *(volatile int*)(a.ctr + t) = 0;
    }
  }
}

// One launch over N <= OUU_KLP_MAX_TILES * 128 samples.
static ouu_status kl_project_launch(const double* m, int N, int nn, const CUtensorMap& tw, int BN, int rm,
                                    const float* bias, float* xi, int* err, int* ctr, int num_sms, cudaStream_t s,
                                    const float* zsrc, float* zdst, int nz) {
  // fields tensor map: sample rows (n^2 even) or sample pairs (n^2 odd)
  // A base that is not 16-byte aligned (a slice starting at an odd sample) cannot be a
  // tensor map's base: every row then goes by plain loads.
  const int pair = nn & 1;
  const int n_tma = ((uintptr_t)m & 15) ? 0 : (pair ? N / 2 * 2 : N);
  CUtensorMap tm;
  if (n_tma > 0) {
    const bool okm = pair ? ouu_tmap_2d(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, m, 2 * (uint64_t)nn, (uint64_t)(N / 2),
                                        16 * (uint64_t)nn, 66, 64, CU_TENSOR_MAP_SWIZZLE_NONE)
                          : ouu_tmap_2d(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, m, (uint64_t)nn, (uint64_t)N,
                                        8 * (uint64_t)nn, 64, 128, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!okm) {
      ouu_set_error("tensor map for the fields failed (alignment or driver entry point)");
      return OUU_ERR_INVALID_ARG;
    }
  } else {
    tm = tw;   // never read: every row goes by plain loads
  }
  KlpArgs a;
  a.pair = pair;
  a.n_tma = n_tma;
  a.m = m;
  a.N = N;
  a.nn = nn;
  a.KBt = (nn + 63) / 64;
  a.BN = BN;
  a.rm = rm;
  a.T = (N + 127) / 128;
  a.ctr = ctr;
  a.bulk = (rm % 4 == 0 && ((uintptr_t)xi & 15) == 0 && (size_t)128 * rm * 4 <= 2 * (size_t)KLP_F64_STAGE) ? 1 : 0;
  a.bias = bias;
  a.xi = xi;
  a.err = err;
  a.zsrc = zsrc;
  a.zdst = zdst;
  a.nz = zsrc && zdst ? nz : 0;
  const size_t smem = 1024 + 2 * KLP_A_STAGE + 2 * (size_t)BN * 128 + 2 * KLP_F64_STAGE + 17 * 8 + 16;
  OUU_CUDA_TRY(ouu_smem_limit((const void*)k_kl_project, smem));
  const long long U = (long long)a.T * a.KBt;
  const int grid = (int)std::min<long long>(U, (long long)std::max(1, num_sms));
  OUU_CUDA_TRY(cudaMemsetAsync(xi, 0, (size_t)N * rm * 4, s));
  OUU_CUDA_TRY(launch_pdl(k_kl_project, dim3(grid), dim3(KLP_THREADS), smem, s, tw, tm, a));
  return OUU_OK;
}

ouu_status ouu_kl_project(const double* m, int N, int nn, const __nv_bfloat16* W, int ldw, int rm, const float* bias,
                          float* xi, int* err, int* ctr, int num_sms, cudaStream_t s, const float* zsrc, float* zdst,
                          int nz) {
  OUU_CHECK_ARG(m && W && bias && xi && err && ctr, "null argument");
  OUU_CHECK_ARG(N >= 1 && nn >= 1 && rm >= 1 && rm <= 240, "KL projection sizes: N, n^2 >= 1, 1 <= r_m <= 240");
  OUU_CHECK_ARG(((uintptr_t)m & 7) == 0, "fields must be 8-byte aligned");
  OUU_CHECK_ARG(((uintptr_t)xi & 3) == 0, "xi must be 4-byte aligned");
  const int BN = (rm + 15) / 16 * 16;
  CUtensorMap tw;
  if (!ouu_tmap_bf16(&tw, W, (uint64_t)nn, (uint64_t)rm, (uint64_t)ldw, (uint32_t)BN)) {
    ouu_set_error("tensor map for the KL basis failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  // chunks of at most OUU_KLP_MAX_TILES tiles (one tile counter each); a chunk's first sample
  // is a multiple of 128, so its base keeps the fields' 16-byte alignment
  const int chunk = OUU_KLP_MAX_TILES * 128;
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int nc = std::min(chunk, N - n0);
    if (ouu_status st = kl_project_launch(m + (size_t)n0 * nn, nc, nn, tw, BN, rm, bias, xi + (size_t)n0 * rm, err,
                                          ctr, num_sms, s, n0 == 0 ? zsrc : nullptr, zdst, nz))
      return st;
  }
  return OUU_OK;
}

// Kernel-level entry used by the projection numerics test (declared in include/ouu_kernels.h).
extern "C" ouu_status ouu_kernel_kl_project(const double* m, int N, int nn, const void* W, int ldw, int rm,
                                            const float* bias, float* xi, int* err_dev, void* stream) {
  int dev = 0, sms = 0;
  OUU_CUDA_TRY(cudaGetDevice(&dev));
  OUU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  static int* ctr = nullptr;   // tile counters of this entry (one device per process)
  if (!ctr) {
    OUU_CUDA_TRY(cudaMalloc((void**)&ctr, (OUU_KLP_MAX_TILES + 1) * sizeof(int)));
    OUU_CUDA_TRY(cudaMemset(ctr, 0, (OUU_KLP_MAX_TILES + 1) * sizeof(int)));
  }
  return ouu_kl_project(m, N, nn, (const __nv_bfloat16*)W, ldw, rm, bias, xi, err_dev, ctr, sms, (cudaStream_t)stream);
}
