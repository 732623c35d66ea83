// The evaluation network of the reduced-basis neural operator (Sec. 3.3) in one kernel, each
// 128-sample tile on a cluster of 4 CTAs, each CTA computing a quarter of the columns of
// every layer: forward [xi; z] -> width -> width -> width -> phi with GELU (gelu.cuh), the reduced
// QoI Q = 1/2 ||phi + c||^2 + const with its seed s (phi + c), and the reverse-mode gradient
// grad_z Q = W0z^T (s'(a1) * W1^T (s'(a2) * W2^T (s'(a3) * W3^T seed))).
// The layers' BF16 activations pass through the handle's evaluation buffers (L2-resident,
// alternating between two of them so that no layer overwrites an operand another CTA may
// still read); each CTA's epilogue warps publish their slice of a layer's output and arrive
// on an "input complete" mbarrier in every CTA of the cluster, and a CTA loads the next
// layer's operand by TMA once its barrier has seen all 64 arrivals.  Per CTA:
//   warps 0..15 : build the CTA's columns of the layer-0 input from xi (FP32) and z; then per
//                 layer: TMEM -> shared staging (warp w reads TMEM lanes 32 (w mod 4) .. + 31),
//                 and a coalesced pass over the staged slice: the layer's function, BF16
//                 activations and FP32 side outputs (gelu'(a), phi, grad_z Q) to global
//   warp 16     : TMA producer: the CTA's rows of the weights through a 7-stage ring (a whole
//                 layer ahead, during the previous epilogue), and, once the layer's input is
//                 complete, all of the tile's input K blocks at once (up to 7 x 64 columns
//                 stay resident; the staging tile of the epilogue reuses their space once the
//                 MMAs are done)
//   warp 17     : tcgen05.mma issuer (M = 128, N = the CTA's columns); allocates and frees
//                 the tensor memory
// The layers can run as two launches, [0, 4) (forward and reduced QoI) and [4, 8) (reverse
// mode), so that work needing only Q can run beside the second one.
// Every mbarrier wait is bounded; on a timeout the CTA skips the remaining work (still
// arriving on its peers' barriers) and raises *err.  The only unbounded waits are the two
// cluster barriers every thread reaches unconditionally: after the barriers' initialisation
// and before exit (no CTA leaves while a peer may still arrive on its barriers).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "dino.cuh"
#include "gelu.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#define MLC_CS 4                        // CTAs per cluster: column quarters of every layer
#define MLC_EPI_WARPS 16
#define MLC_PROD_WARP 16
#define MLC_MMA_WARP 17
#define MLC_THREADS (18 * 32)
#define MLC_STAGES 7                    // weight ring: a whole layer's weights ahead of its input
#define MLC_KBMAX 7                     // resident input K blocks: K <= 448
#define MLC_NCMAX 128                   // columns of one CTA's slice (TMEM columns, weight box rows)
#define MLC_A_BYTES (128 * 64 * 2)
#define MLC_W_BYTES (MLC_NCMAX * 64 * 2)
#define MLC_SROW (MLC_NCMAX + 4)        // staging row stride in floats
#define MLC_LAYERS 8
#define MLC_QMAX 8                      // quads per epilogue thread: 128 rows x 32 quads / 512
#define MLC_SMEM (1024 + MLC_KBMAX * MLC_A_BYTES + MLC_STAGES * MLC_W_BYTES + (MLC_KBMAX + 2 * MLC_STAGES + 5) * 8 + 16)
static_assert(128 * MLC_SROW * 4 <= MLC_KBMAX * MLC_A_BYTES, "the staging tile lives in the input blocks");

enum { MLC_GELU_D = 0, MLC_QOI = 1, MLC_SCALE = 2, MLC_LINEAR_OUT = 3 };

struct MlcLayer {
  int K, N, nc, mode;
  const float* bias;            // GELU_D, QOI
  const float* scale;           // QOI: output scale s
  const float* add;             // QOI: c
  float* out_f32;               // GELU_D: gelu'(a); QOI: phi; LINEAR_OUT: grad_z Q
  int ld_f32;
  __nv_bfloat16* out_bf16;      // GELU_D: gelu(a); QOI: seed s (phi + c); SCALE: s'(a) * (g W)
  int ld_bf16;
  const float* aux;             // SCALE: gelu'(a) of the forward layer
  int ld_aux;
};

struct MlcParams {
  CUtensorMap a[MLC_LAYERS];    // layer inputs [M][K] BF16, 64 x 128 boxes (128-byte swizzle)
  CUtensorMap w[MLC_LAYERS];    // layer weights [N][K] BF16, 64 x nc boxes
  MlcLayer L[MLC_LAYERS];
  int M, rm, dz, in0p;
  int l0, l1;                   // the layers [l0, l1) of this launch; l0 > 0: layer l0's input
                                // is already in its evaluation buffer (an earlier launch)
  const float* xi;              // [M][rm]
  const float* zf;              // [dz]
  __nv_bfloat16* x0;            // [M][in0p] layer-0 input, built here
  float* qpart;                 // [M][4] per-CTA partial sums of (phi + c)^2
  double* q_out;                // [M]; null when the QoI layer is not in [l0, l1)
  double* q_mom;                // with q_out: [tiles][2] the tile's sum Q and sum Q^2 (FP64)
  double qconst;
  int* err;
};

static __device__ __forceinline__ uint32_t mlc_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

static __device__ __forceinline__ void mlc_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrival (release, cluster scope) on the barrier at the same shared address in CTA `rank`.
static __device__ __forceinline__ void mlc_arrive_remote(uint64_t* bar, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// Bounded wait (acquire, cluster scope) for the phase of the given parity.
static __device__ __forceinline__ bool mlc_wait_cluster(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(1000000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
}

// Named barrier of the 16 epilogue warps.
static __device__ __forceinline__ void mlc_epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(MLC_EPI_WARPS * 32) : "memory");
}

// This thread's global writes ordered before later TMA (async-proxy) reads in the other CTAs
// of the cluster: the proxy fence, then a release at cluster scope (every reader is in this
// thread's cluster, and it acquires through the cluster-scope mbarrier arrival that follows).
static __device__ __forceinline__ void mlc_publish() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.acq_rel.cluster;" ::: "memory");
}

static __device__ __forceinline__ void mlc_store_bf16x4(__nv_bfloat16* p, const float* v, int nv) {
  if (nv == 4) {
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
  } else {
    for (int j = 0; j < nv; ++j) p[j] = __float2bfloat16(v[j]);
  }
}

static __device__ __forceinline__ void mlc_store_f32x4(float* p, const float* v, int nv) {
  if (nv == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    for (int j = 0; j < nv; ++j) p[j] = v[j];
  }
}

__global__ void __launch_bounds__(MLC_THREADS, 1) k_mlp_cluster(const __grid_constant__ MlcParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                   // input K blocks, then the staging tile
  uint8_t* sW = sA + MLC_KBMAX * MLC_A_BYTES;
  float* stg = (float*)sA;
  uint64_t* bars = (uint64_t*)(sW + MLC_STAGES * MLC_W_BYTES);
  uint64_t* a_full = bars;                              // [MLC_KBMAX] input block kb landed
  uint64_t* w_full = bars + MLC_KBMAX;                  // [MLC_STAGES] weight block landed
  uint64_t* w_empty = w_full + MLC_STAGES;              // [MLC_STAGES] MMA: weight stage consumed
  uint64_t* acc_full = w_empty + MLC_STAGES;            // MMA: the layer's accumulator is complete
  uint64_t* acc_empty = acc_full + 1;                   // epilogue: accumulator read into staging
  // cluster: layer l's input is complete, on barrier l % 2 in its phase l / 2.  Two barriers:
  // an arrival for layer l + 2 can only follow this CTA's own completion of layer l (through
  // its peers' waits on layer l + 1), never overtake an arrival for layer l
  uint64_t* layer_in = acc_full + 2;                    // [2]
  uint64_t* mma_done = acc_full + 4;
  uint32_t* tslot = (uint32_t*)(acc_full + 5);
  __shared__ float s_cb[3][MLC_NCMAX];                  // the layer's bias, scale, add per column
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = mlc_cluster_rank();
  const int m0 = (int)(blockIdx.x / MLC_CS) * 128;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < MLC_KBMAX; ++i) mbar_init(&a_full[i], 1);
    for (int i = 0; i < MLC_STAGES; ++i) {
      mbar_init(&w_full[i], 1);
      mbar_init(&w_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, MLC_EPI_WARPS);
    mbar_init(&layer_in[0], MLC_CS * MLC_EPI_WARPS);
    mbar_init(&layer_in[1], MLC_CS * MLC_EPI_WARPS);
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == MLC_MMA_WARP) tmem_alloc(tslot, MLC_NCMAX);
  if (warp == MLC_PROD_WARP && lane < 2 * MLC_LAYERS) {   // the launch's descriptors, off the critical path
    const int ll = lane < MLC_LAYERS ? lane : lane - MLC_LAYERS;
    if (ll >= P.l0 && ll < P.l1) tmap_prefetch(lane < MLC_LAYERS ? &P.a[ll] : &P.w[ll]);
  }
  // The first layer's weights do not come from earlier kernels: their copies start before the
  // wait on those kernels (the ring's first stages, free at launch).
  int wpre = 0;
  {
    const MlcLayer& L = P.L[P.l0];
    wpre = min((L.K + 63) / 64, MLC_STAGES);
  }
  __syncthreads();   // the barriers are initialised
  if (warp == MLC_PROD_WARP && lane == 0) {
    const MlcLayer& L = P.L[P.l0];
    for (int kb = 0; kb < wpre; ++kb) {
      mbar_expect_tx(&w_full[kb], (uint32_t)L.nc * 128u);
      tma_load_2d(sW + kb * MLC_W_BYTES, &P.w[P.l0], kb * 64, (int)rank * L.nc, &w_full[kb]);
    }
  }
  pdl_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  mlc_cluster_sync();   // every CTA's barriers exist before the first remote arrival
  const uint32_t tmem = *tslot;

  if (warp == MLC_PROD_WARP) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int gw = 0, wissued = wpre;
      int a_uses[MLC_KBMAX];
#pragma unroll
      for (int i = 0; i < MLC_KBMAX; ++i) a_uses[i] = 0;
      bool ok = true;
      for (int l = P.l0; l < P.l1 && ok; ++l) {
        const MlcLayer& L = P.L[l];
        const int li = l - P.l0;   // barrier bookkeeping counts the launch's own layers
        const int KB = (L.K + 63) / 64, pre = min(KB, MLC_STAGES), wrow = (int)rank * L.nc;
        const uint32_t wbytes = (uint32_t)L.nc * 128u;
        auto load_w = [&](int kb) {   // weight block kb of this layer into the ring
          const int f = gw + kb, s = f % MLC_STAGES;
          if (f >= MLC_STAGES && !mbar_wait(&w_empty[s], ((uint32_t)(f / MLC_STAGES) & 1u) ^ 1u)) return false;
          mbar_expect_tx(&w_full[s], wbytes);
          tma_load_2d(sW + s * MLC_W_BYTES, &P.w[l], kb * 64, wrow, &w_full[s]);
          wissued = f + 1;
          return true;
        };
        for (int kb = l == P.l0 ? wpre : 0; kb < pre && ok; ++kb) ok = load_w(kb);   // ahead of the layer's input
        if (!ok) break;
        // the layer's input is complete in every CTA of the cluster; on a timeout the input is
        // still loaded, so that every barrier armed here completes before the CTA exits
        if (!mlc_wait_cluster(&layer_in[li & 1], (uint32_t)(li >> 1) & 1u)) ok = false;
        asm volatile("fence.proxy.async.global;" ::: "memory");
        // all of the layer's input blocks at once (multicasting each block from one CTA of the
        // cluster to all four measured slower: each CTA then waits for its slowest peer)
        for (int kb = 0; kb < KB; ++kb) {
          mbar_expect_tx(&a_full[kb], MLC_A_BYTES);
          tma_load_2d(sA + kb * MLC_A_BYTES, &P.a[l], kb * 64, m0, &a_full[kb]);
          ++a_uses[kb];
        }
        for (int kb = pre; kb < KB && ok; ++kb) ok = load_w(kb);
        gw += KB;
        if (ok && l + 1 < P.l1) {
          // the input blocks are overwritten only once the epilogue of this layer is done (the
          // next layer's input wait follows it), so nothing else to wait for here
        }
      }
      if (!ok) s_fail = 1;
      // drain: every copy issued has landed before the CTA exits
      for (int kb = 0; kb < MLC_KBMAX; ++kb)
        if (a_uses[kb] > 0 && !mbar_wait(&a_full[kb], (uint32_t)(a_uses[kb] - 1) & 1u)) s_fail = 1;
      for (int f = max(0, wissued - MLC_STAGES); f < wissued; ++f)
        if (!mbar_wait(&w_full[f % MLC_STAGES], (uint32_t)(f / MLC_STAGES) & 1u)) s_fail = 1;
    }
  } else if (warp == MLC_MMA_WARP) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int gw = 0;
      uint32_t apar = 0;   // bit kb: parity of the next completion of a_full[kb]
      bool ok = true, any = false;
      for (int l = P.l0; l < P.l1 && ok; ++l) {
        const MlcLayer& L = P.L[l];
        const int li = l - P.l0;
        const int KB = (L.K + 63) / 64;
        const uint32_t idesc =
            (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(L.nc >> 3) << 17) | ((128u >> 4) << 24);
        if (li > 0 && !mbar_wait(acc_empty, (uint32_t)(li - 1) & 1u)) {   // previous accumulator read
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < KB; ++kb, ++gw) {
          const int s = gw % MLC_STAGES;
          if (!mbar_wait(&a_full[kb], (apar >> kb) & 1u) || !mbar_wait(&w_full[s], (uint32_t)(gw / MLC_STAGES) & 1u)) {
            ok = false;
            break;
          }
          apar ^= 1u << kb;
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + kb * MLC_A_BYTES), b0 = smem_u32(sW + s * MLC_W_BYTES);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc_mma(tmem, smem_desc_sw128(a0 + k * 32), smem_desc_sw128(b0 + k * 32), idesc, (kb | k) != 0 ? 1u : 0u);
          tc_commit(&w_empty[s]);
          any = true;
        }
        if (ok) tc_commit(acc_full);
      }
      if (!ok) s_fail = 1;
      if (any) {
        tc_commit(mma_done);
        if (!mbar_wait(mma_done, 0)) s_fail = 1;
      }
    }
  } else {
    // ------------------------------------------------------------------ input build + epilogues
    const int q = warp & 3, grp = warp >> 2, et = threadIdx.x;
    constexpr int NT = MLC_EPI_WARPS * 32;
    if (P.l0 > 0) {   // the first layer's input came from an earlier launch (complete after pdl_wait)
      __syncwarp();
      if (lane == 0)
        for (uint32_t r = 0; r < MLC_CS; ++r) mlc_arrive_remote(&layer_in[0], r);
    } else {  // this CTA's quad-aligned quarter of the layer-0 input columns: [xi (rm); z (dz); 0]
      const int cw = ((P.in0p / 4 + MLC_CS - 1) / MLC_CS) * 4;
      const int cb = (int)rank * cw, ce = min(P.in0p, cb + cw), nq = max(0, ce - cb) / 4;
      float4 xv[MLC_QMAX];
#pragma unroll
      for (int i = 0; i < MLC_QMAX; ++i) {   // all loads first: one round trip
        const int e = et + i * NT;
        xv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < 128 * nq) {
          const int tr = e / nq, c = cb + 4 * (e - tr * nq), row = m0 + tr;
          if (row < P.M) {
            if (c + 3 < P.rm) {   // r_m % 4 == 0: a quad is all xi or all z / padding
              xv[i] = __ldg(reinterpret_cast<const float4*>(P.xi + (size_t)row * P.rm + c));
            } else {
              float v[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int cc = c + j - P.rm;
                v[j] = cc >= 0 && cc < P.dz ? __ldg(P.zf + cc) : 0.f;
              }
              xv[i] = make_float4(v[0], v[1], v[2], v[3]);
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < MLC_QMAX; ++i) {
        const int e = et + i * NT;
        if (e < 128 * nq) {
          const int tr = e / nq, c = cb + 4 * (e - tr * nq), row = m0 + tr;
          const float v[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
          if (row < P.M) mlc_store_bf16x4(P.x0 + (size_t)row * P.in0p + c, v, 4);
        }
      }
      mlc_publish();
      __syncwarp();
      if (lane == 0)
        for (uint32_t r = 0; r < MLC_CS; ++r) mlc_arrive_remote(&layer_in[0], r);
    }
    bool live = true;
    for (int l = P.l0; l < P.l1; ++l) {
      const MlcLayer& L = P.L[l];
      const int li = l - P.l0;
      const int c0 = (int)rank * L.nc, QPR = L.nc / 4, NQ = 128 * QPR;
      // Before acc_full of this layer every epilogue warp of this CTA finished the previous
      // layer (the input of this one waited for their arrivals): the staging tile (in the
      // input blocks, which this layer's MMAs no longer read) and s_cb are free.
      float cb0 = 0.f, cb1 = 0.f, cb2 = 0.f;   // the layer's per-column constants, loaded early
      if (et < L.nc && c0 + et < L.N) {
        if (L.bias) cb0 = __ldg(L.bias + c0 + et);
        if (L.scale) cb1 = __ldg(L.scale + c0 + et);
        if (L.add) cb2 = __ldg(L.add + c0 + et);
      }
      // quad e = et + i NT of the slice: row tr_i, quad cq_i, stepped without dividing
      const int tr_s = NT / QPR, cq_s = NT - tr_s * QPR, tr0 = et / QPR, cq0 = et - tr0 * QPR;
      float4 ax[MLC_QMAX];   // SCALE: the forward layer's gelu'(a), loaded before the accumulator is ready
      if (L.mode == MLC_SCALE) {
#pragma unroll
        for (int i = 0, tr = tr0, cq = cq0; i < MLC_QMAX; ++i, tr += tr_s + (cq + cq_s >= QPR), cq += cq_s - (cq + cq_s >= QPR ? QPR : 0)) {
          const int e = et + i * NT, c = c0 + 4 * cq, row = m0 + tr;
          ax[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (e < NQ && row < P.M && c < L.N) {
            const float* ap = L.aux + (size_t)row * L.ld_aux + c;
            if (c + 3 < L.N) {
              ax[i] = __ldcg(reinterpret_cast<const float4*>(ap));
            } else {
              float x[4] = {0.f, 0.f, 0.f, 0.f};
              for (int j = 0; j < L.N - c; ++j) x[j] = __ldcg(ap + j);
              ax[i] = make_float4(x[0], x[1], x[2], x[3]);
            }
          }
        }
      }
      if (live) live = __all_sync(0xffffffffu, mbar_wait(acc_full, (uint32_t)li & 1u) ? 1 : 0) != 0;
      if (!live && lane == 0) s_fail = 1;
      tc_fence_after();
      const int nch = (L.nc + 15) / 16;
      if (live)
        for (int k = grp; k < nch; k += 4) {
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * k), v);
          float4* sp = reinterpret_cast<float4*>(stg + (q * 32 + lane) * MLC_SROW + 16 * k);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            sp[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]), __uint_as_float(v[4 * j + 2]),
                                __uint_as_float(v[4 * j + 3]));
        }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      if (et < L.nc) {
        s_cb[0][et] = cb0;
        s_cb[1][et] = cb1;
        s_cb[2][et] = cb2;
      }
      mlc_epi_sync();   // the staging tile and the constants are complete
      if (live && L.mode == MLC_QOI) {
        // whole rows per warp, lanes over the row's quads; the row's partial (phi + c)^2 sum (the
        // 8 rows of a warp unrolled, so that their loads and reductions overlap)
#pragma unroll
        for (int tr = warp; tr < 128; tr += MLC_EPI_WARPS) {
          const int row = m0 + tr, cq = 4 * lane, c = c0 + cq;
          float sq = 0.f;
          if (lane < QPR && c < L.N) {
            const float4 a4 = *reinterpret_cast<const float4*>(stg + tr * MLC_SROW + cq);
            const float acc[4] = {a4.x, a4.y, a4.z, a4.w};
            const int nv = min(4, L.N - c);
            float phi[4], sv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const bool cin = j < nv;
              phi[j] = cin ? (acc[j] + s_cb[0][cq + j]) * s_cb[1][cq + j] : 0.f;
              const float t = cin ? phi[j] + s_cb[2][cq + j] : 0.f;
              sq += t * t;
              sv[j] = cin ? t * s_cb[1][cq + j] : 0.f;
            }
            if (row < P.M) {
              mlc_store_f32x4(L.out_f32 + (size_t)row * L.ld_f32 + c, phi, nv);
              mlc_store_bf16x4(L.out_bf16 + (size_t)row * L.ld_bf16 + c, sv, nv);
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
          if (lane == 0 && row < P.M) P.qpart[(size_t)row * MLC_CS + rank] = sq;
        }
      } else if (live && L.mode == MLC_SCALE) {
#pragma unroll
        for (int i = 0, tr = tr0, cq = cq0; i < MLC_QMAX; ++i, tr += tr_s + (cq + cq_s >= QPR), cq += cq_s - (cq + cq_s >= QPR ? QPR : 0)) {
          const int e = et + i * NT, c = c0 + 4 * cq, row = m0 + tr;
          if (e < NQ && row < P.M && c < L.N) {
            const float4 a4 = *reinterpret_cast<const float4*>(stg + tr * MLC_SROW + (c - c0));
            const float o[4] = {a4.x * ax[i].x, a4.y * ax[i].y, a4.z * ax[i].z, a4.w * ax[i].w};
            mlc_store_bf16x4(L.out_bf16 + (size_t)row * L.ld_bf16 + c, o, min(4, L.N - c));
          }
        }
      } else if (live) {
#pragma unroll
        for (int i = 0, tr = tr0, qq = cq0; i < MLC_QMAX; ++i, tr += tr_s + (qq + cq_s >= QPR), qq += cq_s - (qq + cq_s >= QPR ? QPR : 0)) {
          const int e = et + i * NT, cq = 4 * qq, c = c0 + cq, row = m0 + tr;
          if (e >= NQ || row >= P.M || c >= L.N) continue;
          const int nv = min(4, L.N - c);
          const float4 a4 = *reinterpret_cast<const float4*>(stg + tr * MLC_SROW + cq);
          const float acc[4] = {a4.x, a4.y, a4.z, a4.w};
          if (L.mode == MLC_GELU_D) {
            float o[4], y[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) gelu_and_d1(acc[j] + s_cb[0][cq + j], o[j], y[j]);   // one exp for both
            mlc_store_bf16x4(L.out_bf16 + (size_t)row * L.ld_bf16 + c, o, nv);
            mlc_store_f32x4(L.out_f32 + (size_t)row * L.ld_f32 + c, y, nv);
          } else {   // MLC_LINEAR_OUT
            mlc_store_f32x4(L.out_f32 + (size_t)row * L.ld_f32 + c, acc, nv);
          }
        }
      }
      if (l + 1 < P.l1) {   // this warp's part of the next layer's input is published
        mlc_publish();
        __syncwarp();
        if (lane == 0)
          for (uint32_t r = 0; r < MLC_CS; ++r) mlc_arrive_remote(&layer_in[(li + 1) & 1], r);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MLC_MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, MLC_NCMAX);
  }
  mlc_cluster_sync();   // no CTA leaves while a peer may arrive on its barriers; partial sums visible
  if (P.q_out && rank == 0 && threadIdx.x < 128) {
    const int row = m0 + threadIdx.x;
    double qv = 0.0;
    if (row < P.M) {
      const float* p = P.qpart + (size_t)row * MLC_CS;
      qv = P.qconst + 0.5 * (double)(((p[0] + p[1]) + p[2]) + p[3]);
      P.q_out[row] = qv;
    }
    // the tile's moments for the risk passes (the four warps' shuffle sums, then warp 0)
    double s1 = qv, s2 = qv * qv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    double* red = reinterpret_cast<double*>(smem);   // the input blocks are idle now
    if (lane == 0) {
      red[2 * warp] = s1;
      red[2 * warp + 1] = s2;
    }
    asm volatile("bar.sync 2, 128;" ::: "memory");
    if (threadIdx.x == 0) {
      P.q_mom[2 * (m0 / 128)] = (red[0] + red[2]) + (red[4] + red[6]);
      P.q_mom[2 * (m0 / 128) + 1] = (red[1] + red[3]) + (red[5] + red[7]);
    }
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(P.err, 1);
}

static int mlc_nc(int N) { return ((N + MLC_CS - 1) / MLC_CS + 15) / 16 * 16; }

bool mlp_cluster_fits(const ouu_dino* d) {
  return mlc_nc(d->wd) <= MLC_NCMAX && mlc_nc(d->ru) <= MLC_NCMAX && mlc_nc(d->dz) <= MLC_NCMAX && d->rm % 4 == 0 &&
         d->wd % 8 == 0 && d->in0 <= 64 * MLC_KBMAX && d->wd <= 64 * MLC_KBMAX && d->ru <= 64 * MLC_KBMAX &&
         d->inp_l[0] <= 64 * MLC_QMAX;
}

// One layer: input map over [M][K] at a (leading dimension lda), weight map over rows [0, N)
// x K of the BF16 matrix at w (leading dimension ldw), column slice and epilogue mode.
static bool mlc_layer(MlcParams& P, int l, const __nv_bfloat16* a, int lda, const __nv_bfloat16* w, int ldw, int K,
                      int N, int mode) {
  MlcLayer& L = P.L[l];
  std::memset(&L, 0, sizeof(L));
  L.K = K;
  L.N = N;
  L.nc = mlc_nc(N);
  L.mode = mode;
  return ouu_tmap_bf16(&P.a[l], a, (uint64_t)K, (uint64_t)P.M, (uint64_t)lda, 128u) &&
         ouu_tmap_bf16(&P.w[l], w, (uint64_t)K, (uint64_t)N, (uint64_t)ldw, (uint32_t)L.nc);
}

ouu_status mlp_cluster_eval(ouu_dino* d, int N, int l0, int l1) {
  MlcParams P;   // kernel parameters: the launch copies them, so concurrent handles share nothing
  std::memset(&P, 0, sizeof(P));
  P.M = N;
  P.l0 = l0;
  P.l1 = l1;
  const int wd = d->wd, rup = (d->ru + 7) / 8 * 8, dzp = (d->dz + 7) / 8 * 8, in0p = d->inp_l[0];
  bool ok = mlc_layer(P, 0, d->X0e, in0p, d->Wb[0], d->inp_l[0], d->in0, wd, MLC_GELU_D);
  ok = ok && mlc_layer(P, 1, d->He0, wd, d->Wb[1], d->inp_l[1], wd, wd, MLC_GELU_D);
  ok = ok && mlc_layer(P, 2, d->He1, wd, d->Wb[2], d->inp_l[2], wd, wd, MLC_GELU_D);
  ok = ok && mlc_layer(P, 3, d->He0, wd, d->Wb[3], d->inp_l[3], wd, d->ru, MLC_QOI);
  ok = ok && mlc_layer(P, 4, d->Ge, rup, d->WTb[3], d->outp_l[3], d->ru, wd, MLC_SCALE);
  ok = ok && mlc_layer(P, 5, d->He1, wd, d->WTb[2], d->outp_l[2], wd, wd, MLC_SCALE);
  ok = ok && mlc_layer(P, 6, d->He0, wd, d->WTb[1], d->outp_l[1], wd, wd, MLC_SCALE);
  ok = ok && mlc_layer(P, 7, d->He1, wd, d->WTb[0] + (int64_t)d->rm * d->outp_l[0], d->outp_l[0], wd, d->dz,
                       MLC_LINEAR_OUT);
  if (!ok) {
    ouu_set_error("tensor maps of the cluster network failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  __nv_bfloat16* hout[3] = {d->He0, d->He1, d->He0};
  for (int l = 0; l < 3; ++l) {
    P.L[l].bias = d->d_params + d->offb[l];
    P.L[l].out_f32 = d->Ae[l + 1];
    P.L[l].ld_f32 = wd;
    P.L[l].out_bf16 = hout[l];
    P.L[l].ld_bf16 = wd;
  }
  P.L[3].bias = d->d_params + d->offb[3];
  P.L[3].scale = d->d_oscale;
  P.L[3].add = d->d_cf;
  P.L[3].out_f32 = d->OUTe;
  P.L[3].ld_f32 = rup;
  P.L[3].out_bf16 = d->Ge;
  P.L[3].ld_bf16 = rup;
  __nv_bfloat16* gout[3] = {d->He1, d->He0, d->He1};
  for (int l = 4; l < 7; ++l) {
    P.L[l].aux = d->Ae[7 - l];
    P.L[l].ld_aux = wd;
    P.L[l].out_bf16 = gout[l - 4];
    P.L[l].ld_bf16 = wd;
  }
  P.L[7].out_f32 = d->GQe;
  P.L[7].ld_f32 = dzp;
  P.rm = d->rm;
  P.dz = d->dz;
  P.in0p = in0p;
  P.xi = d->XIe;
  P.zf = d->d_zf;
  P.x0 = d->X0e;
  P.qpart = d->Qpart;
  P.q_out = l0 <= 3 && 3 < l1 ? d->Qe : nullptr;
  P.q_mom = d->Qmom;
  P.qconst = d->qconst;
  P.err = d->d_err;
  const size_t smem = MLC_SMEM;
  OUU_CUDA_TRY(ouu_smem_limit((const void*)k_mlp_cluster, smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MLC_CS * ((N + 127) / 128));
  cfg.blockDim = dim3(MLC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = d->stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = MLC_CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  OUU_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_mlp_cluster, P));
  return OUU_OK;
}
