// The whole evaluation network of the reduced-basis neural operator (Sec. 3.3) in one kernel:
// for a tile of 128 samples, the forward pass [xi; z] -> width -> width -> width -> phi (width,
// r_U and d_Z at most 416, r_M + d_Z at most 448) with GELU
// (gelu.cuh), the reduced QoI Q = 1/2 ||phi + c||^2 + const and its seed s (phi + c), and the
// reverse-mode gradient grad_z Q = W0z^T (s'(a1) * W1^T (s'(a2) * W2^T (s'(a3) * W3^T seed))).
// The activations never leave shared memory: each layer's BF16 output is written, in the
// 128-byte swizzled K-major layout tcgen05.mma reads, over the layer's own input (its MMAs
// have completed by then).  Per CTA:
//   warps 0..15 : build the layer-0 input from xi (FP32) and z, then the epilogue of every
//                 layer: TMEM -> registers (warp w reads TMEM lanes 32 (w mod 4) .. + 31, columns
//                 of group w / 4), the layer's function, BF16 activations into shared memory;
//                 GELU'(a_l) to global FP32 (read back by the reverse layers), phi, Q, grad_z Q
//   warp 16     : TMA producer of the weight blocks of all layers, in order, through a two-stage
//                 ring (it runs ahead into the next layer while the epilogue works)
//   warp 17     : tcgen05.mma issuer (one or two N pieces of 208 columns per K step);
//                 allocates and frees the tensor memory (512 columns: two 208-column pieces)
// Every mbarrier wait is bounded; on a timeout the CTA stops and raises *err.
#include <cuda_bf16.h>

#include <cstring>

#include "dino.cuh"
#include "gelu.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#define MLP_EPI_WARPS 16
#define MLP_PROD_WARP 16
#define MLP_MMA_WARP 17
#define MLP_THREADS (18 * 32)
#define MLP_ABLOCKS 7                      // A buffer: 7 K blocks of 64 columns (448)
#define MLP_ABLOCK (128 * 64 * 2)
#define MLP_PIECE 208                      // rows of one weight box / columns of one MMA
#define MLP_BSTAGE (2 * MLP_PIECE * 128)   // two pieces of 208 rows x 64 BF16

enum { MLP_GELU_D = 0, MLP_QOI = 1, MLP_SCALE = 2, MLP_LINEAR_OUT = 3 };

struct MlpLayer {
  int K, N, npieces, box_rows, mode;
  const float* bias;     // GELU_D, QOI
  const float* scale;    // QOI: output scale s
  const float* add;      // QOI: c
  float* out_f32;        // GELU_D: gelu'(a); QOI: phi; LINEAR_OUT: grad_z Q
  int ld_out;
  const float* aux;      // SCALE: gelu'(a) of the forward layer
  int ld_aux;
};

struct MlpParams {
  CUtensorMap w[8];      // weights of the layers (rows = N, K contiguous)
  MlpLayer L[8];
  int nl, M, rm, dz;
  const float* xi;       // [M][rm]
  const float* zf;       // [dz]
  double* q_out;         // [M]
  double qconst;
  int* err;
};


// Epilogue column group of this warp: [c_begin, c_end) of the layer's N columns.
static __device__ __forceinline__ void mlp_group(int N, int g, int& cb, int& ce) {
  const int cg = ((N + 3) / 4 + 15) / 16 * 16;
  cb = g * cg;
  ce = min(N, cb + cg);
}

// Two 16-byte chunks (16 BF16 values, columns c0 .. c0 + 15, c0 a multiple of 16) of tile row r
// into the swizzled A buffer.
static __device__ __forceinline__ void mlp_store16(uint8_t* abuf, int r, int c0, const float* v) {
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    w[j] = *reinterpret_cast<const uint32_t*>(&p);
  }
  const int kb = c0 >> 6, cc = c0 & 63;
  uint8_t* rowp = abuf + kb * MLP_ABLOCK + r * 128;
  const uint32_t ch = (uint32_t)cc >> 3;   // 16-byte chunk of the 128-byte row
  *reinterpret_cast<uint4*>(rowp + (((ch) ^ (uint32_t)(r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(rowp + (((ch + 1) ^ (uint32_t)(r & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
}

__global__ void __launch_bounds__(MLP_THREADS, 1) k_mlp_eval(const __grid_constant__ MlpParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + MLP_ABLOCKS * MLP_ABLOCK;
  uint64_t* bars = (uint64_t*)(sB + 2 * MLP_BSTAGE);
  uint64_t* b_full = bars + 0;
  uint64_t* b_empty = bars + 2;
  uint64_t* a_ready = bars + 4;
  uint64_t* acc_full = bars + 5;
  uint64_t* mma_done = bars + 6;
  uint32_t* tslot = (uint32_t*)(bars + 8);
  __shared__ float s_rowq[128];
  __shared__ int s_rowc[128];
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&b_full[i], 1);
      mbar_init(&b_empty[i], 1);
    }
    mbar_init(a_ready, MLP_EPI_WARPS);
    mbar_init(acc_full, 1);
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == MLP_MMA_WARP) tmem_alloc(tslot, 512);
  // zero the activation buffer: the padding columns of every layer must hold finite values
  for (int i = threadIdx.x; i < MLP_ABLOCKS * MLP_ABLOCK / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x < 128) {
    s_rowq[threadIdx.x] = 0.f;
    s_rowc[threadIdx.x] = 0;
  }
  pdl_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == MLP_PROD_WARP) {
    // ------------------------------------------------------------------ weight producer
    if (lane == 0) {
      int g = 0, issued = 0;
      bool ok = true;
      for (int l = 0; l < P.nl && ok; ++l) {
        const MlpLayer& L = P.L[l];
        const int KB = (L.K + 63) / 64;
        const uint32_t bytes = (uint32_t)L.npieces * (uint32_t)L.box_rows * 128u;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g & 1;
          if (g >= 2 && !mbar_wait(&b_empty[s], ((uint32_t)(g >> 1) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&b_full[s], bytes);
          for (int p = 0; p < L.npieces; ++p)
            tma_load_2d(sB + s * MLP_BSTAGE + p * MLP_PIECE * 128, &P.w[l], kb * 64, p * MLP_PIECE, &b_full[s]);
          issued = g + 1;
        }
      }
      if (!ok) s_fail = 1;
      for (int j = max(0, issued - 2); j < issued; ++j)
        if (!mbar_wait(&b_full[j & 1], (uint32_t)(j >> 1) & 1u)) s_fail = 1;
    }
  } else if (warp == MLP_MMA_WARP) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int g = 0;
      bool ok = true, any = false;
      for (int l = 0; l < P.nl && ok; ++l) {
        const MlpLayer& L = P.L[l];
        const int KB = (L.K + 63) / 64;
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(L.box_rows >> 3) << 17) |
                               ((128u >> 4) << 24);
        if (!mbar_wait(a_ready, (uint32_t)l & 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g & 1;
          if (!mbar_wait(&b_full[s], (uint32_t)(g >> 1) & 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + kb * MLP_ABLOCK);
          for (int p = 0; p < L.npieces; ++p) {
            const uint32_t b0 = smem_u32(sB + s * MLP_BSTAGE + p * MLP_PIECE * 128);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              tc_mma(tmem + (uint32_t)(p * MLP_PIECE), smem_desc_sw128(a0 + k * 32), smem_desc_sw128(b0 + k * 32),
                     idesc, (kb | k) != 0 ? 1u : 0u);
          }
          tc_commit(&b_empty[s]);
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
    const int q = warp & 3, grp = warp >> 2;
    const int r = q * 32 + lane, row = m0 + r;   // this thread's tile row (TMEM lane)
    const bool in = row < P.M;
    {  // layer 0 input: [xi (rm); z (dz); 0]
      int cb, ce;
      mlp_group(P.L[0].K, grp, cb, ce);
      for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          float x = 0.f;
          if (in && c < P.rm) x = P.xi[(size_t)row * P.rm + c];
          else if (c >= P.rm && c < P.rm + P.dz) x = P.zf[c - P.rm];
          v[j] = x;
        }
        mlp_store16(sA, r, c0, v);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_ready);
    }
    for (int l = 0; l < P.nl; ++l) {
      const MlpLayer& L = P.L[l];
      if (!__all_sync(0xffffffffu, mbar_wait(acc_full, (uint32_t)l & 1u) ? 1 : 0)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      tc_fence_after();
      int cb, ce;
      mlp_group(L.N, grp, cb, ce);
      float sq = 0.f;
      for (int c0 = cb; c0 < ce; c0 += 16) {
        uint32_t u[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, u);
        float v[16];
        if (L.mode == MLP_GELU_D) {
          float dv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = c0 + j;
            gelu_and_d1(__uint_as_float(u[j]) + (c < L.N ? L.bias[c] : 0.f), v[j], dv[j]);
          }
          if (in) {
            float* o = L.out_f32 + (size_t)row * L.ld_out + c0;
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              if (c0 + j + 3 < L.N) *reinterpret_cast<float4*>(o + j) = make_float4(dv[j], dv[j + 1], dv[j + 2], dv[j + 3]);
              else
                for (int jj = j; jj < j + 4 && c0 + jj < L.N; ++jj) o[jj] = dv[jj];
          }
        } else if (L.mode == MLP_QOI) {
          float phi[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = c0 + j;
            const bool cin = c < L.N;
            phi[j] = cin ? (__uint_as_float(u[j]) + L.bias[c]) * L.scale[c] : 0.f;
            const float t = cin ? phi[j] + L.add[c] : 0.f;
            sq += t * t;
            v[j] = cin ? t * L.scale[c] : 0.f;
          }
          if (in) {
            float* o = L.out_f32 + (size_t)row * L.ld_out + c0;
            for (int j = 0; j < 16 && c0 + j < L.N; ++j) o[j] = phi[j];
          }
        } else if (L.mode == MLP_SCALE) {
          float f[16];
          const float* ap = L.aux + (size_t)(in ? row : 0) * L.ld_aux + c0;
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            if (in && c0 + j + 3 < L.N) {
              const float4 t = __ldg(reinterpret_cast<const float4*>(ap + j));
              f[j] = t.x, f[j + 1] = t.y, f[j + 2] = t.z, f[j + 3] = t.w;
            } else {
              for (int jj = j; jj < j + 4; ++jj) f[jj] = (in && c0 + jj < L.N) ? ap[jj] : 0.f;
            }
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(u[j]) * f[j];
        } else {   // MLP_LINEAR_OUT
          if (in) {
            float* o = L.out_f32 + (size_t)row * L.ld_out + c0;
            for (int j = 0; j < 16 && c0 + j < L.N; ++j) o[j] = __uint_as_float(u[j]);
          }
        }
        if (L.mode != MLP_LINEAR_OUT) mlp_store16(sA, r, c0, v);
      }
      if (L.mode == MLP_QOI) {
        // the row's four column groups add their partial sums; the last one to arrive writes Q
        atomicAdd(&s_rowq[r], sq);
        __threadfence_block();
        if (atomicAdd(&s_rowc[r], 1) == 3 && in) P.q_out[row] = P.qconst + 0.5 * (double)atomicAdd(&s_rowq[r], 0.f);
      }
      fence_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_ready);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MLP_MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(P.err, 1);
}

bool mlp_fused_fits(const ouu_dino* d) {
  return d->wd <= 2 * MLP_PIECE && d->ru <= 2 * MLP_PIECE && d->dz <= 2 * MLP_PIECE && d->in0 <= MLP_ABLOCKS * 64 &&
         d->wd <= MLP_ABLOCKS * 64 && d->ru <= MLP_ABLOCKS * 64 && (d->rm % 4) == 0;
}

// Fills one layer: weight map over rows [0, N) x K of the BF16 matrix at base (leading
// dimension ld), epilogue mode and operands.
static bool mlp_layer(MlpParams& P, int l, const __nv_bfloat16* base, int ld, int K, int N, int mode) {
  MlpLayer& L = P.L[l];
  std::memset(&L, 0, sizeof(L));
  L.K = K;
  L.N = N;
  L.npieces = (N + MLP_PIECE - 1) / MLP_PIECE;
  L.box_rows = L.npieces > 1 ? MLP_PIECE : (N + 15) / 16 * 16;
  L.mode = mode;
  return ouu_tmap_bf16(&P.w[l], base, (uint64_t)K, (uint64_t)N, (uint64_t)ld, (uint32_t)L.box_rows);
}

ouu_status mlp_fused_eval(ouu_dino* d, int N) {
  MlpParams P;   // kernel parameters: the launch copies them, so concurrent handles share nothing
  std::memset(&P, 0, sizeof(P));
  const int wd = d->wd, rup = (d->ru + 7) / 8 * 8, dzp = (d->dz + 7) / 8 * 8;
  bool ok = mlp_layer(P, 0, d->Wb[0], d->inp_l[0], d->in0, wd, MLP_GELU_D);
  ok = ok && mlp_layer(P, 1, d->Wb[1], d->inp_l[1], wd, wd, MLP_GELU_D);
  ok = ok && mlp_layer(P, 2, d->Wb[2], d->inp_l[2], wd, wd, MLP_GELU_D);
  ok = ok && mlp_layer(P, 3, d->Wb[3], d->inp_l[3], wd, d->ru, MLP_QOI);
  ok = ok && mlp_layer(P, 4, d->WTb[3], d->outp_l[3], d->ru, wd, MLP_SCALE);
  ok = ok && mlp_layer(P, 5, d->WTb[2], d->outp_l[2], wd, wd, MLP_SCALE);
  ok = ok && mlp_layer(P, 6, d->WTb[1], d->outp_l[1], wd, wd, MLP_SCALE);
  ok = ok && mlp_layer(P, 7, d->WTb[0] + (int64_t)d->rm * d->outp_l[0], d->outp_l[0], wd, d->dz, MLP_LINEAR_OUT);
  if (!ok) {
    ouu_set_error("tensor maps of the fused network failed (alignment or driver entry point)");
    return OUU_ERR_INVALID_ARG;
  }
  for (int l = 0; l < 3; ++l) {
    P.L[l].bias = d->d_params + d->offb[l];
    P.L[l].out_f32 = d->Ae[l + 1];
    P.L[l].ld_out = wd;
  }
  P.L[3].bias = d->d_params + d->offb[3];
  P.L[3].scale = d->d_oscale;
  P.L[3].add = d->d_cf;
  P.L[3].out_f32 = d->OUTe;
  P.L[3].ld_out = rup;
  for (int l = 4; l < 7; ++l) {
    P.L[l].aux = d->Ae[7 - l];
    P.L[l].ld_aux = wd;
  }
  P.L[7].out_f32 = d->GQe;
  P.L[7].ld_out = dzp;
  P.nl = 8;
  P.M = N;
  P.xi = d->XIe;
  P.rm = d->rm;
  P.zf = d->d_zf;
  P.dz = d->dz;
  P.q_out = d->Qe;
  P.qconst = d->qconst;
  P.err = d->d_err;
  const size_t smem = 1024 + MLP_ABLOCKS * MLP_ABLOCK + 2 * MLP_BSTAGE + 16 * 8;
  OUU_CUDA_TRY(ouu_smem_limit((const void*)k_mlp_eval, smem));
  OUU_CUDA_TRY(launch_pdl(k_mlp_eval, dim3((N + 127) / 128), dim3(MLP_THREADS), smem, d->stream, P));
  return OUU_OK;
}
