// BF16 tensor-core GEMM for sm_103a: TMA (SWIZZLE_128B) -> shared memory ->
// tcgen05.mma (kind::f16, FP32 accumulator in tensor memory) -> tcgen05.ld ->
// fused epilogue -> global.   D[M x N] = A[M x K] * B[N x K]^T, A and B K-major.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ouu_internal.cuh"

enum EpiMode {
  EPI_LINEAR = 0,       // y = alpha * acc + bias[c]
  EPI_GELU = 1,         // a = acc + bias[c]; out_f32 = a; bf16 outputs = gelu(a)
  EPI_DGELU_SCALE = 2,  // y = acc * gelu'(aux[(r / aux_rdiv) * ld_aux + c]); out2 = bf16(acc)
  EPI_GELU_D = 3,       // a = acc + bias[c]; out_f32 = gelu'(a); bf16 outputs = gelu(a)
  EPI_SCALE = 4,        // y = acc * aux[(r / aux_rdiv) * ld_aux + c]
  EPI_QOI = 5,          // phi = (acc + bias[c]) * col_scale[c] -> out_f32; v = phi + col_add[c];
                        // bf16 outputs = v * col_scale[c]; out_q[r] = qconst + 1/2 sum_c v^2
                        // (one N tile: N <= 256)
  EPI_DECODE = 6,       // rows r are grid nodes, columns c samples: v = acc + col_add[r] ->
                        // out_f32[c * ld_f32 + r]; out_q[c] += qconst * sum_r (v - col_ref[r])^2
                        // (out_q zeroed beforehand; col_add, col_ref indexed by row)
};

struct EpiParams {
  int mode;
  float alpha;
  const float* bias;              // [N] or null
  const float* col_scale;         // EPI_LINEAR: y *= col_scale[c] after the bias (null: 1)
  float* out_f32;                 // [M][ld_f32] or null
  int ld_f32;
  int accumulate;                 // out_f32 += y instead of =
  __nv_bfloat16* out_bf16;        // [M][ld_bf16] or null
  int ld_bf16;
  __nv_bfloat16* out_t_bf16;      // transposed: [N][ld_t] (element (r, c) at c * ld_t + r) or null
  int ld_t;
  __nv_bfloat16* out2_bf16;       // [M][ld2]: bf16(acc) before scaling (EPI_DGELU_SCALE) or null
  int ld2;
  const float* aux;               // EPI_DGELU_SCALE: pre-activations; EPI_SCALE: factors
  int ld_aux;
  int aux_rdiv;
  int vec;                        // set by ouu_gemm_bf16: vector epilogue accesses are aligned
  const float* col_add;           // EPI_QOI: per-column shift c
  double* out_q;                  // EPI_QOI, EPI_DECODE: [M] per-row quadratic
  double qconst;                  // EPI_QOI: added to every out_q; EPI_DECODE: factor of the sum
  const float* col_ref;           // EPI_DECODE: per-row reference subtracted before squaring
};

// Tensor map of a row-major BF16 matrix [rows][ld] (K = inner, contiguous), box 64 x box_rows.
// Returns false when the driver entry point is unavailable or the encode fails
// (base must be 16-byte aligned and ld a multiple of 8).
bool ouu_tmap_bf16(CUtensorMap* map, const void* base, uint64_t k, uint64_t rows, uint64_t ld, uint32_t box_rows);

// General 2-D tensor map (dims d0 inner, d1 outer; outer stride in bytes, a multiple of 16;
// box0 * esize a multiple of 16; out-of-range elements read as zero).
bool ouu_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, uint32_t esize, const void* base, uint64_t d0, uint64_t d1,
                 uint64_t stride1_bytes, uint32_t box0, uint32_t box1, CUtensorMapSwizzle sw);

// Launch D = A B^T with A = [M][K] (lda), B = [N][K] (ldb), both BF16 row-major; the N
// tile is chosen for the least padding.  err: device int set non-zero when a wait times
// out.  splits > 1: split-K over gridDim.z; only for one FP32 EPI_LINEAR output, which the
// CTAs accumulate atomically and which must be zeroed beforehand.
ouu_status ouu_gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                         const EpiParams& ep, int* err, cudaStream_t s, int splits = 1);

// Autotuning of the N tile: while on, the first call of each (M, N, K, mode, split) shape
// outside stream capture times every candidate tile (a warm-up and three timed launches,
// CUDA events on the call's stream) and keeps the fastest for all later calls of that shape.
// Shapes whose outputs accumulate (accumulate flag, split-K) are not tuned.
void ouu_gemm_set_autotune(int on);
int ouu_gemm_tuned_count();
