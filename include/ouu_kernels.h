/* ouu_kernels.h -- kernel-level entry points of libouu.so used by the numerics
 * tests of individual CUDA kernels (the product calls are in ouu.h).
 *
 * ouu_kernel_gemm_bf16: D[M x N] = A[M x K] * B[N x K]^T on the tcgen05 tensor
 * cores (TMA-fed, BF16 operands, FP32 accumulation in tensor memory), with the
 * fused epilogue `mode` applied to the accumulator acc at row r, column c:
 *   0 LINEAR     : y = alpha * acc + bias[c]
 *   1 GELU       : a = acc + bias[c]; out_f32 = a; BF16 outputs = gelu(a)   (GELU x Phi(x), Phi by A&S 26.2.17)
 *   2 DGELU_SCALE: y = acc * gelu'(aux[(r / aux_rdiv) * ld_aux + c]); out2 = bf16(acc)
 *   3 GELU_D     : a = acc + bias[c]; out_f32 = gelu'(a); BF16 outputs = gelu(a)
 *   4 SCALE      : y = acc * aux[(r / aux_rdiv) * ld_aux + c]
 *   5 QOI        : phi = (acc + bias[c]) s[c] -> out_f32, v = phi + c_add[c], BF16 outputs = v s[c],
 *                  out_q[r] = qconst + 1/2 sum_c v^2 (the reduced QoI of Sec. 3.3 and its seed);
 *                  N <= 256; s, c_add, out_q given by ouu_kernel_gemm_qoi_bf16
 * These are the dense layers of the reduced-basis network of Sec. 3.3 (forward
 * values, forward-mode control-Jacobian tangents, and their adjoints).
 * A, B: device BF16 row-major with leading dimensions lda, ldb (multiples of 8,
 * 16-byte aligned bases).  Outputs (each may be NULL): out_f32 [M][ld_f32]
 * (overwritten, or incremented when accumulate != 0), out_bf16 [M][ld_bf16],
 * out_t_bf16 transposed [N][ld_t], out2_bf16 [M][ld2].  err_dev: device int set
 * to 1 if a pipeline wait timed out (the kernel then returns without hanging).
 * Launches on `stream`; returns INVALID_ARG for bad sizes/alignment.
 *
 * ouu_kernel_kl_project: the fused KL projection of Sec. 3.3's input reduction,
 *   xi[s][c] = bias[c] + sum_k bf16(m[s][k]) W[c][k],   s < N, c < rm, k < nn,
 * reading the FP64 fields m [N][nn] (device, 8-byte aligned, row-major) once; the
 * rounding to BF16 goes through FP32 (both to nearest even).  W: device BF16
 * [rm][ldw] (ldw a multiple of 8, >= nn).  bias: device FP32 [rm], added once per row.
 * xi: device FP32 [N][rm], overwritten; any 4-byte aligned address (partial sums are added
 * by atomics, 16-byte vector ones and TMA bulk reductions of whole rows when rm % 4 == 0 and
 * xi is 16-byte aligned).  rm <= 240.
 * err_dev as above.
 *
 * ouu_kernel_risk_weights: the per-sample risk weights of the SAA gradient (Sec. 2.1-2.2)
 * from the QoIs q_dev [N] (device FP64): for each of the n_risks (1..4) host descriptors,
 * w_dev[r][i] (device FP64, [n_risks][N]) with grad rho = sum_i w[r][i] grad Q_i, and on the
 * host out_host[3r + 0..2] = rho, d rho / dt, t (t = t* when t_optimal).  Mean + variance:
 * w = (1 + 2 kappa (Q_i - Qbar)) / N; smoothed CVaR: w = s'_eps(Q_i - t) / (N (1 - beta)).
 * With gq_dev (device FP32 per-sample gradients [N][ldg], dz columns used), also
 * grad_host[r][j] = sum_i w[r][i] gq[i][j] (FP64 sums), the SAA gradient of the risk.
 * Synchronises `stream`; allocates its own scratch (test entry only).
 *
 * ouu_kernel_dino_network: the MR-DINO evaluation network of Sec. 3.3 (layer-0 input
 * [xi; z] in BF16, three GELU layers, output layer phi with the reduced QoI
 * Q = 1/2 ||phi + c||^2 + const and, when gradq_dev is given, the reverse-mode
 * grad_z Q) from given projection coordinates xi_dev (device FP32 [n_samples][r_M]) instead
 * of from fields, in network mode `mode` (0 per-layer kernels, 1 one kernel per 128-sample
 * tile, 2 4-CTA clusters; see ouu_dino_set_fused_network), so that the modes can be
 * compared on identical inputs.  z_host: d_Z controls.  Outputs (device, each may be NULL):
 * q_dev [n_samples] FP64, phi_dev [n_samples][r_U] FP32, gradq_dev [n_samples][d_Z] FP64.
 * The handle's own network mode is restored; synchronises the handle's stream. */
#ifndef OUU_KERNELS_H
#define OUU_KERNELS_H

#include "ouu.h"

#ifdef __cplusplus
extern "C" {
#endif

ouu_status ouu_kernel_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                                float alpha, const float* bias, const float* aux, int ld_aux, int aux_rdiv,
                                float* out_f32, int ld_f32, int accumulate, void* out_bf16, int ld_bf16,
                                void* out_t_bf16, int ld_t, void* out2_bf16, int ld2, int* err_dev, void* stream);

ouu_status ouu_kernel_gemm_qoi_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                   const float* bias, const float* col_scale, const float* col_add, double qconst,
                                   float* out_f32, int ld_f32, void* out_bf16, int ld_bf16, double* out_q, int* err_dev,
                                   void* stream);

ouu_status ouu_kernel_risk_weights(const double* q_dev, int N, const ouu_risk_desc* risks, int n_risks, double* w_dev,
                                   double* out_host, const float* gq_dev, int ldg, int dz, double* grad_host,
                                   void* stream);

/* Number of GEMM shapes the tile autotuner has timed so far (ouu_batch_create with
 * autotune != 0 tunes the MR-DINO layer shapes). */
int ouu_kernel_gemm_tuned_shapes(void);

ouu_status ouu_kernel_kl_project(const double* m, int N, int nn, const void* W, int ldw, int rm, const float* bias,
                                 float* xi, int* err_dev, void* stream);

ouu_status ouu_kernel_dino_network(ouu_dino_t d, const float* xi_dev, int n_samples, const double* z_host, int mode,
                                   double* q_dev, float* phi_dev, double* gradq_dev);

#ifdef __cplusplus
}
#endif
#endif /* OUU_KERNELS_H */
