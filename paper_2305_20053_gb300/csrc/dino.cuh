// MR-DINO (reduced-basis derivative-informed neural operator, Sec. 3.3-3.4) handle.
#pragma once
#include <cuda_bf16.h>

#include "ouu_internal.cuh"
#include "tc_gemm.cuh"

#define DINO_LAYERS 4   // three GELU hidden layers + linear output

struct ouu_dino {
  ouu_dino_desc desc;
  cudaStream_t stream;
  int n, nn, nnp, dz, rm, ru, wd, in0, num_sms;
  int maxB, maxE, R, BR;
  double h;
  // parameters: flat FP32 [W0, b0, W1, b1, W2, b2, W3, b3], W_l row-major [out][in]
  int in_l[DINO_LAYERS], out_l[DINO_LAYERS], inp_l[DINO_LAYERS], outp_l[DINO_LAYERS];
  size_t offW[DINO_LAYERS], offb[DINO_LAYERS], n_params;
  float *d_params = nullptr, *d_grad = nullptr, *d_adam_m = nullptr, *d_adam_v = nullptr;
  int adam_t = 0;
  __nv_bfloat16* Wb[DINO_LAYERS] = {};    // [out][inp]
  __nv_bfloat16* WTb[DINO_LAYERS] = {};   // [in][outp]
  // bases
  int bases_ready = 0;
  float* d_phi = nullptr;          // [ru][nn] FP32, zero on the boundary
  double* d_phi64 = nullptr;       // [ru][nn] FP64
  double* d_ubar = nullptr;        // [nn]
  double* d_ut = nullptr;          // [nn] target state
  double* d_c = nullptr;           // [ru]  c = h^2 Phi^T (ubar - ut)
  float* d_cf = nullptr;           // [ru]  c in FP32 (the output layer's QoI epilogue)
  float* d_oscale = nullptr;       // [ru]  fixed output scale: phi = s * (W3 h3 + b3)
  // POD decode u_w = Phi phi + ubar as one GEMM over K = 3 rup with split BF16 operands:
  // [phi_hi | phi_hi | phi_lo] x [Phi_hi | Phi_lo | Phi_hi]^T
  __nv_bfloat16* d_dec_b = nullptr;   // [nn][3 rup]  the basis side
  __nv_bfloat16* d_dec_a = nullptr;   // [maxE][3 rup] the coefficient side of the current call
  float* d_ubarf = nullptr;        // [nn] ubar in FP32
  float* d_utf = nullptr;          // [nn] target state in FP32, zero on the boundary
  double* d_qdec = nullptr;        // [maxE] decoded QoIs when the caller passes none
  double qconst = 0.0;
  __nv_bfloat16* d_wkl = nullptr;  // [rm][nnp] KL projection rows
  int* d_kl_order = nullptr;       // [rm] flat mode index of each KL coordinate
  float* d_klbias = nullptr;       // [rm] -mbar * sum_p W_KL[k][p] (bias of the projection GEMM)
  // training buffers (batch <= maxB)
  __nv_bfloat16 *X0 = nullptr, *X0T = nullptr;
  float* A[4] = {};                // pre-activations a_1..a_3 (index 1..3) [maxB][wd]
  __nv_bfloat16* HS[4] = {};       // stacked [h_l; hdot_l]  [BR][wd]   (index 1..3)
  __nv_bfloat16* HST[4] = {};      // transposed [wd][BR]               (index 1..3)
  __nv_bfloat16* AD[4] = {};       // tangent pre-activations [R][wd]   (index 2..3)
  float* OUT = nullptr;            // [BR][ru]  stacked [phi; J^T]
  __nv_bfloat16 *GO = nullptr, *GOT = nullptr;   // [BR][ru], [ru][BR]
  float* GH = nullptr;             // [BR][wd]
  __nv_bfloat16 *GA = nullptr, *GAT = nullptr;   // [BR][wd], [wd][BR]
  float* GAv = nullptr;            // [maxB][wd]
  float* d_gov = nullptr;          // [maxB][ru] FP32 gradient of the loss w.r.t. phi
  __nv_bfloat16* GA1T = nullptr;   // [wd][maxB]
  double* d_loss_part = nullptr;   // [256]
  double* d_loss = nullptr;        // [2]
  // evaluation buffers (n_samples <= maxE)
  float* XIe = nullptr;            // [maxE][rm]
  __nv_bfloat16* X0e = nullptr;    // [maxE][in0p]
  float* Ae[4] = {};               // [maxE][wd] (index 1..3)
  __nv_bfloat16 *He0 = nullptr, *He1 = nullptr;   // ping-pong [maxE][wd]
  float* OUTe = nullptr;           // [maxE][ru]
  __nv_bfloat16* Ge = nullptr;     // [maxE][ru] seed phi + c
  float* GQe = nullptr;            // [maxE][dz]
  double* Qe = nullptr;            // [maxE]
  float* Qpart = nullptr;          // [maxE][4] per-CTA partial QoI sums of the cluster network
  double* Qmom = nullptr;          // [maxE / 128 + 1][2] per-tile sum Q, sum Q^2 of the cluster network
  float* d_zf = nullptr;           // [max(maxB, 1) * dz] FP32 controls of the current call
  double* h_pin = nullptr;         // pinned host scratch
  const float* h_pin_dev = nullptr;   // h_pin as the device addresses it (mapped), or null
  int* d_err = nullptr;
  int* d_klp_ctr = nullptr;        // [OUU_KLP_MAX_TILES] tile counters of the KL projection
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // cast | projection | network phase marks
  // CUDA graph of the risk evaluation (captured on a private stream, replayed on `stream`)
  cudaStream_t cap = nullptr;
  // second stream of a risk evaluation: the risk selection on Q runs there beside the
  // network's reverse mode (forked after the forward part, joined before the weighted sums)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool graph_marks = false;        // the captured risk graph records ev[0] / ev[2] around the projection
  cudaGraphExec_t gexec = nullptr;
  const void* gkey_p = nullptr;
  const double* gkey_m = nullptr;
  int gkey_N = 0, gkey_nr = 0;
  int use_graphs = 1;
  int fused_mlp = 2;               // evaluation network: 0 per-layer kernels, 1 one kernel per
                                   // 128-sample tile (mlp_fused.cu), 2 one kernel over 4-CTA
                                   // clusters (mlp_cluster.cu); 1 and 2 when the sizes fit
  bool capturing = false;
  uint64_t eval_count = 0;         // evaluations so far (a pending ouu_shard_qoi names the one it ran)
  int jac_route = 0;               // Jacobian data: 0 the cheaper of the two, 1 forward, 2 adjoint
  // held-out check against the plain path (ouu_dino_validate): passed for the problem with this
  // serial; cleared whenever parameters, bases or output scale change
  int val_ok = 0;
  uint64_t val_serial = 0;
};

// The network d may stand in for the plain path on n_samples samples of problem p: it passed
// its held-out check against p since it last changed (capi.cu; OUU_BACKEND_AUTO).
bool dino_trusted(const ouu_dino* d, const ouu_problem* p, int n_samples);

// DINO forward/backward pieces used by the C ABI (dino.cu).
ouu_status dino_eval_core(ouu_dino* d, const double* m_dev, int N, const double* z_host, bool want_grad);
// dino_eval_core with the gradient, in two parts on d->stream: dino_eval_forward enqueues the
// projection and the network up to the reduced QoI (Qe is complete once its work is), and
// dino_eval_reverse the reverse mode (GQe).  *split = false: the network runs as one launch
// (another network mode, or sizes beyond the cluster kernel) and the forward call enqueued
// all of it; dino_eval_reverse is then not called.
ouu_status dino_eval_forward(ouu_dino* d, const double* m_dev, int N, const double* z_host, bool* split);
ouu_status dino_eval_reverse(ouu_dino* d, int N);
// Decoded states u[N][nn] (FP32) = Phi phi_i + ubar from the coefficients phi [N][ldphi] (FP32),
// and the decoded QoI q[N] = 1/2 h^2 sum over the interior (u - u_t)^2 (FP64), on d->stream.
ouu_status dino_decode(ouu_dino* d, const float* phi, int ldphi, int N, float* u, double* q);

// The evaluation network in one fused kernel per 128-sample tile (mlp_fused.cu): layer-0
// input from XIe and d_zf, forward with GELU (gelu' to Ae), reduced QoI (Qe, OUTe), reverse
// mode to GQe.  mlp_fused_fits: the handle's sizes fit the kernel (width, r_u, d_Z <= 416).
bool mlp_fused_fits(const ouu_dino* d);
ouu_status mlp_fused_eval(ouu_dino* d, int N);
// The same network with each 128-sample tile on a cluster of 4 CTAs, each CTA computing a
// quarter of every layer's columns; the layers' activations pass through the handle's
// evaluation buffers in L2 (mlp_cluster.cu).  mlp_cluster_fits: width, r_U, r_M + d_Z <= 448,
// d_Z <= 512, r_M % 4 == 0, width % 8 == 0.
// The layers [l0, l1) of the eight (three GELU layers and the QoI layer forward, four reverse):
// [0, 8) in one launch, or [0, 4) and [4, 8) as two.
bool mlp_cluster_fits(const ouu_dino* d);
ouu_status mlp_cluster_eval(ouu_dino* d, int N, int l0 = 0, int l1 = 8);

// The whole MR-DINO risk evaluation enqueued on d->stream (capi.cu); the problem's risk
// descriptors must be in p->d_risks.
ouu_status dino_enqueue_risk(ouu_problem* p, ouu_dino* d, const double* m_dev, int n_samples, int n_risks,
                             const double* z_host);
// Completes a basis whose FP64 Phi and ubar are in place (FP32 copy, reduced-QoI terms).
ouu_status dino_install_bases(ouu_dino* d);
// Sum_i w[r][i] grad_z Q_i of the last evaluation into out [n_w][d_Z] (device).
// Jacobian-data solves (pde.cu): jy[i][j][r] = h^2 Phi_r . J(u_i)^-1 g_j.
// Fused KL projection of FP64 fields (kl_project.cu): xi[N][rm] = bf16(m) W^T + bias with
// W = [rm][ldw] BF16 (K = nn contiguous); xi is zeroed here.  m 8-byte aligned, rm <= 240.
// ctr: device scratch of OUU_KLP_MAX_TILES + 1 ints, zero before the first call (the per-tile
// unit counters and an arrival count; each launch leaves them zero); N above
// OUU_KLP_MAX_TILES * 128 runs as several launches.
#define OUU_KLP_MAX_TILES 512
// zsrc / zdst / nz: the launch also copies nz floats from zsrc (device-addressable, e.g. mapped
// pinned host memory) to zdst, for work that follows it in the stream (the network's controls).
ouu_status ouu_kl_project(const double* m, int N, int nn, const __nv_bfloat16* W, int ldw, int rm, const float* bias,
                          float* xi, int* err, int* ctr, int num_sms, cudaStream_t s, const float* zsrc = nullptr,
                          float* zdst = nullptr, int nz = 0);

// route 0: forward (d_Z solves per sample), 1: adjoint (r_u solves per sample).
void launch_pde_jacobian_data(const PdeArgs& a, int nslots, const float* phi, int ru, float* jy, int route,
                              cudaStream_t s);
