/* ouu.h -- C ABI of the GB300 (sm_103a) SAA risk + gradient library for
 * PDE-constrained optimisation under uncertainty (arXiv 2305.20053, Luo,
 * O'Leary-Roseberry, Chen, Ghattas).
 *
 * Problem (Sec. 2, Eq. for min_z rho(Q)(z) + P(z)): the state u(m, z) solves the
 * semilinear elliptic equation of Sec. 4.2,
 *      -div(e^m grad u) + r u^3 = sum_j z_j f_j   on (0,1)^2,  u = 0 on the boundary,
 * with m a Matern Gaussian random field (Sec. 2, C = (-gamma Lap + delta I)^-2),
 * f_j Gaussian sources on an L x L lattice (Sec. 4.2), and the tracking QoI
 * Q(u) = 1/2 ||u - sin(pi x) sin(pi y)||^2_{L2} (Sec. 4.2, with a factor 1/2).
 * The risk of Q over N fixed samples of m is the sample average approximation of
 * Sec. 2.2 (mean + kappa * variance, or the smoothed CVaR of Sec. 2.1 in its
 * Rockafellar-Uryasev form), and its gradient in z is the chain rule of Sec. 2.3
 * with one adjoint solve per sample (plain backend) or automatic differentiation
 * through the reduced-basis neural operator of Sec. 3.3 (MR-DINO backend); the AUTO backend
 * takes the surrogate only after it passed a held-out check against the plain backend.
 *
 * Discretisation: n x n vertex grid, h = 1/(n-1), n = 2^k + 1 (5 <= n <= 1025);
 * grid arrays are row-major [iy * n + ix] over all n*n nodes (x fastest);
 * controls are indexed j = jy * L + jx (x fastest).
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers allocated by the caller, who owns
 *    them; they must stay valid until the work queued on the problem's stream has
 *    completed.  Pointers named *_host / *_out are host memory.
 *  - All device work is ordered on the CUDA stream given at creation.  Calls that
 *    return host results synchronise that stream before returning.
 *  - The library allocates its workspaces at creation (ouu_create_problem,
 *    ouu_dino_create); the per-call paths allocate nothing.
 *  - Every call returns an ouu_status; on failure, ouu_last_error() gives a
 *    message for the calling thread.  Calls on one handle are not re-entrant;
 *    distinct handles may be used concurrently on distinct streams.
 */
#ifndef OUU_H
#define OUU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OUU_OK = 0,
  OUU_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported grid */
  OUU_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  OUU_ERR_OOM = 3,           /* workspace allocation at creation failed */
  OUU_ERR_NOT_CONVERGED = 4, /* some sample hit newton_maxit (per-sample status set) */
  OUU_ERR_NONFINITE = 5,     /* NaN/Inf met in a residual or input */
  OUU_ERR_STATE = 6          /* handle not ready for this call (e.g. DINO bases not built) */
} ouu_status;

typedef enum { OUU_RISK_MEAN_VAR = 0, OUU_RISK_CVAR_SMOOTH = 1 } ouu_risk_kind;
/* OUU_BACKEND_AUTO: the MR-DINO surrogate when it passed its held-out check against the plain
 * path for this problem (ouu_dino_validate), else the plain path. */
typedef enum { OUU_BACKEND_PDE = 0, OUU_BACKEND_DINO = 1, OUU_BACKEND_AUTO = 2 } ouu_backend;

/* Per-sample status words written by the solve calls. */
enum { OUU_SAMPLE_OK = 0, OUU_SAMPLE_NOT_CONVERGED = 1, OUU_SAMPLE_NONFINITE = 2 };

typedef struct {
  int n;               /* nodes per side, 2^k + 1 */
  double reaction_r;   /* r in the state equation (Sec. 4.2) */
  double gamma, delta; /* prior operator -gamma Lap + delta I (Sec. 2) */
  double m_mean;       /* constant prior mean mbar */
  int lattice_L;       /* L x L sources, d_Z = L^2 */
  double bump_width;   /* source width sigma (Sec. 4.2) */
  double newton_rtol;  /* stop when ||R||_2 <= rtol ||f||_2, then one more step */
  int newton_maxit;
  double cg_rtol;      /* relative residual of each inner MG-PCG solve (FP32) */
  int cg_maxit;
  int max_samples;     /* capacity: largest n_samples of any later call */
} ouu_problem_desc;

typedef struct {
  ouu_risk_kind kind;
  double kappa;        /* mean + kappa * variance */
  double beta, eps;    /* smoothed CVaR level and smoothing width (Sec. 2.1) */
  double t;            /* CVaR auxiliary variable when t_optimal == 0 */
  int t_optimal;       /* 1: t = argmin_t rho(z, t) (bisection on d rho / dt) */
} ouu_risk_desc;

typedef struct {
  int newton_min, newton_max;   /* Newton steps over samples (state solve) */
  double newton_mean;
  int cg_total;                 /* inner CG iterations summed over samples and solves */
  int adjoint_solves;           /* adjoint solves performed (samples with nonzero weight) */
  int n_not_converged;
  float ms_state;               /* PDE: batched state solve; DINO: projection + network (CUDA events) */
  float ms_weights;             /* risk weights / t*; DINO: the weighted pass (t* runs beside the
                                   network's reverse mode, inside ms_network) */
  float ms_adjoint;             /* batched adjoint solve */
  float ms_reduce;              /* weighted adjoint sum and G^T */
  float ms_total;               /* whole evaluation on the device */
  float ms_project;             /* DINO: fused KL projection of the FP64 fields (also measured in a
                                   replayed evaluation, by event nodes of its graph) */
  float ms_network;             /* DINO: network forward + reverse-mode gradient */
} ouu_eval_stats;

typedef struct ouu_problem* ouu_problem_t;
typedef struct ouu_dino* ouu_dino_t;

/* Fills *desc with the defaults of the 129 x 129 workload: r = 1, gamma = 0.1,
 * delta = 1, mbar = 0, L = 10, sigma = 0.05, newton_rtol = 1e-10, newton_maxit = 30,
 * cg_rtol = 1e-6, cg_maxit = 200, max_samples = 4096. */
void ouu_default_problem_desc(ouu_problem_desc* desc);

/* Creates a problem handle bound to `cuda_stream` (a cudaStream_t, or NULL for the
 * legacy default stream) on the current device and allocates its workspace for
 * up to desc->max_samples samples.  Errors: INVALID_ARG (grid not 2^k+1 with
 * 5 <= n <= 1025, L outside [1, 64], widths <= 0, L * n * 8 bytes above the device's
 * shared memory per block), OOM, CUDA. */
ouu_status ouu_create_problem(const ouu_problem_desc* desc, void* cuda_stream, ouu_problem_t* out);
ouu_status ouu_destroy_problem(ouu_problem_t p);

/* Draws the Gaussian random fields of samples first_index .. first_index+n_samples-1
 * (Sec. 2: m ~ N(mbar, (-gamma Lap + delta I)^-2), homogeneous Neumann) by their
 * Karhunen-Loeve expansion (Sec. 3.3) in the DCT-II eigenbasis of the discrete
 * Neumann Laplacian: m = mbar + n sum_{k1,k2} lambda^-1 xi v_k1(ix) v_k2(iy),
 * lambda = delta + gamma (mu_k1 + mu_k2), mu_k = 4 n^2 sin^2(pi k / 2n).
 * The standard normals xi come from Philox4x32-10 (key = seed, counter =
 * (mode pair, sample index, tag)) and Box-Muller, so any subset of samples is
 * reproducible.  Output m_dev: [n_samples][n][n] float64, device.  FP64. */
ouu_status ouu_sample_fields(ouu_problem_t p, uint64_t seed, int64_t first_index, int n_samples,
                             double* m_dev);

/* Solves the state equation (Sec. 4.2) for each sample by Newton's method with an
 * FP64 residual and geometric-multigrid-preconditioned CG (FP32) for each Newton
 * step, and evaluates the QoI.  m_dev: [n_samples][n][n] fields; z_dev: controls,
 * sample i uses z_dev + i * z_stride (z_stride = 0: one shared control of d_Z
 * entries).  Outputs (device): u_dev [n_samples][n][n] (boundary zero), q_dev
 * [n_samples], status_dev [n_samples] (OUU_SAMPLE_*).  u_dev may be NULL when the
 * states are not needed.  Returns NOT_CONVERGED / NONFINITE if any sample failed. */
ouu_status ouu_pde_solve_batch(ouu_problem_t p, const double* m_dev, int n_samples, const double* z_dev,
                               int64_t z_stride, double* u_dev, double* q_dev, int32_t* status_dev);

/* Adjoint solves (Sec. 2.3): J(u_i) lambda_i = dQ/du(u_i) = h^2 (u_i - u_t) with
 * J = A_h(m_i) + 3 r diag(u_i^2) (symmetric), by FP32 MG-PCG inside FP64
 * iterative refinement to a relative residual of 1e-12, and the per-sample
 * gradient grad_z Q_i = G^T lambda_i (G: the source matrix, since dR/dz = -G).
 * Inputs: m_dev, u_dev (states from ouu_pde_solve_batch).  Outputs (device, each
 * may be NULL): lambda_dev [n_samples][n][n], gradq_dev [n_samples][d_Z]. */
ouu_status ouu_adjoint_batch(ouu_problem_t p, const double* m_dev, const double* u_dev, int n_samples,
                             double* lambda_dev, double* gradq_dev);

/* Risk measure and its gradient over the sample average of Sec. 2.2 at the
 * control z_host[d_Z] for the n_samples fields in m_dev, for n_risks risk measures
 * at once (1 <= n_risks <= 4).  Backend PDE: one batched state solve, the risk
 * weights, then one adjoint solve per sample whose weight is nonzero in some
 * risk, accumulating sum_i w_i lambda_i and applying G^T once.  Backend DINO:
 * the MR-DINO surrogate (`dino` must be non-NULL and trained), see
 * ouu_dino_eval.  Backend AUTO: DINO when `dino` passed ouu_dino_validate against this
 * problem since its last change and can take n_samples, else PDE (ouu_last_backend tells
 * which ran).  Outputs (host): risk_out[n_risks], grad_z_out[n_risks][d_Z],
 * grad_t_out[n_risks] (d rho / dt for CVaR, 0 for mean+var), t_out[n_risks]
 * (t used; may be NULL), stats (may be NULL).  Synchronises the stream. */
ouu_status ouu_risk_and_grad(ouu_problem_t p, ouu_backend backend, ouu_dino_t dino, const double* m_dev,
                             int n_samples, const ouu_risk_desc* risks, int n_risks, const double* z_host,
                             double* risk_out, double* grad_z_out, double* grad_t_out, double* t_out,
                             ouu_eval_stats* stats);

/* Backend of the last ouu_risk_and_grad on p that returned OUU_OK (OUU_BACKEND_PDE or
 * OUU_BACKEND_DINO); -1 before any, or for p == NULL. */
int ouu_last_backend(ouu_problem_t p);

/* Held-out check of the surrogate with the plain path as the reference (the paper's accuracy
 * study of Sec. 4 as a gate): at each of the n_z controls z_host [n_z][d_Z], both backends
 * evaluate the n_risks risks over the held-out fields m_dev [n_samples][n][n] (samples not
 * used for training); the largest relative risk error |rho_DINO - rho_PDE| / |rho_PDE| and
 * the largest relative gradient error ||g_DINO - g_PDE|| / ||g_PDE|| over controls and risks
 * go to risk_err_out / grad_err_out (host, nullable).  The network passes when they are
 * <= risk_tol and <= grad_tol (passed_out, nullable: 1 or 0); OUU_BACKEND_AUTO then uses it
 * for this problem until its parameters, bases or output scale change or it takes a training
 * step.  A failed check, or an error part-way, leaves it unused by AUTO.  Errors as
 * ouu_risk_and_grad; INVALID_ARG for n_z < 1 or a negative or non-finite tolerance. */
ouu_status ouu_dino_validate(ouu_problem_t p, ouu_dino_t d, const double* m_dev, int n_samples,
                             const ouu_risk_desc* risks, int n_risks, const double* z_host, int n_z,
                             double risk_tol, double grad_tol, double* risk_err_out, double* grad_err_out,
                             int* passed_out);

/* ---------------------------------------------------------------------------------------
 * One sample average spread over ranks (one process per GPU).  Sec. 2.2 defines the risk over
 * ONE fixed sample set and Sec. 2.3 its gradient as ONE weighted sum over it; rank k holds the
 * contiguous block [first_k, first_k + n_k) of the n_total samples.  The weights need the
 * mean and, for CVaR, t* of ALL the QoIs, so one evaluation takes two exchanges, both done by
 * the caller (e.g. NCCL through torch.distributed):
 *   1. ouu_shard_qoi on every rank: the QoIs of its block, q_local_dev [n_k] (device FP64);
 *   2. all-gather: q_all_dev [n_total] = the ranks' q_local in rank order (8 n_total bytes);
 *   3. ouu_shard_risk_partial on every rank: risk values, d rho / dt and t from all QoIs
 *      (the same on every rank), and this rank's gradient part
 *      grad_part_out[r][j] = sum over its samples of w_r,i (grad_z Q_i)_j;
 *   4. all-reduce (sum, FP64) of grad_part_out over ranks: grad_z rho (n_risks * d_Z values).
 * With one rank (n_total = n_k, first = 0) this gives ouu_risk_and_grad's results up to the
 * order of the final sums. */

/* Phase 1: the QoIs of this rank's n_local fields m_dev [n_local][n][n] at z_host [d_Z]
 * (backend PDE: Newton state solves, kept in the problem's workspace for phase 2; DINO: the
 * network with its reverse-mode gradients, kept in the network's buffers; AUTO as in
 * ouu_risk_and_grad).  Output q_local_dev [n_local] (device FP64).  Synchronises.  Errors as
 * ouu_risk_and_grad. */
ouu_status ouu_shard_qoi(ouu_problem_t p, ouu_backend backend, ouu_dino_t dino, const double* m_dev, int n_local,
                         const double* z_host, double* q_local_dev);
/* Phase 2, after the all-gather: q_all_dev [n_total] (device FP64) holds every rank's QoIs and
 * this rank's block starts at first_local.  Outputs (host): risk_out[n_risks],
 * grad_part_out[n_risks][d_Z] (this rank's part of the gradient; the plain backend solves the
 * adjoints of its samples with a nonzero weight here), grad_t_out[n_risks], t_out[n_risks]
 * (nullable).  `dino` must be the network of the pending phase 1 (NULL for the plain path).
 * Errors: STATE without a pending ouu_shard_qoi on p (each phase 1 serves one phase 2), or
 * when the network has evaluated other samples since (its buffers hold the per-sample
 * gradients of phase 1: every rank needs its own network handle); INVALID_ARG for a block
 * outside [0, n_total). */
ouu_status ouu_shard_risk_partial(ouu_problem_t p, ouu_dino_t dino, const double* q_all_dev, int n_total,
                                  int64_t first_local, const ouu_risk_desc* risks, int n_risks, double* risk_out,
                                  double* grad_part_out, double* grad_t_out, double* t_out);

/* Allocation-free variant of ouu_pde_solve_batch.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they call in -- code under a device-memory budget or pool that forbids new
 * cudaMalloc calls, or a plug-in handed a stream and buffers by a host
 * application that owns every device allocation -- and that therefore cannot
 * create a problem handle (ouu_create_problem allocates its workspace).
 * It runs the same per-sample Newton / MG-PCG state solve and QoI as
 * ouu_pde_solve_batch, with the same results, for the problem described by
 * *desc (desc->max_samples is ignored); m_dev, z_dev, z_stride, u_dev, q_dev and
 * status_dev mean what they mean there, and all five pointers are required.
 * All scratch (tables, per-CTA solver slots, the work counter) lives in one
 * file-scope device array of 8 MiB that every GPU which loads the library holds
 * until the process exits; under lazy module loading (CUDA_MODULE_LOADING=LAZY, the
 * default) the array may be committed only when the library's module is first used
 * on that device, which can be this call.  Grids that do not fit one solver slot in
 * it (n > 257) are rejected with OUU_ERR_INVALID_ARG.  Throughput: the array holds
 * a few solver slots only (about 9 at n = 129, 2 at n = 257, one slot per CTA), so
 * the solve runs on that many SMs rather than all of them; ouu_pde_solve_batch
 * is the fast path.  The call makes no cudaMalloc, cudaFree or other allocating
 * call.  Every call looks up the array's device address (cudaGetSymbolAddress,
 * which allocates nothing) with the calling thread's current device; make the
 * first call on a device before any stream capture.  The array keeps the last
 * call's contents; each call clears what must start at zero.  All calls share the
 * one array, so calls whose GPU work overlaps (other streams, other threads) race:
 * serialise them.  Synchronises `cuda_stream` (a cudaStream_t or NULL) before
 * returning, like ouu_pde_solve_batch. */
ouu_status ouu_pde_solve_batch_noalloc(const ouu_problem_desc* desc, const double* m_dev, int n_samples,
                                       const double* z_dev, int64_t z_stride, double* u_dev, double* q_dev,
                                       int32_t* status_dev, void* cuda_stream);

/* ------------------------------------------------------------------ MR-DINO
 * Reduced-basis neural operator of Sec. 3.3: u_w(m, z) = Phi phi_w(m_r, z) + ubar,
 * m_r the whitened coordinates of m on the r_m leading Karhunen-Loeve modes of
 * the prior (Sec. 3.3, KLE; mode order: decreasing prior variance, ties by
 * (k1 + k2, k1)), Phi the r_u leading modes of the mass-weighted POD of training
 * states (Sec. 3.3, M = h^2 I on interior nodes, Phi^T M Phi = I), phi_w a dense
 * net [m_r; z] -> width -> width -> width -> r_u with GELU x Phi(x) (Phi by Abramowitz &
 * Stegun 26.2.17, within 5e-7 of the exact function) and a linear
 * output layer.  The control Jacobian d_z phi_w is carried in forward mode
 * (Sec. 3.2); training minimises the reduced-space DINO loss of Sec. 3.4,
 *   (1/B) sum_i ||phi_i - y_i||^2 + jac_weight ||d_z phi_i - Y_i||_F^2,
 * y_i = Phi^T M (u_i - ubar), Y_i = Phi^T M d_z u_i, by Adam (beta = 0.9, 0.999,
 * eps = 1e-8).  GEMMs run on the tcgen05 tensor cores in BF16 with FP32
 * accumulation; FP32 master weights and Adam moments.
 *
 * Parameter vector (FP32, flat): [W0, b0, W1, b1, W2, b2, W3, b3], W_l row-major
 * [out][in]; W0 is width x (r_m + d_Z) with the KL inputs first, W3 is r_u x width.
 * The output is phi = s * (W3 h3 + b3) with the fixed scale s of
 * ouu_dino_set_output_scale. */
typedef struct {
  int n;              /* grid of the states (nodes per side), 2^k + 1 */
  int lattice_L;      /* d_Z = L^2 controls */
  int r_m, r_u;       /* reduced ranks of m (KL, <= 240) and u (POD, <= 256) */
  int width;          /* hidden width (three hidden layers), multiple of 8 */
  int max_batch;      /* largest training batch (also the Jacobian chunk of ouu_dino_eval) */
  int max_eval;       /* largest n_samples of an evaluation */
  double gamma, delta, m_mean;   /* prior of m (defines the KL basis) */
  double jac_weight;  /* weight of the Jacobian loss term: 1 = MR-DINO, 0 = MR-NO */
} ouu_dino_desc;

/* Defaults of the 129 x 129 workload: L = 10, r_m = r_u = 200, width 400,
 * max_batch 256, max_eval 4096, gamma 0.1, delta 1, mbar 0, jac_weight 1. */
void ouu_default_dino_desc(ouu_dino_desc* desc);

/* Allocates the network, its Adam state and all work buffers on the current
 * device; parameters start at zero (set them with ouu_dino_set_params).  Builds
 * the KL projection rows for the prior in *desc. */
ouu_status ouu_dino_create(const ouu_dino_desc* desc, void* cuda_stream, ouu_dino_t* out);
ouu_status ouu_dino_destroy(ouu_dino_t d);
/* Number of FP32 entries of the flat parameter vector. */
size_t ouu_dino_num_params(ouu_dino_t d);
/* Copies the parameters in (host FP32, n = ouu_dino_num_params) and resets Adam. */
ouu_status ouu_dino_set_params(ouu_dino_t d, const float* params_host, size_t n);
ouu_status ouu_dino_get_params(ouu_dino_t d, float* params_host, size_t n);

/* Installs the POD basis: phi_dev [r_u][n*n] (zero on the boundary) and
 * ubar_dev [n*n], both FP64 device.  Also forms c = Phi^T M (ubar - u_t) and the
 * constant of the reduced QoI (Sec. 3.3: Q(u_w) = 1/2 ||phi + c||^2 + const). */
ouu_status ouu_dino_set_bases(ouu_dino_t d, const double* phi_dev, const double* ubar_dev);
/* Builds the basis from n_states training states u_dev [n_states][n][n] (FP64
 * device): ubar = mean, snapshot Gram C = (U - ubar) M (U - ubar)^T (FP64), its
 * eigenpairs by cyclic parallel Jacobi (FP64), Phi = (U - ubar)^T V Lambda^-1/2
 * for the r_u largest eigenvalues, each mode's largest-magnitude entry positive.
 * eig_host (nullable): the n_states eigenvalues, descending.  Then as set_bases. */
ouu_status ouu_dino_build_bases(ouu_dino_t d, const double* u_dev, int n_states, double* eig_host);
/* Fixed per-mode output scale s (host FP32 [r_u], positive): the network output is
 * phi = s * (W3 h3 + b3), a reparametrisation that lets every reduced coordinate
 * be learned at unit scale (the loss is unchanged).  Starts at 1;
 * ouu_dino_build_bases sets s_k = sqrt(lambda_k / n_states), the RMS of mode k. */
ouu_status ouu_dino_set_output_scale(ouu_dino_t d, const float* s_host);
ouu_status ouu_dino_get_output_scale(ouu_dino_t d, float* s_host);
/* Copies the installed basis out (FP64 device, layouts as in set_bases). */
ouu_status ouu_dino_get_bases(ouu_dino_t d, double* phi_dev, double* ubar_dev);

/* Checkpoint of the whole network state to the file at `path`: FP32 parameters, the Adam
 * moments and step count (so that training resumes where it stopped), the output scale,
 * and the POD basis with its mean state when built.  Format: the 8 bytes "OUUDINO1", a
 * 64-byte header (int32 version = 1, n, lattice_L, r_m, r_u, width, Adam step, bases flag;
 * double gamma, delta, m_mean; uint64 parameter count), then the arrays in that order,
 * little-endian.  ouu_dino_load restores it into a handle created with the same sizes and
 * prior (the KL rows are rebuilt at creation) and refuses another network's file, a
 * truncated file or one with bytes after its last array (INVALID_ARG, message set). */
ouu_status ouu_dino_save(ouu_dino_t d, const char* path);
ouu_status ouu_dino_load(ouu_dino_t d, const char* path);

/* Network inputs: xi_dev [n][r_m] FP32 = whitened KL coordinates of m_dev
 * [n][n*n] (BF16 tensor-core projection, FP32 accumulation). */
ouu_status ouu_dino_project_fields(ouu_dino_t d, const double* m_dev, int n_samples, float* xi_dev);
/* Output targets: y_dev [n][r_u] FP32 = Phi^T M (u_i - ubar) (FP32). */
ouu_status ouu_dino_project_states(ouu_dino_t d, const double* u_dev, int n_samples, float* y_dev);
/* Jacobian targets (Sec. 3.4, implicit function theorem): jy_dev [n][d_Z][r_u] FP32,
 * jy[i][j] = Phi^T M J(u_i)^-1 g_j, by min(d_Z, r_u) linearised solves per sample sharing
 * one operator set-up (MG-PCG, FP32, relative residual cg_rtol of `p`): the forward route
 * solves J x = g_j for each control j and projects on the POD modes; the adjoint route
 * (d_Z > r_u) solves J lam_r = M Phi_r for each mode r (J is symmetric) and takes
 * g_j . lam_r.  u_dev: states of (m_dev, z_i). */
ouu_status ouu_dino_jacobian_data(ouu_problem_t p, ouu_dino_t d, const double* m_dev, const double* u_dev,
                                  int n_samples, float* jy_dev);
/* Route of ouu_dino_jacobian_data: 0 (default) the one with fewer solves, 1 forward, 2 adjoint.
 * Errors: INVALID_ARG for another value. */
ouu_status ouu_dino_set_jacobian_route(ouu_dino_t d, int route);

/* One Adam step on the minibatch idx_dev[0..batch-1] (device int32 indices into
 * the data arrays): xi_dev [*][r_m], z_dev [*][d_Z], y_dev [*][r_u],
 * jy_dev [*][d_Z][r_u] (all FP32 device).  loss_out (host, nullable): the loss
 * of this batch before the step (synchronises when given). */
ouu_status ouu_dino_train_step(ouu_dino_t d, const float* xi_dev, const float* z_dev, const float* y_dev,
                               const float* jy_dev, const int32_t* idx_dev, int batch, float lr, double* loss_out);
/* Loss and its gradient (host FP32, flat parameter layout) on a minibatch, no update. */
ouu_status ouu_dino_loss_grad(ouu_dino_t d, const float* xi_dev, const float* z_dev, const float* y_dev,
                              const float* jy_dev, const int32_t* idx_dev, int batch, float* grad_host,
                              double* loss_out);

/* Surrogate evaluation at the shared control z_host[d_Z] for the fields m_dev
 * [n_samples][n][n]: KL projection, network, reduced QoI.  Outputs (device, each
 * nullable): phi_dev [n][r_u] FP32, jphi_dev [n][d_Z][r_u] FP32 (forward-mode
 * d_z phi), q_dev [n] FP64 (Q(u_w) by the reduced form), gradq_dev [n][d_Z]
 * FP64 (grad_z Q by reverse mode through the network), u_dev [n][n][n] FP32 (the
 * decoded states u_w = Phi phi + ubar of Sec. 3.3, as ouu_dino_decode).  Synchronises. */
ouu_status ouu_dino_eval(ouu_dino_t d, const double* m_dev, int n_samples, const double* z_host, float* phi_dev,
                         float* jphi_dev, double* q_dev, double* gradq_dev, float* u_dev);

/* POD decode of Sec. 3.3: u_w = Phi phi + ubar for the reduced coefficients phi_dev
 * [n_samples][r_u] (FP32 device, e.g. ouu_dino_eval's phi_dev) into u_dev [n_samples][n][n]
 * (FP32 device; zero on the boundary), and the QoI of the decoded states,
 * q_dev[i] = 1/2 h^2 sum over the interior of (u_w - u_t)^2 (FP64 device, nullable), which
 * equals the reduced form 1/2 ||phi + c||^2 + const of ouu_dino_eval up to rounding.  One
 * tensor-core GEMM (K = 3 r_u: phi and Phi each split into two BF16 parts, three of the four
 * cross products kept, FP32 accumulation, about 16 significant bits) with the sum of squares
 * fused into its epilogue.  Synchronises.  Errors: STATE before the bases are installed,
 * INVALID_ARG for n_samples outside [1, max_eval]. */
ouu_status ouu_dino_decode(ouu_dino_t d, const float* phi_dev, int n_samples, float* u_dev, double* q_dev);

/* DINO risk evaluations in ouu_risk_and_grad are replayed from a CUDA graph that is
 * captured (on a private stream, after one eager evaluation) for each new combination
 * of (problem, m_dev, n_samples, n_risks); enable = 0 turns this off (every call then
 * enqueues its kernels eagerly and reports per-phase times in ouu_eval_stats; a replayed
 * evaluation in network mode 2 reports ms_total and ms_project).  The controls of a call
 * travel through the network's pinned host buffer, which the captured graph reads when it
 * runs: calls on one network do not overlap (each synchronises before returning). */
ouu_status ouu_dino_set_graphs(ouu_dino_t d, int enable);

/* How the evaluation network with a gradient (projection output -> forward layers -> reduced
 * QoI -> reverse-mode z-gradient) runs; every mode has the same arithmetic.
 *   mode 0: one tensor-core GEMM kernel per layer, fused epilogues;
 *   mode 1: one kernel, one CTA per 128-sample tile holding the activations in shared memory
 *           (width, r_U, d_Z <= 416, r_M + d_Z <= 448, r_M % 4 == 0); the GELU epilogues of a
 *           layer then run on one SM per tile, slower than mode 0 at thousands of samples;
 *   mode 2 (default): one kernel, each 128-sample tile on a cluster of 4 CTAs, each computing a quarter of
 *           every layer's columns, activations passed through L2 (width, r_U, r_M + d_Z <= 448,
 *           d_Z <= 512, r_M % 4 == 0, width % 8 == 0).  In ouu_risk_and_grad it runs as two
 *           launches (forward with the reduced QoI, then reverse mode), with the risk's t*
 *           search beside the second on another branch of the evaluation's graph.
 * A mode whose size limits the network exceeds falls back to mode 0.  ouu_batch_create with
 * autotune picks per network by timing.  Returns OUU_ERR_INVALID_ARG for another mode. */
ouu_status ouu_dino_set_fused_network(ouu_dino_t d, int mode);

/* Thread-local message of the last failed call ("" if none).  Copies at most
 * len-1 bytes plus a terminating zero into buf; returns the full length. */
size_t ouu_last_error(char* buf, size_t len);

/* Number of samples one persistent launch keeps in flight (one per CTA). */
int ouu_problem_slots(ouu_problem_t p);

/* ---------------------------------------------------------------------------------------
 * Uneven batches: many OUU problems (different grids, sample counts, control counts,
 * risks, plain or MR-DINO backend) evaluated together, the risk and z-gradient of each at
 * its own z (Sec. 2.1-2.3 per problem).  The paper evaluates one problem at a time; this
 * is a throughput interface for many concurrent problems.
 *
 * Execution, captured once into one CUDA graph and replayed by later runs:
 *   - the state solves of every sample of every plain problem in ONE persistent launch
 *     (tasks (problem, sample), largest grids first, pulled by one CTA per SM), then each
 *     problem's risk weights, then the adjoint solves in one persistent launch, then each
 *     problem's G^T sum;
 *   - each MR-DINO problem's evaluation on a concurrent branch of the graph.
 * With autotune != 0, ouu_batch_create times every MR-DINO problem's evaluation with the
 * per-layer GEMM kernels (their N tiles tuned per layer shape by measurement) and with the
 * one-kernel networks, and keeps the fastest for that network (ouu_dino_set_fused_network).
 *
 * Each item names its own problem handle and, for MR-DINO, its own network (items must
 * not share either: the handle's arena holds the item's results, the network's buffers
 * its evaluation), its fields m_dev [n_samples][n][n] (device, caller-owned,
 * unchanged between runs) and 1..4 risk descriptors; MR-DINO items name a network built
 * for the same grid and controls with max_eval >= n_samples.  The batch runs on the
 * stream of the first item's problem. */
typedef struct ouu_batch* ouu_batch_t;

typedef struct {
  ouu_problem_t problem;
  ouu_backend backend;
  ouu_dino_t dino;              /* OUU_BACKEND_DINO and _AUTO items, else NULL; an AUTO item
                                 * takes DINO at create when the network passed its held-out
                                 * check for the item's problem, else PDE */
  const double* m_dev;
  int n_samples;
  const ouu_risk_desc* risks;   /* copied at create */
  int n_risks;
} ouu_batch_item;

ouu_status ouu_batch_create(const ouu_batch_item* items, int n_items, int autotune, ouu_batch_t* out);
void ouu_batch_destroy(ouu_batch_t b);

/* One evaluation of every item.  z_hosts[k]: item k's controls (host, d_Z of its problem).
 * Outputs per item k (host arrays, like ouu_risk_and_grad): risk_out[k][n_risks],
 * grad_z_out[k][n_risks * d_Z], grad_t_out[k][n_risks], t_out[k][n_risks] (t_out may be
 * NULL).  item_ms (may be NULL): per item, MR-DINO items their graph branch's time, plain
 * items their share of the two persistent launches (SM cycles of their tasks / SM count /
 * clock).  total_ms (may be NULL): the whole batch on the device.  Synchronises. */
ouu_status ouu_batch_run(ouu_batch_t b, const double* const* z_hosts, double* const* risk_out,
                         double* const* grad_z_out, double* const* grad_t_out, double* const* t_out,
                         double* item_ms, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* OUU_H */
