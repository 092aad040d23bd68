/*
 * libidm -- learned parameter initializer (no counterpart in the paper).
 *
 * The paper fits every vehicle from a fixed, knowledge-free initial guess
 * (Sec. IV-A: v0 50, T 1, s0 5, a_max 10, b 2) and is training-free
 * (Sec. V-C).  This part adds a small network that maps a short observed
 * prefix of a vehicle's trajectory and its leader's to an initial guess of
 * (v0, T, s0, a_max, b), so that gradient fitting (idm_fit) starts closer
 * to the solution.  The plain initial guess remains the fallback.
 *
 * Network: 80 -> 256 -> 256 -> 256 -> 5, GELU (erf form, erf evaluated
 * with Abramowitz & Stegun 7.1.26 to 1.5e-7) after the three
 * hidden layers, sigmoid on the output mapped linearly onto the parameter
 * box: theta_q = lo_q + (hi_q - lo_q) * sigmoid(o_q).  153,605 parameters.
 * Weights and activations are bf16, products accumulate in FP32 on the
 * tensor cores (tcgen05.mma, accumulator in tensor memory); the optimizer
 * keeps FP32 master weights (Adam, beta 0.9 / 0.999, eps 1e-8).
 *
 * Flat parameter order (float32, IDM_MLP_N_PARAMS values): W1 [256][80],
 * b1 [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256], W4 [5][256],
 * b4 [5]; layer l computes z = W_l h + b_l (row = output unit).
 *
 * Features (80 per vehicle, from what a fit has: the initial state and the
 * observed targets).  Observation j = 0..19 is at step j * obs_stride;
 * y_0 = p_init, y_j = targets row j-1.  For the vehicle (e) and its leader
 * (l), in this order: x_e[0..19], v_e[0..19], x_l[0..19], v_l[0..19], with
 *   x[j] = (y[j] - y_e[0]) / 100 m,
 *   v[0] = v_init / 30 m/s, v[j] = (y[j+1] - y[j-1]) / (2 obs_stride dt) / 30.
 * A lane head gets a virtual leader 200 m ahead at its own speed:
 *   x_l[j] = x_e[j] + 2, v_l[j] = v_e[j].
 * Training labels are the normalized true parameters (theta_q - lo_q) /
 * (hi_q - lo_q); the loss is their mean squared error over the batch and
 * the 5 outputs, L = sum (sigmoid(o) - label)^2 / (5 B).
 *
 * Conventions (memory, streams, error codes) are those of idm.h; bf16
 * arrays are passed as void* holding IEEE bfloat16 values.
 */
#ifndef IDM_MLP_H_
#define IDM_MLP_H_

#include <stddef.h>
#include <stdint.h>

#include "idm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define IDM_MLP_IN 80
#define IDM_MLP_HIDDEN 256
#define IDM_MLP_OUT 5
#define IDM_MLP_PREFIX 20
#define IDM_MLP_N_PARAMS 153605

typedef struct idm_mlp idm_mlp_t;

/* ---- BF16 tensor-core GEMM ----------------------------------------------
 * C[M][N] = A[M][K] . B[N][K]^T with A, B bf16 row-major (K contiguous),
 * FP32 accumulation and FP32 output C (row-major, N contiguous).
 * Requirements: M >= 1; N a multiple of 16; K a multiple of 16; A, B, C
 * 16-byte aligned.  status (device uint32, required) receives
 * IDM_STATUS_TIMEOUT if a bounded wait inside the kernel gave up (C is then
 * incomplete).  Allocates nothing.  This is the building block of the MLP;
 * it is exported so that it can be tested on its own. */
int idm_gemm_bf16(const void *A, const void *B, int32_t M, int32_t N, int32_t K, float *C, uint32_t *status,
                  void *stream);

/* The activation the network's kernels use, on n values (device arrays;
 * either output may be NULL): gelu(z) = z Phi(z) and gelu'(z) = Phi(z) +
 * z phi(z), with erf from Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7).
 * Exported so that the approximation can be tested on its own. */
int idm_mlp_gelu_eval(const float *z, float *gelu_out, float *gelu_grad_out, int32_t n, void *stream);

/* ---- network object -------------------------------------------------------
 * Creates the network on the current device with workspace for batches of
 * up to max_batch rows (>= 1; memory ~ 9 KB per row plus 3 MB).  Weights
 * start at zero: set them with idm_mlp_set_weights.  Returns IDM_ERR_CUDA
 * if an allocation fails. */
int idm_mlp_create(idm_mlp_t **mlp, int32_t max_batch);
int idm_mlp_destroy(idm_mlp_t *mlp);
const char *idm_mlp_last_error(const idm_mlp_t *mlp);

/* Load FP32 weights (device [IDM_MLP_N_PARAMS], flat order above) into the
 * master copy, refresh the bf16 copies and reset the Adam state. */
int idm_mlp_set_weights(idm_mlp_t *mlp, const float *weights, void *stream);
/* Copy the FP32 master weights to weights (device [IDM_MLP_N_PARAMS]). */
int idm_mlp_get_weights(idm_mlp_t *mlp, float *weights, void *stream);

/* Sticky device status of the network's kernels (IDM_STATUS_* bits);
 * synchronises the stream.  Returns IDM_ERR_TIMEOUT if a bounded wait gave
 * up, IDM_ERR_NONFINITE for a non-finite loss. */
int idm_mlp_status(idm_mlp_t *mlp, void *stream, uint32_t *bits);
/* Clear the sticky status word (synchronises the stream). */
int idm_mlp_clear_status(idm_mlp_t *mlp, void *stream);

/* Bound on the polls of each wait of the network's tensor-core kernels for
 * the tensor core, the copies or another role of the CTA (0 restores the
 * default of 2^26 polls; every wait also gives up after 2 s).  A kernel
 * whose wait runs out sets IDM_STATUS_TIMEOUT, lets every role of the CTA
 * give up, waits (with the default bound) for the copies and tensor-core
 * work it has issued, frees its tensor memory and returns; later calls run
 * normally.  No counterpart in the paper: it lets a test exercise that path
 * with a wait that cannot finish in one poll. */
int idm_mlp_set_wait_limit(idm_mlp_t *mlp, uint32_t polls);

/* ---- features ---------------------------------------------------------------
 * Feature rows for the vehicles perm[r] (r < n_rows; perm NULL = identity)
 * of a scene in head-first lane order (idm.h).
 *   targets: [K/obs_stride][N] observed positions (row j-1 = step j*obs_stride);
 *     needs K / obs_stride >= IDM_MLP_PREFIX.
 *   X (out): bf16 [n_rows][IDM_MLP_IN].
 *   label_params, labels (optional, both or neither): labels[r][q] =
 *     (theta_q - box_lo[q]) / (box_hi[q] - box_lo[q]) of vehicle perm[r] for
 *     q = v0, T, s0, a_max, b; box_lo, box_hi are HOST [5].
 * lane_off must be valid (idm.h); it is only read.  A perm entry outside
 * [0, N) leaves its row of X (and labels) unwritten. */
int idm_mlp_features(const idm_scene_t *scene, const float *p_init, const float *v_init, const idm_sim_t *sim,
                     const float *targets, int32_t obs_stride, const int32_t *perm, int32_t n_rows, void *X,
                     const idm_params_t *label_params, float *labels, const float *box_lo, const float *box_hi,
                     void *stream);

/* ---- inference --------------------------------------------------------------
 * Output of the network for X (bf16 [B][IDM_MLP_IN], 1 <= B <= max_batch):
 * out (device float [B][5]) = sigmoid(o). */
int idm_mlp_forward(idm_mlp_t *mlp, const void *X, int32_t B, float *out, void *stream);

/* Initial parameters for a fit: for each row r < B, params->{v0, T, s0,
 * a_max, b}[r] = box_lo + (box_hi - box_lo) * sigmoid(o) (box HOST [5]);
 * params->delta is not touched.  B may exceed max_batch: larger inputs are
 * processed in chunks of 131,072 rows through two activation buffers
 * (128 MiB) that the first such call allocates and the network keeps. */
int idm_mlp_predict_params(idm_mlp_t *mlp, const void *X, int32_t B, idm_params_t *params, const float *box_lo,
                           const float *box_hi, void *stream);

/* ---- training -------------------------------------------------------------------
 * Loss and gradient for one batch without updating: loss_out (device
 * double, may be NULL), grad (device float [IDM_MLP_N_PARAMS], flat order).
 * labels: device float [B][5].  1 <= B <= max_batch. */
int idm_mlp_loss_grad(idm_mlp_t *mlp, const void *X, const float *labels, int32_t B, double *loss_out, float *grad,
                      void *stream);

/* One Adam step (learning rate lr) on the batch; loss_out (device double,
 * may be NULL) receives the loss before the update. */
int idm_mlp_train_step(idm_mlp_t *mlp, const void *X, const float *labels, int32_t B, float lr, double *loss_out,
                       void *stream);

/* n_steps Adam steps over a training set of n_samples rows (X bf16
 * [n_samples][IDM_MLP_IN], labels [n_samples][5]): step s uses rows
 * [(s mod n_batches) * batch, +batch) with n_batches = n_samples / batch
 * (the tail is not used; shuffle the rows beforehand, e.g. with the perm
 * argument of idm_mlp_features), learning rate linear from lr0 (step 0) to
 * lr1 (last step).  loss_hist (device double [n_steps], may be NULL). */
int idm_mlp_train(idm_mlp_t *mlp, const void *X, const float *labels, int64_t n_samples, int32_t batch,
                  int32_t n_steps, float lr0, float lr1, double *loss_hist, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IDM_MLP_H_ */
