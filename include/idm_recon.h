/*
 * libidm -- single-trajectory filtering and reconstruction mode of
 * arXiv 2412.16750 (Sec. IV-A "Trajectory Filtering & Reconstruction";
 * optimisation settings and metrics of Sec. V-B).
 *
 * Model.  Every trajectory i is one ego vehicle simulated with the modified
 *   IDM (Eq. 1-3 with the bounds of Sec. III-C) behind a virtual leader: at
 *   step k the gap to the leader is dp[k][i] and the speed difference (own
 *   speed minus the leader's, Sec. III-A) is dv[k][i].  Both are free
 *   variables, fitted together with five IDM parameters (v0, T, s0, a_max,
 *   b; delta stays fixed) by minimising the summed absolute error between
 *   every observed position and the simulated position at the observation's
 *   nearest step (the reconstruction loss of Sec. IV-A, summed over the
 *   trajectories).  The gap floor IDM_GAP_FLOOR applies to dp (derivative 0
 *   below it).
 *
 * Observations.  A CSR over trajectories: trajectory i owns observations
 *   obs_off[i] .. obs_off[i+1]-1, in non-decreasing time order, with
 *   timestamps obs_t (s, measured from the trajectory's first observation)
 *   and positions obs_p (m).  The nearest step of a timestamp t is
 *   k = floor(t / dt + 1/2), evaluated in double precision (ties go to the
 *   later step).  Trajectory i is simulated for K[i] = the nearest step of
 *   its last observation.  Observations at step 0 (the given initial state)
 *   do not enter the loss.
 *
 * Initial state (Sec. V-B): p_init = the first observed position, v_init =
 *   (second - first observed position) / (their time difference), clamped
 *   at 0 (speeds stay non-negative, Sec. III-C); v_init = 0 with fewer than
 *   two observations or equal first timestamps, p_init = 0 with none.
 *
 * Layout.  Per-step arrays are time-major with a row stride `ld` >= n_traj
 *   elements: element (k, i) sits at [k * ld + i].  dp, dv, A and the
 *   gradients of dp, dv have k_max rows (step k = 0 .. k_max-1); P and V have
 *   k_max + 1 rows (row 0 = the initial state).  k_max must be >= every
 *   K[i].  Rows k >= K[i] of trajectory i are not read; outputs there hold
 *   the final state (P, V) or 0 (A and gradients).  Per-trajectory arrays
 *   (K, p_init, v_init, parameters) have n_traj elements.
 *
 * Memory, streams, errors.  As for the rest of libidm (idm.h): device
 *   arrays owned by the caller unless marked HOST; asynchronous on `stream`;
 *   the context owns its workspace (the per-step tape of the adjoint, the
 *   observation index and the Adam moments).  Argument errors are found on
 *   the host before any launch (IDM_ERR_ARG); a non-finite state or
 *   gradient sets IDM_STATUS_NONFINITE in the context's status word, and a
 *   malformed observation CSR or decreasing timestamps set
 *   IDM_STATUS_BAD_OBS (see idm_status).  Floating point: FP32 state,
 *   positions as an FP32 pair, FP64 loss sums.
 */
#ifndef IDM_RECON_H_
#define IDM_RECON_H_

#include <stddef.h>
#include <stdint.h>

#include "idm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Error code of idm_status when IDM_STATUS_BAD_OBS is set. */
#define IDM_ERR_OBS 7

/* Device status bit: obs_off not non-decreasing from 0, a timestamp below
 * the previous one of its trajectory, or an observation whose nearest step
 * lies outside [0, k_max]. */
#define IDM_STATUS_BAD_OBS 16u

/* Observed trajectories of one call. */
typedef struct {
    int32_t n_traj;          /* N >= 0 */
    int32_t k_max;           /* rows of the per-step arrays, >= max K[i], >= 1 */
    int32_t ld;              /* row stride of the per-step arrays, >= n_traj */
    int64_t n_obs;           /* HOST value: obs_off[n_traj], < 2^28 */
    const int32_t *obs_off;  /* [N+1] */
    const float *obs_t;      /* [n_obs] */
    const float *obs_p;      /* [n_obs] */
    const int32_t *obs_k;    /* [n_obs] nearest steps, from idm_recon_prepare */
    const int32_t *K;        /* [N] steps per trajectory, from idm_recon_prepare */
    const float *p_init;     /* [N] initial position */
    const float *v_init;     /* [N] initial speed, >= 0 */
    float dt;                /* step length (s), > 0 (paper: 0.1 filtering, 1.0 reconstruction) */
    float a_min;             /* deceleration bound of Sec. III-C, < 0 (paper: -10) */
} idm_recon_t;

/* Nearest steps, horizons and initial states of N trajectories (the rules
 * stated above).
 *   obs_off[N+1], obs_t, obs_p [n_obs] (device, in).
 *   obs_k [n_obs], K [N], p_init [N], v_init [N] (device, out).
 *   k_max_out (HOST out, may be NULL): max K[i]; when given, the call waits
 *     for the stream to read it back.
 * A malformed CSR or decreasing timestamps set IDM_STATUS_BAD_OBS. */
int idm_recon_prepare(idm_ctx_t *ctx, int32_t N, int64_t n_obs, const int32_t *obs_off, const float *obs_t,
                      const float *obs_p, float dt, int32_t *obs_k, int32_t *K, float *p_init, float *v_init,
                      int32_t *k_max_out, void *stream);

/* Simulate every trajectory for its K[i] steps (Eq. 3).
 *   params (device, each [N]): the IDM parameters of each trajectory.
 *   dp, dv (device, k_max rows): the virtual leader.
 *   P, V ([k_max+1] rows), A ([k_max] rows) (device out, each may be NULL):
 *     positions (the FP32 value of the position pair), speeds and bounded
 *     accelerations a*. */
int idm_recon_forward(idm_ctx_t *ctx, const idm_recon_t *rec, const idm_params_t *params, const float *dp,
                      const float *dv, float *P, float *V, float *A, void *stream);

/* Reconstruction loss L = sum_i sum_j |P[k_ij][i] - obs_p[j]| and its
 * gradients, with the subgradient sign(0) = 0.
 *   loss_out (device, double, may be NULL): L.
 *   grad (device out, members may be NULL): dL/d(v0, T, s0, a_max, b, delta).
 *   g_dp, g_dv (device out, k_max rows, may be NULL): dL/d dp, dL/d dv.
 *   g_p_init, g_v_init (device out [N], may be NULL). */
int idm_recon_loss_grad(idm_ctx_t *ctx, const idm_recon_t *rec, const idm_params_t *params, const float *dp,
                        const float *dv, double *loss_out, idm_params_t *grad, float *g_dp, float *g_dv,
                        float *g_p_init, float *g_v_init, void *stream);

/* n_iter Adam iterations (Sec. V-B: 500 iterations, learning rate linear
 * from lr0 = 0.1 to lr1 = 0.01) on (v0, T, s0, a_max, b), projected onto
 * [box_lo[q], box_hi[q]], and on every dp[k][i], dv[k][i] with k < K[i]
 * (unconstrained).  Adam: beta1 0.9, beta2 0.999, eps 1e-8, zero initial
 * moments; the learning rate of iteration t (0-based) is lr0 + (lr1 - lr0)
 * t / (n_iter - 1).  The trajectories are independent, so the whole fit is
 * one kernel launch: every thread runs all iterations of its trajectory.
 *   params, dp, dv (device, in/out).
 *   box_lo, box_hi (HOST, [5], order v0, T, s0, a_max, b).
 *   loss_hist (device out, double [n_iter], may be NULL): L before update t. */
int idm_recon_fit(idm_ctx_t *ctx, const idm_recon_t *rec, idm_params_t *params, float *dp, float *dv,
                  int32_t n_iter, float lr0, float lr1, const float *box_lo, const float *box_hi,
                  double *loss_hist, void *stream);

/* Metrics of Sec. V-B for the current parameters and virtual leader:
 *   out[0] Pos.: mean over all observations of |P[k_ij][i] - obs_p[j]| /
 *          (|last - first observed position of trajectory i|), trajectories
 *          of zero length skipped;
 *   out[1], out[2]: mean and standard deviation of |a*| over every simulated
 *          step of every trajectory;
 *   out[3] Imp.: fraction of trajectories with some |a*| > 10 m/s^2.
 * out (device, double [4]). */
int idm_recon_metrics(idm_ctx_t *ctx, const idm_recon_t *rec, const idm_params_t *params, const float *dp,
                      const float *dv, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IDM_RECON_H_ */
