/*
 * libidm_cpu -- multi-threaded CPU backend of the differentiable IDM
 * simulator of arXiv 2412.16750, the counterpart of the paper's 16-thread
 * CPU mode (Sec. V-A, Fig. 1: the CPU is faster for small vehicle counts,
 * the GPU beyond about 20K vehicles).
 *
 * A separate library with HOST pointers only: it is an explicit backend a
 * caller chooses, never a fallback of the CUDA library (libidm.so has no CPU
 * path).  The model, loss and optimiser are those of include/idm.h:
 *   - Eq. 1-3 with the softplus bounds of Sec. III-C, the gap floor
 *     IDM_GAP_FLOOR (derivative 0 below it), a lane head sees no leader;
 *   - vehicles lane by lane, each lane head first (leader of i = i-1);
 *   - loss L = sum_i (1/n_obs) sum_{j=1..n_obs} (P[j s][i] - targets[j-1][i])^2,
 *     n_obs = floor(K / s);
 *   - Adam (0.9, 0.999, 1e-8), learning rate lr0 + (lr1 - lr0) t / (n_iter-1),
 *     projection onto the box, delta not fitted.
 * Floating point: FP32 state with the position as an FP32 pair (as the CUDA
 * path), FP64 loss and parameter-gradient sums.  Results do not depend on
 * the thread count (lanes are independent; every reduction runs in lane
 * order).
 *
 * Threads: n_threads <= 0 uses the OpenMP default (all cores).  Lanes are
 * scheduled dynamically; every thread keeps the tape of the lane it works on
 * (speed and gap of every vehicle at every step) and, in idm_cpu_fit, runs
 * all iterations of a lane before taking the next, so a lane's working set
 * stays in the core's cache.
 *
 * Errors: IDM_OK, or IDM_ERR_ARG (argument check, nothing computed),
 * IDM_ERR_WORKSPACE (a host allocation failed) or IDM_ERR_NONFINITE (a
 * non-finite state or gradient; outputs are still written).
 */
#ifndef IDM_CPU_H_
#define IDM_CPU_H_

#include <stdint.h>

#include "idm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters on the host: six arrays of n_vehicles (v0, T, s0, a_max, b,
 * delta), the notation of idm_params_t. */
typedef idm_params_t idm_cpu_params_t;

/* Lanes on the host: lane l holds vehicles [lane_off[l], lane_off[l+1])
 * (lane_off[0] = 0, non-decreasing, lane_off[n_lanes] = n_vehicles);
 * length[n_vehicles] are the vehicle lengths (a follower's gap subtracts its
 * leader's length). */
typedef struct {
    int32_t n_lanes;
    int32_t n_vehicles;
    const int32_t *lane_off;
    const float *length;
} idm_cpu_scene_t;

/* Number of threads an n_threads <= 0 call uses. */
int idm_cpu_max_threads(void);

/* K steps from (p_init, v_init) (v_init >= 0).  traj, vtraj (HOST out,
 * [(K+1) * n_vehicles] time-major, may be NULL): positions (the FP32 value
 * of the pair) and speeds, row 0 = the initial state. */
int idm_cpu_forward(int n_threads, const idm_cpu_scene_t *scene, const idm_cpu_params_t *params,
                    const float *p_init, const float *v_init, const idm_sim_t *sim, float *traj, float *vtraj);

/* The loss of the header comment and its gradients.
 *   targets (HOST, [n_obs * n_vehicles], row j-1 = step j * obs_stride).
 *   loss_out (HOST, may be NULL); grad (HOST out, members may be NULL);
 *   g_p_init, g_v_init (HOST out [n_vehicles], may be NULL). */
int idm_cpu_loss_grad(int n_threads, const idm_cpu_scene_t *scene, const idm_cpu_params_t *params,
                      const float *p_init, const float *v_init, const idm_sim_t *sim, const float *targets,
                      int32_t obs_stride, double *loss_out, idm_cpu_params_t *grad, float *g_p_init,
                      float *g_v_init);

/* n_iter Adam iterations on (v0, T, s0, a_max, b) of params (HOST, in/out),
 * box_lo / box_hi [5]; loss_hist (HOST out [n_iter], may be NULL): the loss
 * before update t. */
int idm_cpu_fit(int n_threads, const idm_cpu_scene_t *scene, idm_cpu_params_t *params, const float *p_init,
                const float *v_init, const idm_sim_t *sim, const float *targets, int32_t obs_stride,
                int32_t n_iter, float lr0, float lr1, const float *box_lo, const float *box_hi,
                double *loss_hist);

#ifdef __cplusplus
}
#endif

#endif /* IDM_CPU_H_ */
