/*
 * libidm -- GB300 (sm_103a) library for the parallel differentiable
 * Intelligent Driver Model simulator of arXiv 2412.16750
 * ("Gradient-based Trajectory Optimization with Parallelized Differentiable
 * Traffic Simulation").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Vehicle order.  Vehicles are stored lane by lane, each lane head first, so
 *   the leader h(i) of a vehicle i that is not a lane head is i-1
 *   (Sec. III-A).  idm_layout produces this order from unsorted input.
 * Memory.  Every array argument is DEVICE memory owned by the caller unless
 *   the comment says "host".  The library never frees caller memory.  The
 *   context owns its workspace (segment tables, initial gaps, checkpoints,
 *   reduction scratch, Adam moments), grown on demand up to the cap given to
 *   idm_ctx_create.
 * Streams.  Every call is asynchronous on the given cudaStream_t (passed as
 *   void*; NULL = legacy default stream).  Outputs are valid once the stream
 *   has reached the call.  One context must not be used by two streams at
 *   the same time.
 * Floating point.  State and parameters are float32 (IEEE binary32); loss
 *   values are float64.  Positions are integrated as a float32 pair
 *   (displacement + rounding error) so that they keep ~1e-5 m over 1,000
 *   steps.
 * Parameters.  idm_params_t holds six arrays of length N in the paper's
 *   notation of Eq. 1-2: v0 = v_targ (desired speed), T = T_pref (time
 *   headway), s0 = s_min (minimum gap), a_max, b = a_pref (comfortable
 *   deceleration), delta (free-road exponent).
 * Errors.  Every entry point returns IDM_OK or one of the codes below and
 *   never aborts.  Argument errors are detected on the host before anything
 *   is launched.  Conditions only the device can see (a lane longer than the
 *   configured maximum, a non-finite state, a malformed lane_off) set bits
 *   of the context's status word; idm_status synchronises the stream and
 *   reports them.  idm_last_error returns a description of the last error.
 */
#ifndef IDM_H_
#define IDM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IDM_OK 0
#define IDM_ERR_ARG 1          /* bad argument (null pointer, size, range) */
#define IDM_ERR_WORKSPACE 2    /* workspace would exceed the context's cap */
#define IDM_ERR_CUDA 3         /* a CUDA runtime call failed */
#define IDM_ERR_NONFINITE 4    /* device status: non-finite state or gradient */
#define IDM_ERR_TIMEOUT 5      /* reserved for bounded device waits */
#define IDM_ERR_LANE 6         /* device status: lane longer than max_lane or lane_off malformed */

/* Device status bits reported by idm_status. */
#define IDM_STATUS_LANE_TOO_LONG 1u
#define IDM_STATUS_BAD_LANE_OFF 2u
#define IDM_STATUS_NONFINITE 4u
#define IDM_STATUS_TIMEOUT 8u   /* a bounded device wait gave up (tensor-core kernels) */

/* Gap floor (m): the gap is max(p_h - p - length_h, IDM_GAP_FLOOR), with zero
 * derivative below the floor.  The paper is silent on gaps <= 0. */
#define IDM_GAP_FLOOR 0.1f

/* Kink band (m/s^2) of the lower bound a_lb = max(-v/dt, a_min) of Sec. III-C:
 * a vehicle-step counts as near the kink when |-v/dt - a_min| is below it
 * (for dt = 0.1 s and a_min = -10 m/s^2: speeds within 0.05 m/s of 1 m/s),
 * where the derivative of a_lb jumps between -1/dt and 0. */
#define IDM_KINK_BAND 0.5f

typedef struct idm_ctx idm_ctx_t;

/* Lane structure of a scene in head-first order.
 *   lane_off[n_lanes+1] (device): lane l holds vehicles
 *     [lane_off[l], lane_off[l+1]); lane_off[0] = 0, lane_off[n_lanes] =
 *     n_vehicles, non-decreasing.  Empty lanes are allowed.
 *   length[n_vehicles] (device): vehicle lengths (m); the gap of a follower
 *     subtracts its LEADER's length (Sec. III-A).
 *   max_lane (host value): an upper bound on the longest lane, used to pick
 *     the kernel variant; at most idm_max_lane_supported().  A lane longer
 *     than max_lane is not simulated and sets IDM_STATUS_LANE_TOO_LONG. */
typedef struct {
    int32_t n_lanes;
    int32_t n_vehicles;
    int32_t max_lane;
    const int32_t *lane_off;
    const float *length;
} idm_scene_t;

/* Per-vehicle IDM parameters (device, each [n_vehicles]; may be NULL when
 * the scene has no vehicles). */
typedef struct {
    float *v0, *T, *s0, *a_max, *b, *delta;
} idm_params_t;

/* Simulation settings shared by all vehicles of a call. */
typedef struct {
    int32_t K;       /* number of Euler steps, >= 1 (Eq. 3) */
    float dt;        /* step length (s), > 0 */
    float a_min;     /* maximum deceleration bound of Sec. III-C, < 0 (paper: -10) */
} idm_sim_t;

/* ---- context ----------------------------------------------------------- */

/* Create a context on the current CUDA device.  workspace_cap_bytes bounds
 * the device memory the context may hold (0 = no bound).  *ctx receives the
 * handle.  Returns IDM_ERR_ARG if ctx is NULL. */
int idm_ctx_create(idm_ctx_t **ctx, size_t workspace_cap_bytes);

/* Release the context and its workspace (synchronises the device first).
 * NULL is accepted. */
int idm_ctx_destroy(idm_ctx_t *ctx);

/* Description of the last error on this context (static storage owned by
 * the context; valid until the next call on it). */
const char *idm_last_error(const idm_ctx_t *ctx);

/* Synchronise `stream` and report the device status word accumulated since
 * the last idm_status call, then clear it.  *flags (host, may be NULL)
 * receives the IDM_STATUS_* bits.  Returns IDM_ERR_LANE or IDM_ERR_NONFINITE
 * when the matching bits are set, IDM_OK otherwise. */
int idm_status(idm_ctx_t *ctx, uint32_t *flags, void *stream);

/* Event counters of the modelling choices the paper leaves open (Sec. III-C):
 * when counting is on (idm_set_event_counting, default off), every
 * idm_forward and idm_batch_forward on this context adds, over the steps
 * k = 0..K-1 it evaluates and every vehicle,
 *   gap_floor_hits: vehicle-steps whose raw gap (p_h - p - length_h) is below
 *                   IDM_GAP_FLOOR (the floor applies and its derivative is 0),
 *   kink_near:      vehicle-steps with |-v/dt - a_min| < IDM_KINK_BAND (the
 *                   lower bound is within the band of its kink; the strict
 *                   -v/dt > a_min rule picks the branch there),
 * both decided in FP32 as the step evaluates them.  The counts accumulate
 * across calls until read.  idm_event_counts synchronises `stream`, returns
 * both counts (host uint64, either pointer may be NULL) and clears them. */
int idm_set_event_counting(idm_ctx_t *ctx, int on);
int idm_event_counts(idm_ctx_t *ctx, void *stream, uint64_t *gap_floor_hits, uint64_t *kink_near);

/* Kernel shape.  Whole lanes are packed into segments of at most
 * 32 * vpt * warps_per_segment vehicles, each simulated by warps_per_segment
 * warps of one block.  vpt: vehicles per thread (2, 4 or 8; 0 = choose);
 * warps_per_segment: 1, 2, 4 or 8 (0 = choose; with both 0 the library
 * takes vpt 4 x 4 warps, 8 x 4 for lanes over 512 vehicles and 8 x 8 over
 * 1024, except for a scene small enough that its segments of 2 vehicles per
 * thread fit 16 warps per SM, where it takes vpt 2 with the fewest warps
 * that hold the longest lane: such a call is bound by the latency of each
 * step, not by throughput); ckpt_interval: steps between stored checkpoints of the adjoint
 * (1..64, default 8); warps_per_block: 1..16 (default 8; rounded to a
 * multiple of warps_per_segment; the adjoint caps it by its shared-memory
 * tape and by its register budget: 4 warps for vpt 4 with segments of up to
 * 4 warps, 8 otherwise).  The forward runs the same segments with 8
 * vehicles per thread where the capacity allows (e.g. 8 x 2 warps for the
 * adjoint's 4 x 4). */
int idm_set_tuning(idm_ctx_t *ctx, int vpt, int warps_per_segment, int ckpt_interval, int warps_per_block);

/* How idm_fit runs its iterations (see idm_fit).  IDM_FIT_AUTO (default):
 * the single launch when K <= ckpt_interval (then the forward runs in the
 * first iteration only: its one checkpoint is the initial state) or N * K <=
 * 2^30 vehicle-steps, provided its loss partials (see idm_fit) fit in 256
 * MB; else the graph (at 2^30 vehicle-steps the two take the same time: the
 * graph's forward kernel runs at its own, higher occupancy).  The graph is always used by idm_fit_eval and while profiling
 * is on (idm_set_profiling times every launch of the graph).  Returns
 * IDM_ERR_ARG for another value. */
#define IDM_FIT_AUTO 0
#define IDM_FIT_GRAPH 1
#define IDM_FIT_SINGLE_LAUNCH 2
int idm_set_fit_mode(idm_ctx_t *ctx, int mode);

/* The form the last idm_fit / idm_fit_eval on this context ran in
 * (IDM_FIT_GRAPH or IDM_FIT_SINGLE_LAUNCH); 0 before the first fit or for a
 * NULL context. */
int idm_last_fit_form(const idm_ctx_t *ctx);

/* Longest lane the library can simulate (vehicles): 32 * 8 * 8 = 2048. */
int idm_max_lane_supported(void);

/* Bytes of workspace a loss/gradient call on this scene would hold. */
size_t idm_workspace_bytes(const idm_ctx_t *ctx, const idm_scene_t *scene, const idm_sim_t *sim);

/* ---- scene layout (Sec. III-A: the leader is the vehicle directly ahead in
 * the same lane) ------------------------------------------------------- */

/* Order N unsorted vehicles by (lane ascending, position descending,
 * original index ascending).
 *   lane_id[N] (device, int32 in [0, n_lanes)), pos[N] (device, float32).
 *   perm[N] (device out): perm[j] = original index of the j-th vehicle.
 *   lane_off[n_lanes+1] (device out): lane CSR offsets.
 *   *max_lane_out (device out, int32, may be NULL): longest lane.
 * Lane ids outside [0, n_lanes) set IDM_STATUS_BAD_LANE_OFF and those
 * vehicles are dropped from the counts.  Lanes longer than 4096 vehicles set
 * IDM_STATUS_LANE_TOO_LONG and are left unsorted within the lane. */
int idm_layout(idm_ctx_t *ctx, int32_t N, int32_t n_lanes, const int32_t *lane_id,
               const float *pos, int32_t *perm, int32_t *lane_off, int32_t *max_lane_out,
               void *stream);

/* dst[j] = src[perm[j]] for j < N, for `count` float32 arrays given as
 * arrays of device pointers in HOST memory (srcs[count], dsts[count]).
 * Every perm[j] must lie in [0, N) (idm_layout's output does). */
int idm_gather(idm_ctx_t *ctx, int32_t N, const int32_t *perm, int count,
               const float *const *srcs, float *const *dsts, void *stream);

/* Column gather of a row-major [n_rows][N] float32 matrix whose columns are
 * vehicles (e.g. observed targets): dst[r*N + j] = src[r*N + perm[j]].
 * Every perm[j] must lie in [0, N).  src and dst must not overlap. */
int idm_gather_rows(idm_ctx_t *ctx, int32_t N, int32_t n_rows, const int32_t *perm,
                    const float *src, float *dst, void *stream);

/* ---- forward (Eq. 1-3 with the Sec. III-C bounds) -------------------- */

/* Simulate sim->K steps from (p_init, v_init).
 *   traj[(K+1)*N] (device out, may be NULL): positions, time-major
 *     (row k = step k, row 0 = p_init).
 *   vtraj[(K+1)*N] (device out, may be NULL): speeds, time-major.
 * v_init must be >= 0. */
int idm_forward(idm_ctx_t *ctx, const idm_scene_t *scene, const idm_params_t *params,
                const float *p_init, const float *v_init, const idm_sim_t *sim,
                float *traj, float *vtraj, void *stream);

/* ---- adjoint from trajectory gradients -------------------------------- */

/* Reverse-time adjoint of idm_forward for a scalar loss L whose gradients
 * with respect to the simulated trajectory are given densely:
 *   gP[(K+1)*N] (device): dL/dP, row k = step k (row 0 is the direct
 *     dependence on p_init); gV[(K+1)*N] (device, may be NULL): dL/dV.
 *   grad (device out, each [N], overwritten; any member may be NULL):
 *     dL/dtheta for the six parameters.
 *   grad_p_init, grad_v_init (device out [N], may be NULL).
 * The trajectory is recomputed from checkpoints taken every ckpt_interval
 * steps, so no trajectory input is needed. */
int idm_backward(idm_ctx_t *ctx, const idm_scene_t *scene, const idm_params_t *params,
                 const float *p_init, const float *v_init, const idm_sim_t *sim,
                 const float *gP, const float *gV, idm_params_t *grad, float *grad_p_init,
                 float *grad_v_init, void *stream);

/* ---- fused squared-error loss and gradient (Sec. IV-A) --------------- */

/* L = sum_i (1/n_obs) sum_{j=1..n_obs} (P[j*s, i] - targets[j-1, i])^2 with
 * n_obs = floor(K / s), s = obs_stride >= 1 (n_obs = 0 gives L = 0).
 *   targets[n_obs*N] (device): observed positions, row j-1 = step j*s.
 *   loss_out (device, double, may be NULL): receives L.
 *   grad (device out, members may be NULL): dL/dtheta.
 *   grad_p_init, grad_v_init (device out, may be NULL). */
int idm_loss_grad(idm_ctx_t *ctx, const idm_scene_t *scene, const idm_params_t *params,
                  const float *p_init, const float *v_init, const idm_sim_t *sim,
                  const float *targets, int32_t obs_stride, double *loss_out,
                  idm_params_t *grad, float *grad_p_init, float *grad_v_init, void *stream);

/* ---- gradient-based fit (Sec. IV-A, Sec. V-B) ------------------------ */

/* n_iter iterations of {forward with loss, adjoint, Adam on (v0, T, s0,
 * a_max, b), projection onto [box_lo[q], box_hi[q]]}; delta is not changed.
 * The learning rate of iteration t (0-based) is lr0 + (lr1 - lr0) t /
 * (n_iter - 1); Adam uses beta1 0.9, beta2 0.999, eps 1e-8, zero initial
 * moments.  The n_iter iterations (1 <= n_iter <= 100000) run in one of two
 * forms with identical results (idm_set_fit_mode):
 *   - graph: one forward and one adjoint launch per iteration (the forward
 *     in the first iteration only when K <= ckpt_interval), captured once
 *     into a CUDA graph, cached on the context for calls with identical
 *     arguments, and launched on `stream` as one graph;
 *   - single launch: one persistent kernel in which each group of warps
 *     carries its lane segments through all n_iter iterations (lanes never
 *     interact, so no iteration waits for the rest of the scene), plus one
 *     reduction of the loss history.
 * Workspace of the single launch: 8 * n_iter * min(n_lanes, 2 * ceil(N /
 * cap) + 1024) * warps_per_segment bytes of loss partials (cap = 32 * vpt *
 * warps_per_segment).
 *   params (device, in/out): initial guess in, fitted values out.
 *   box_lo, box_hi (HOST, [5], order v0, T, s0, a_max, b).
 *   loss_hist (device out, double [n_iter], may be NULL): loss at the
 *     parameters before update t. */
int idm_fit(idm_ctx_t *ctx, const idm_scene_t *scene, idm_params_t *params,
            const float *p_init, const float *v_init, const idm_sim_t *sim,
            const float *targets, int32_t obs_stride, int32_t n_iter, float lr0, float lr1,
            const float *box_lo, const float *box_hi, double *loss_hist, void *stream);

/* idm_fit that also scores every iterate against a second target set
 * (no counterpart in the paper; used to measure the error of the fitted
 * trajectory against the noise-free truth while fitting to noisy targets).
 *   eval_targets (device, same layout as targets): second target set.
 *   eval_hist (device out, double [n_iter]): the loss L of the parameters
 *     before update t against eval_targets, computed by the same forward
 *     that writes the checkpoints (no extra simulation).
 * Both must be given, or both NULL (then this is idm_fit).  The updates are
 * identical to idm_fit's. */
int idm_fit_eval(idm_ctx_t *ctx, const idm_scene_t *scene, idm_params_t *params,
                 const float *p_init, const float *v_init, const idm_sim_t *sim,
                 const float *targets, int32_t obs_stride, int32_t n_iter, float lr0, float lr1,
                 const float *box_lo, const float *box_hi, double *loss_hist,
                 const float *eval_targets, double *eval_hist, void *stream);

/* ---- batched uneven scenarios ------------------------------------------ */

/* Many independent scenes in one launch.  Scenario s owns lanes
 * [scen_lane_off[s], scen_lane_off[s+1]) of the common lane CSR, and is
 * simulated for K[s] steps of dt[s] with observed steps j*obs_stride[s].
 * Per-scenario time-major arrays are concatenated in scenario order:
 *   trajectories: scenario s is a [(K[s]+1)][N_s] block,
 *   targets:      scenario s is a [floor(K[s]/obs_stride[s])][N_s] block,
 * where N_s is the scenario's vehicle count (idm_batch_sizes gives the
 * totals).  The host plans the launch (scenario table, warp segments,
 * longest-first order) and uploads it to the context's workspace; the
 * upload synchronises `stream`. */
typedef struct {
    int32_t n_scen;
    const int32_t *scen_lane_off;  /* HOST [n_scen+1], from 0 to n_lanes */
    const int32_t *K;              /* HOST [n_scen], >= 1 */
    const float *dt;               /* HOST [n_scen], > 0 */
    const int32_t *obs_stride;     /* HOST [n_scen], >= 1 (NULL: every step) */
    float a_min;                   /* shared deceleration bound, < 0 */
    int32_t n_lanes;
    int32_t n_vehicles;
    const int32_t *lane_off_host;  /* HOST [n_lanes+1] lane CSR (head-first lanes) */
    const int32_t *lane_off;       /* DEVICE [n_lanes+1], the same values */
    const float *length;           /* DEVICE [n_vehicles] */
} idm_batch_t;

/* Element counts of the concatenated trajectory, target and checkpoint
 * arrays of a batch (host only; any output may be NULL). */
int idm_batch_sizes(const idm_batch_t *batch, int ckpt_interval, int64_t *traj_elems, int64_t *target_elems,
                    int64_t *ckpt_elems);

/* Positions of every scenario (concatenated [(K_s+1)][N_s] blocks). */
int idm_batch_forward(idm_ctx_t *ctx, const idm_batch_t *batch, const idm_params_t *params,
                      const float *p_init, const float *v_init, float *traj, void *stream);

/* Per-scenario squared-error losses L_s (the single-scene definition applied
 * to each scenario; device double [n_scen], may be NULL), their sum
 * (device double, may be NULL), and the gradients of the sum. */
int idm_batch_loss_grad(idm_ctx_t *ctx, const idm_batch_t *batch, const idm_params_t *params,
                        const float *p_init, const float *v_init, const float *targets, double *scen_loss,
                        double *loss_total, idm_params_t *grad, float *grad_p_init, float *grad_v_init,
                        void *stream);

/* idm_fit over a batch: n_iter Adam iterations on the sum of the scenario
 * losses, the whole fit one CUDA graph or one persistent launch (the rule of
 * idm_set_fit_mode with N * K the batch's sum over scenarios and K its
 * longest horizon; identical results).  loss_hist (device
 * double [n_iter], may be NULL) receives the summed loss before each update,
 * scen_loss (device double [n_scen], may be NULL) the per-scenario losses of
 * the last iteration. */
int idm_batch_fit(idm_ctx_t *ctx, const idm_batch_t *batch, idm_params_t *params, const float *p_init,
                  const float *v_init, const float *targets, int32_t n_iter, float lr0, float lr1,
                  const float *box_lo, const float *box_hi, double *loss_hist, double *scen_loss, void *stream);

/* ---- loss and gradient without allocation ------------------------------ */

/* Size of the library's built-in device scratch array (16 MiB). */
#define IDM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* idm_loss_grad for callers that cannot allocate device memory: an
 * application whose device memory belongs to its own allocator or pool (a
 * cudaMalloc inside a library would bypass it and fragment what it manages),
 * or one that admits work only against a memory budget fixed up front.  The
 * paper has no counterpart; this is a deployment convenience.  No context is
 * needed and nothing is allocated: the scratch (segments, counters, status,
 * initial gaps, loss partials, checkpoints, the compensated gradient totals)
 * lives in one IDM_NOALLOC_SCRATCH_BYTES static device array that every GPU
 * loading the library holds until the process exits.
 *   Arguments, argument checks and results are those of idm_loss_grad; the
 *   kernel shape is the default (checkpoint interval 8).
 *   status_out (device uint32, may be NULL): receives the device status word
 *   (IDM_STATUS_* bits) of this call, since there is no context to query.
 * Limit: the scratch must hold about 16*n_lanes + 4*N + 64*n_lanes +
 * 20*N*ceil(K/8) bytes, plus about 48*N bytes when K > 256 (plus 256-byte alignment
 * of each piece), i.e. about N * ceil(K/8) <= 800,000 vehicle-checkpoints;
 * larger problems return IDM_ERR_WORKSPACE before anything is launched.
 * The first call in a CUDA context looks up the array's device address
 * (cudaGetSymbolAddress) and caches it per context; make that first call
 * before any stream capture.  Every call shares the one array and overwrites
 * it: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Returns IDM_OK, IDM_ERR_ARG,
 * IDM_ERR_WORKSPACE or IDM_ERR_CUDA (no message string is kept). */
int idm_loss_grad_noalloc(const idm_scene_t *scene, const idm_params_t *params, const float *p_init,
                          const float *v_init, const idm_sim_t *sim, const float *targets, int32_t obs_stride,
                          double *loss_out, idm_params_t *grad, float *grad_p_init, float *grad_v_init,
                          uint32_t *status_out, void *stream);

/* ---- measurement ------------------------------------------------------ */

/* When on, idm_fit records CUDA events around every forward and adjoint
 * launch of its graph (on the launching stream). */
int idm_set_profiling(idm_ctx_t *ctx, int on);

/* Synchronise `stream`, then report the summed device time (ms) of the
 * forward and adjoint launches of the last profiled idm_fit and the number
 * of iterations recorded (*n_launches).  Any output pointer may be NULL. */
int idm_phase_times(idm_ctx_t *ctx, void *stream, double *fwd_ms, double *bwd_ms, int32_t *n_launches);

#ifdef __cplusplus
}
#endif
#endif /* IDM_H_ */
