// Internal types shared by the kernels and the C-ABI layer of libidm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace idm {

// One scenario: a contiguous range of lanes/vehicles simulated with its own
// horizon, step and observation stride.  Time-major arrays of the scenario
// ([K+1][n_veh] trajectories, [n_obs][n_veh] targets, checkpoints) start at
// the given element offsets.
struct ScenDesc {
    int veh_begin;      // first vehicle (global index)
    int n_veh;          // vehicles in the scenario (row length of its arrays)
    int K;              // steps
    int obs_stride;     // observed steps are k = s, 2s, ... <= K
    int n_obs;          // floor(K / s)
    float dt, inv_dt, a_min;
    float inv_nobs;     // 1 / n_obs (0 if none)
    int pad;
    long long traj_off;  // element offset of row 0 of the trajectories
    long long tgt_off;   // element offset of the targets (row j-1 = step j*s)
    long long ckpt_off;  // element offset of the checkpoints
};

// The segment builder packs lanes in this many contiguous chunks (one
// thread each, next-fit inside a chunk), so n vehicles in lanes no longer
// than the capacity give at most 2 n / cap + SEG_BUILD_CHUNKS segments.
constexpr int SEG_BUILD_CHUNKS = 1024;

// One warp segment: whole lanes packed into at most 32*VPT slots.
struct Seg {
    int veh_begin;  // global index of slot 0
    int n_veh;      // occupied slots
    int scen;       // scenario index
    int pad;
};

// Everything a simulation kernel reads or writes (passed by value).
struct SimArgs {
    const Seg *seg;
    const int *n_seg;
    int *work;                  // persistent work counter (zeroed before launch)
    const ScenDesc *scen_tab;   // NULL: every segment uses scen0
    ScenDesc scen0;
    const float *g0;            // initial raw gap (+inf for lane heads)
    int G;                      // warps per segment (1, 2, 4 or 8)
    const float *v0, *T, *s0, *am, *b, *delta;
    const float *p_init, *v_init;
    float *traj, *vtraj;
    const float *targets;
    double *loss_part;          // [n_seg * G] per-warp loss
    float *ckpt;
    int C;                      // checkpoint interval (steps)
    int tape_T;                 // adjoint tape depth (steps, <= C); tape_T < C uses sub_ckpt
    float *sub_ckpt;            // [ceil(C/tape_T)-1][4][N_total] states inside a checkpoint segment
    unsigned *status;
    // adjoint
    const float *gP, *gV;       // dense trajectory gradients (scenario-local time-major)
    float *g_v0, *g_T, *g_s0, *g_am, *g_b, *g_delta, *g_p_init, *g_v_init;
    // Adam (fit)
    float *adam_m, *adam_v;     // [5][N_total]
    int iter;                   // 0-based iteration of the fit
    int n_iter;
    int N_total;
    float lr0, lr1;
    float lo[5], hi[5];
    // forward only: squared error against a second target set (same layout
    // as targets), per warp like loss_part; NULL = off
    const float *eval_targets;
    double *eval_part;
    // adjoint: 1 = copy the next checkpoint segment's targets and checkpoint
    // into double-buffered shared stages while the current segment runs
    // (needs more shared memory), 0 = load each segment when it starts
    int bwd_pf;
    // adjoint: compensated running totals of the six factored gradient sums,
    // per segment 6 x (capacity / 2) float4 (16-byte aligned); needed
    // (non-NULL) when a horizon exceeds GSUM_FOLD_STEPS
    float *gsum;
    // forward: event counters (NULL = not counted): [0] vehicle-steps with the
    // raw gap below the floor, [1] vehicle-steps within IDM_KINK_BAND of the
    // kink of the lower bound max(-v/dt, a_min)
    unsigned long long *events;
};

// Steps of FP32 accumulation between two compensated folds of the gradient
// sums (idm_adjoint.cuh); a call whose longest horizon exceeds it needs gsum:
// gsum_bytes(segments, capacity) bytes.
inline size_t gsum_bytes(size_t n_seg, int capacity) { return n_seg * (size_t)capacity * 12 * sizeof(float); }
constexpr int GSUM_FOLD_STEPS = 256;

// Floats per vehicle of a stored state (checkpoints, sub-checkpoints, the
// adjoint's state stage): position high and low parts, speed, raw gap and the
// compensation of the speed sum (State2).
constexpr int STATE_ROWS = 5;

// Launchers (idm_sim.cu).  Return cudaError_t of the launch.
cudaError_t launch_prep_gap(const int *lane_off, int n_lanes, const float *p_init, const float *length,
                            int N, float *g0, unsigned *status, cudaStream_t st);
cudaError_t launch_build_segments(const int *lane_off, int n_lanes, const int *scen_lane_off, int n_scen,
                                  int cap, int N, Seg *seg, int *n_seg, unsigned *status, cudaStream_t st);
// The kernel shape (vehicles per thread, warps per segment) of each launch is
// passed explicitly; the forward and the adjoint may differ as long as
// 32 * vpt * G (the segment capacity the segments were packed for) agrees.
cudaError_t launch_forward(int vpt, int G, bool traj, bool vtraj, bool ckpt, const SimArgs &a, int grid, int wpb,
                           cudaStream_t st);
cudaError_t launch_backward(int vpt, int G, bool dense_seed, bool adam, bool want_delta, const SimArgs &a,
                            int grid, int wpb, cudaStream_t st);
size_t backward_smem_bytes(int vpt, bool dense_seed, int T, int G, int wpb, bool prefetch);
size_t forward_smem_bytes(int vpt, int G, int wpb);
// Largest adjoint block (warps) for a shape: 4 for 4 vehicles per thread in
// segments of up to 4 warps (register budget), else 8.
int backward_max_warps(int vpt, int G);
// Adjoint warps per SM the register budgets allow for a shape.
int backward_resident_warps(int vpt, int G);
cudaError_t launch_loss_finalize(const double *loss_part, const int *n_seg, int per_seg, double *out, cudaStream_t st);
// Single-launch fit (idm_fused.cuh): every Adam iteration of every segment
// in one persistent launch of the adjoint's shape (vpt, G, wpb, tape depth
// and prefetch of `a`); loss partial of iteration it at
// loss_part[it * part_stride + ...].  The grid is capped at the resident
// blocks.
cudaError_t launch_fit_fused(int vpt, int G, const SimArgs &a, long long part_stride, int grid, int wpb,
                             cudaStream_t st);
// Losses of iterations 0..n_iter-1 of a single-launch fit into out[n_iter],
// each summed in the order of launch_loss_finalize.
cudaError_t launch_loss_finalize_iters(const double *loss_part, long long stride, const int *n_seg, int per_seg,
                                       int n_iter, double *out, cudaStream_t st);
int occupancy_blocks(int vpt, int G, bool backward, bool dense_seed, bool adam, bool want_delta, int wpb, size_t smem,
                     bool sub = false);
// Kernel shapes (vehicles per thread, warps per segment) with compiled
// adjoint and single-launch fit kernels; X(V, G) per shape.
#define IDM_SHAPES(X) \
    X(2, 1) X(2, 2) X(2, 4) X(2, 8) X(4, 1) X(4, 2) X(4, 4) X(4, 8) X(8, 1) X(8, 2) X(8, 4) X(8, 8)
// Per shape (idm_shape_v<V>_g<G>.cu): the forward kernel (with or without
// event counting), the adjoint kernel for dense or target seeds, fused Adam,
// the delta gradient and tape blocks with sub-checkpoints, and the
// single-launch fit kernel (tape blocks or not).
#define IDM_DECLARE_SHAPE(V, GW)                                             \
    void *forward_fn_v##V##_g##GW(bool count);                                \
    void *backward_fn_v##V##_g##GW(bool dense, bool adam, bool wd, bool sub); \
    void *fused_fn_v##V##_g##GW(bool sub);
IDM_SHAPES(IDM_DECLARE_SHAPE)
#undef IDM_DECLARE_SHAPE

// Layout (idm_layout.cu).
cudaError_t launch_layout(int N, int n_lanes, const int32_t *lane_id, const float *pos, int32_t *perm,
                          int32_t *lane_off, int32_t *max_lane, int *counts, int *cursor, unsigned *status,
                          cudaStream_t st);
cudaError_t launch_gather(int N, const int32_t *perm, int count, const float *const *srcs, float *const *dsts,
                          cudaStream_t st);
cudaError_t launch_gather_rows(int N, int n_rows, const int32_t *perm, const float *src, float *dst, cudaStream_t st);

}  // namespace idm
