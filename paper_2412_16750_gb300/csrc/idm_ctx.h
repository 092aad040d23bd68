// Internal: the libidm context, its workspace and the launch planning shared
// by the single-scene entry points (idm_abi.cu) and the batched ones
// (idm_batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "../../include/idm.h"
#include "idm_internal.h"

namespace idm {
namespace abi {

struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

enum Ctl { CTL_NSEG = 0, CTL_WORK_F = 1, CTL_WORK_B = 2, CTL_ITER = 3, CTL_N = 8 };

// Launch plan of one call.
struct Prep {
    int vpt = 1;    // adjoint shape: vehicles per thread
    int G = 1;      //               warps per segment
    int vpt_f = 1;  // forward shape (same segment capacity 32 * vpt * G)
    int G_f = 1;
    int wpb_f = 1;  // warps per block of the forward (a multiple of G_f)
    int grid_f = 1, grid_b = 1;
    int wpb_b = 1;  // warps per block of the adjoint (bounded by its shared-memory tape)
    int loss_per_seg = 1;
    int k_max = 0;  // longest horizon of the call (steps)
    SimArgs a;
};

}  // namespace abi
}  // namespace idm

struct idm_ctx {
    int device = 0;
    int n_sm = 1;
    size_t cap = 0;
    size_t held = 0;
    char err[512] = {0};
    int vpt_req = 0;
    int G_req = 0;
    int C = 8;
    int wpb = 8;
    idm::abi::Buf seg, ctl, status, g0, ckpt, loss_part, loss_tmp, adam_m, adam_v, lay_counts, lay_cursor, eval_part, sub_ckpt;
    idm::abi::Buf scen_tab, scen_seg_off, scen_seg_idx, lane_off_dev;  // batched scenarios
    idm::abi::Buf rec_oyy, rec_oyc, rec_multi, rec_tape, rec_mom, rec_thm, rec_acc, rec_kmax;  // reconstruction mode
    idm::abi::Buf fit_part;            // single-launch fit: loss partials of every iteration
    idm::abi::Buf gsum;                // adjoint: compensated totals of the gradient sums [6][2][N]
    int fit_mode = IDM_FIT_AUTO;
    int last_fit_form = 0;             // IDM_FIT_GRAPH or IDM_FIT_SINGLE_LAUNCH of the last idm_fit (0: none)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t fit_exec = nullptr;
    unsigned char fit_key[640] = {0};  // arguments the cached fit graph was captured with
    size_t fit_key_len = 0;
    int profiling = 0;
    int count_events = 0;              // idm_forward / idm_batch_forward add to the event counters
    int no_alloc = 0;                  // planning-only context: ensure() fails instead of allocating
    std::vector<cudaEvent_t> ev;       // per fit iteration: fwd begin/end, adjoint begin/end
    int ev_used = 0;                   // iterations recorded by the cached graph
};

namespace idm {
namespace abi {

int fail(idm_ctx *c, int code, const char *fmt, ...);
int cuda_fail(idm_ctx *c, cudaError_t e, const char *what);
int ensure(idm_ctx *c, Buf &b, size_t bytes, const char *name);
int ensure_status(idm_ctx *c);
// The status buffer: status word (unsigned) at byte 0, the two 64-bit event
// counters (gap-floor hits, kink band) at byte STATUS_EVENTS_OFF.
constexpr size_t STATUS_BYTES = 32;
constexpr size_t STATUS_EVENTS_OFF = 16;
// Event counters for a forward launch of this context (NULL when off).
unsigned long long *event_counters(idm_ctx *c);
// Kernel shape for a call: the context's request, else 4 x 4 (8 x 4, 8 x 8
// for longer lanes), or for a scene that fits one wave of 2-vehicle warps
// the latency shape 2 x G.
int pick_shape(idm_ctx *c, int max_lane, long long n_vehicles, int n_lanes, int *vpt, int *G);
// Forward shape for the segment capacity of the adjoint shape (vpt, G).
void forward_shape(int vpt, int G, int *vpt_f, int *G_f);
// Parameter arrays: required unless the scene has no vehicles.
int check_params(idm_ctx *c, const idm_params_t *p, bool all, long long n_vehicles);
// Scene (lanes, lengths, max_lane) and simulation settings (K >= 1, finite
// dt > 0, finite a_min < 0) of the single-scene calls.
int check_scene(idm_ctx *c, const idm_scene_t *s);
int check_sim(idm_ctx *c, const idm_sim_t *s);
int forward_grid(idm_ctx *c, Prep *P, int L);
int backward_grid(idm_ctx *c, Prep *P, bool dense, bool adam, bool want_delta, int L);
// Capture (or reuse) the n_iter-iteration fit graph for plan P and launch it.
// finalize(it, stream) enqueues the loss reduction of iteration it.  With
// eval_targets and eval_hist set, each iteration's forward also records the
// loss against eval_targets in eval_hist[it] (single scene only).
// The single-launch fit of plan P (single scene or batch): Adam state and
// the [n_iter][stride] loss partials in the workspace, moments and work
// counter cleared, the persistent kernel launched.  The caller reduces the
// partials.
int launch_single_fit(idm_ctx *c, Prep &P, int n_iter, size_t N, const float *box_lo, const float *box_hi, float lr0,
                      float lr1, long long stride, cudaStream_t st);
// The fit of a single scene as one persistent launch (no eval targets, no
// per-launch profiling); same results as run_fit_graph with single-scene
// loss reduction.
int run_fit_single(idm_ctx *c, Prep &P, int n_iter, size_t N, int n_lanes, const float *box_lo, const float *box_hi,
                   float lr0, float lr1, double *loss_hist, cudaStream_t st);
// IDM_FIT_AUTO picks the single launch when K fits one checkpoint interval
// (its forward then runs once) or up to this many vehicle-steps per
// iteration (N * K).  Measured on GB300, single launch over graph: 1.5x at
// 2e6-4e6 vehicle-steps, 1.2x at 2e7, 1.06x at 2e8, 1.01x at 6e8, 1.00x at
// 2e9 (where the graph's forward kernel, at its own higher occupancy, makes
// up for the launch boundaries).
constexpr double IDM_SINGLE_LAUNCH_MAX_VEHICLE_STEPS = 1073741824.0;
// ... and only while its loss partials (8 bytes per warp segment and
// iteration) stay within this much workspace.
constexpr double IDM_SINGLE_LAUNCH_MAX_PARTIAL_BYTES = 268435456.0;
long long single_launch_stride(const Prep &P, size_t N, int n_lanes);
int run_fit_graph(idm_ctx *c, Prep &P, int n_iter, size_t N, const float *box_lo, const float *box_hi, float lr0,
                  float lr1, double *loss_hist, const void *extra_key, size_t extra_len, cudaStream_t st,
                  cudaError_t (*finalize)(idm_ctx *, const Prep &, int, double *, cudaStream_t),
                  const float *eval_targets = nullptr, double *eval_hist = nullptr);

}  // namespace abi
}  // namespace idm

#define IDM_CK(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return idm::abi::cuda_fail(c, e_, #call); \
    } while (0)
