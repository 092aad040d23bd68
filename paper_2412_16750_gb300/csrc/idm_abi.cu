// C-ABI of libidm (declared in include/idm.h): argument checks, the context
// and its workspace, kernel-variant selection and the fit's CUDA graph.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>
#include <cmath>
#include <new>

#include "../../include/idm.h"
#include "../../include/idm_lanes.h"
#include "../../include/idm_recon.h"
#include "idm_ctx.h"
#include "idm_internal.h"

using idm::ScenDesc;
using idm::Seg;
using idm::SimArgs;
using namespace idm::abi;

namespace idm {
namespace abi {

int fail(idm_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(idm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, IDM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call) IDM_CK(call)

int ensure(idm_ctx *c, Buf &b, size_t bytes, const char *name)
{
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return IDM_OK;
    if (c->no_alloc) return fail(c, IDM_ERR_WORKSPACE, "%s would need an allocation", name);
    size_t want = c->held - b.n + bytes;
    if (c->cap && want > c->cap)
        return fail(c, IDM_ERR_WORKSPACE, "workspace for %s needs %zu bytes in total, cap is %zu", name, want,
                    c->cap);
    if (b.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
        cudaFree(b.p);
        c->held -= b.n;
        b.p = nullptr;
        b.n = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, IDM_ERR_WORKSPACE, "cudaMalloc of %zu bytes for %s failed: %s", bytes, name,
                    cudaGetErrorString(e));
    }
    b.n = bytes;
    c->held += bytes;
    return IDM_OK;
}

// Kernel shape: VPT vehicles per thread, G warps per segment (capacity
// 32*VPT*G vehicles).  The default packs several 100-vehicle lanes into one
// 512-slot segment (VPT 4, G 4).
// The device status word accumulates across calls until idm_status reads
// and clears it, so it must start at zero when first allocated.
int ensure_status(idm_ctx *c)
{
    if (c->status.p) return IDM_OK;
    int rc = ensure(c, c->status, STATUS_BYTES, "status");
    if (rc) return rc;
    cudaError_t e = cudaMemset(c->status.p, 0, STATUS_BYTES);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // before any stream of the caller uses it
    if (e != cudaSuccess) return cuda_fail(c, e, "clearing the status word");
    return IDM_OK;
}

unsigned long long *event_counters(idm_ctx *c)
{
    if (!c->count_events || !c->status.p) return nullptr;
    return reinterpret_cast<unsigned long long *>(static_cast<char *>(c->status.p) + STATUS_EVENTS_OFF);
}

int pick_shape(idm_ctx *c, int max_lane, long long n_vehicles, int n_lanes, int *vpt, int *G)
{
    int v = c->vpt_req, g = c->G_req;
    if (v == 0 && g == 0) {
        // 4 vehicles per thread x 4 warps (512 slots); 8 x 4 and 8 x 8 for
        // lanes longer than 512 and 1024
        v = 4;
        g = 4;
        if (max_lane > 512) v = 8;
        if (max_lane > 1024) g = 8;
        // a scene whose segments fit one wave of 2-vehicle warps (16 per SM)
        // is bound by the latency of each warp's step, not by throughput:
        // 2 vehicles per thread (the fewest instructions per step) and the
        // fewest warps per segment that hold the longest lane (measured on
        // GB300, loss + gradient over 100 steps: 0.15 -> 0.11 ms at 100
        // vehicles, 0.20 -> 0.12 ms at 16,000, 0.32 -> 0.17 ms at 64,000)
        int g2 = 1;
        while (64 * g2 < max_lane && g2 < 8) g2 <<= 1;
        if (64 * g2 >= max_lane) {
            const long long cap2 = 64LL * g2;
            const long long segs = std::min<long long>(n_lanes, 2 * ((n_vehicles + cap2 - 1) / cap2) + 1);
            if (segs * g2 <= 16LL * c->n_sm) {
                v = 2;
                g = g2;
            }
        }
    } else if (v == 0) {
        v = 2;
        while (32 * v * g < max_lane && v < 8) v <<= 1;
    } else if (g == 0) {
        g = 1;
        while (32 * v * g < max_lane && g < 8) g <<= 1;
    }
    if (32 * v * g < max_lane)
        return fail(c, IDM_ERR_ARG, "max_lane %d exceeds %d vehicles per segment (vpt %d, %d warps)", max_lane,
                    32 * v * g, v, g);
    *vpt = v;
    *G = g;
    return IDM_OK;
}

int check_scene(idm_ctx *c, const idm_scene_t *s)
{
    if (!s) return fail(c, IDM_ERR_ARG, "scene is NULL");
    if (s->n_lanes < 1) return fail(c, IDM_ERR_ARG, "n_lanes must be >= 1 (got %d)", s->n_lanes);
    if (s->n_vehicles < 0) return fail(c, IDM_ERR_ARG, "n_vehicles must be >= 0");
    if (!s->lane_off) return fail(c, IDM_ERR_ARG, "lane_off is NULL");
    if (s->n_vehicles > 0 && !s->length) return fail(c, IDM_ERR_ARG, "length is NULL");
    if (s->max_lane < 0 || s->max_lane > idm_max_lane_supported())
        return fail(c, IDM_ERR_ARG, "max_lane %d outside [0, %d]", s->max_lane, idm_max_lane_supported());
    return IDM_OK;
}

int check_params(idm_ctx *c, const idm_params_t *p, bool all, long long n_vehicles)
{
    if (!p) return fail(c, IDM_ERR_ARG, "params is NULL");
    if (n_vehicles == 0) return IDM_OK;  // nothing is read or written
    if (!p->v0 || !p->T || !p->s0 || !p->a_max || !p->b || (all && !p->delta))
        return fail(c, IDM_ERR_ARG, "a parameter array is NULL");
    return IDM_OK;
}

int check_sim(idm_ctx *c, const idm_sim_t *s)
{
    if (!s) return fail(c, IDM_ERR_ARG, "sim is NULL");
    if (s->K < 1) return fail(c, IDM_ERR_ARG, "K must be >= 1 (got %d)", s->K);
    if (!(s->dt > 0.0f) || !std::isfinite(s->dt)) return fail(c, IDM_ERR_ARG, "dt must be finite and > 0");
    if (!(s->a_min < 0.0f) || !std::isfinite(s->a_min)) return fail(c, IDM_ERR_ARG, "a_min must be finite and < 0");
    return IDM_OK;
}

// Common preparation of a single-scene call: buffers, initial gaps and warp
// segments.
static int prepare(idm_ctx *c, const idm_scene_t *sc, const idm_params_t *pr, const float *p_init, const float *v_init,
            const idm_sim_t *sim, bool need_ckpt, bool need_loss, int obs_stride, Prep *P, cudaStream_t st)
{
    int rc;
    if ((rc = pick_shape(c, sc->max_lane, sc->n_vehicles, sc->n_lanes, &P->vpt, &P->G))) return rc;
    const int N = sc->n_vehicles, L = sc->n_lanes;
    const int G = P->G;
    if ((rc = ensure(c, c->seg, sizeof(Seg) * (size_t)L, "segments"))) return rc;
    if ((rc = ensure(c, c->ctl, sizeof(int) * CTL_N, "control"))) return rc;
    if ((rc = ensure_status(c))) return rc;
    if ((rc = ensure(c, c->g0, sizeof(float) * (size_t)N, "initial gaps"))) return rc;
    if ((rc = ensure(c, c->loss_part, sizeof(double) * (size_t)L * G, "loss partials"))) return rc;
    if ((rc = ensure(c, c->loss_tmp, sizeof(double) * 2, "loss scalar"))) return rc;
    // an interval longer than the horizon gives the same single checkpoint
    // segment; clamping it lets the adjoint's tape be only K steps deep
    const int C = std::min(c->C, sim->K);
    const int n_ck = (sim->K + C - 1) / C;
    if (need_ckpt &&
        (rc = ensure(c, c->ckpt, sizeof(float) * idm::STATE_ROWS * (size_t)n_ck * N, "checkpoints")))
        return rc;

    SimArgs &a = P->a;
    memset(&a, 0, sizeof a);
    a.seg = (const Seg *)c->seg.p;
    a.n_seg = (const int *)c->ctl.p + CTL_NSEG;
    a.scen_tab = nullptr;
    ScenDesc &s0 = a.scen0;
    s0.veh_begin = 0;
    s0.n_veh = N;
    s0.K = sim->K;
    s0.obs_stride = obs_stride > 0 ? obs_stride : 1;
    s0.n_obs = sim->K / s0.obs_stride;
    s0.dt = sim->dt;
    s0.inv_dt = 1.0f / sim->dt;
    s0.a_min = sim->a_min;
    s0.inv_nobs = s0.n_obs > 0 ? 1.0f / (float)s0.n_obs : 0.0f;
    s0.traj_off = s0.tgt_off = s0.ckpt_off = 0;
    a.g0 = (const float *)c->g0.p;
    a.v0 = pr->v0; a.T = pr->T; a.s0 = pr->s0; a.am = pr->a_max; a.b = pr->b; a.delta = pr->delta;
    a.p_init = p_init;
    a.v_init = v_init;
    a.loss_part = (double *)c->loss_part.p;
    a.ckpt = (float *)c->ckpt.p;
    a.C = C;
    a.status = (unsigned *)c->status.p;
    a.N_total = N;
    a.G = G;
    (void)need_loss;

    CK(cudaMemsetAsync(c->ctl.p, 0, sizeof(int) * 3, st));
    CK(idm::launch_prep_gap(sc->lane_off, L, p_init, sc->length, N, (float *)c->g0.p, a.status, st));
    CK(idm::launch_build_segments(sc->lane_off, L, nullptr, 0, 32 * P->vpt * G, N, (Seg *)c->seg.p,
                                  (int *)c->ctl.p + CTL_NSEG, a.status, st));
    P->loss_per_seg = G;
    P->k_max = sim->K;
    return forward_grid(c, P, L);
}

void forward_shape(int vpt, int G, int *vpt_f, int *G_f)
{
    // the forward carries fewer live values per vehicle, so it prefers 8
    // vehicles per thread (4 pairs of independent chains) for the same
    // segment capacity, else 4
    const int cap = 32 * vpt * G;
    if (cap % 256 == 0 && cap / 256 >= 1 && cap / 256 <= 8) {
        *vpt_f = 8;
        *G_f = cap / 256;
    } else if (cap % 128 == 0 && cap / 128 >= 1 && cap / 128 <= 8) {
        *vpt_f = 4;
        *G_f = cap / 128;
    } else {
        *vpt_f = vpt;
        *G_f = G;
    }
}

int forward_grid(idm_ctx *c, Prep *P, int L)
{
    forward_shape(P->vpt, P->G, &P->vpt_f, &P->G_f);
    const int G = P->G_f;
    // 8 vehicles per thread: blocks of up to 12 warps (their register budget,
    // one block per SM); otherwise the context's warps per block
    P->wpb_f = P->vpt_f == 8 ? std::max(G, (12 / G) * G) : std::max(G, (c->wpb / G) * G);
    // few segments: fewer per block, so that they spread over more SMs
    P->wpb_f = std::min(P->wpb_f, G * std::max(1, (L + c->n_sm - 1) / c->n_sm));
    const int warps_needed = L * G;  // segments <= lanes
    const int blocks_needed = (warps_needed + P->wpb_f - 1) / P->wpb_f;
    int occ_f = idm::occupancy_blocks(P->vpt_f, G, false, false, false, false, P->wpb_f, 0);
    P->grid_f = std::min(blocks_needed, c->n_sm * occ_f);
    P->grid_f = P->grid_f < 1 ? 1 : P->grid_f;
    return IDM_OK;
}

int backward_grid(idm_ctx *c, Prep *P, bool dense, bool adam, bool want_delta, int L)
{
    const size_t smem_max = 227 * 1024;
    const size_t sm_smem = 228 * 1024;
    const int G = P->G;
    const size_t reg_cap = std::max(1, idm::backward_resident_warps(P->vpt, G) / G);  // groups per SM by registers
    auto groups_per_sm = [&](int T, bool pf) -> size_t {
        const size_t b = idm::backward_smem_bytes(P->vpt, dense, T, G, G, pf);
        return b > smem_max ? 0 : sm_smem / (b + 1024);
    };
    // tape depth: the checkpoint interval, or less when a deeper tape would
    // cost resident groups (blocks inside a checkpoint segment then restart
    // from sub-checkpoints written by an extra forward pass)
    const int C = P->a.C;  // the call's checkpoint interval (at most its longest horizon)
    int T = C;
    const size_t want = std::min(reg_cap, std::max<size_t>(groups_per_sm(1, false), 1));
    while (T > 1 && groups_per_sm(T, false) < want) --T;
    if (groups_per_sm(T, false) == 0)
        return fail(c, IDM_ERR_ARG, "adjoint tape does not fit shared memory for vpt %d x %d warps", P->vpt, G);
    // prefetching the next block doubles two stages; use it when it does not
    // cost a resident group per SM
    const bool pf = groups_per_sm(T, true) >= std::min(reg_cap, groups_per_sm(T, false));
    P->a.bwd_pf = pf ? 1 : 0;
    P->a.tape_T = T;
    if (T < C) {
        const size_t rows = (size_t)((C + T - 1) / T - 1);
        int rc;
        if ((rc = ensure(c, c->sub_ckpt, sizeof(float) * idm::STATE_ROWS * rows * (size_t)std::max(P->a.N_total, 1),
                         "sub-checkpoints")))
            return rc;
        P->a.sub_ckpt = (float *)c->sub_ckpt.p;
    } else {
        P->a.sub_ckpt = nullptr;
    }
    // compensated totals of the gradient sums (folded only past the window),
    // for the most segments the packing can produce (L: lanes of a single
    // scene, or the batch's segments)
    if (P->k_max > idm::GSUM_FOLD_STEPS && P->a.N_total > 0) {
        const long long cap = 32LL * P->vpt * G;
        const long long n_seg = std::min<long long>(
            L, 2 * (((long long)P->a.N_total + cap - 1) / cap) + idm::SEG_BUILD_CHUNKS);
        int rc;
        if ((rc = ensure(c, c->gsum, idm::gsum_bytes((size_t)n_seg, (int)cap), "gradient totals"))) return rc;
        P->a.gsum = (float *)c->gsum.p;
    } else {
        P->a.gsum = nullptr;
    }
    const size_t per_group = idm::backward_smem_bytes(P->vpt, dense, T, G, G, pf);
    int groups = std::max(1, std::min(c->wpb / G, (int)(smem_max / per_group)));
    groups = std::max(1, std::min(groups, idm::backward_max_warps(P->vpt, G) / G));
    groups = std::min(groups, std::max(1, (L + c->n_sm - 1) / c->n_sm));  // few segments: spread over the SMs
    P->wpb_b = groups * G;
    size_t smem = per_group * groups;
    int occ_b = idm::occupancy_blocks(P->vpt, G, true, dense, adam, want_delta, P->wpb_b, smem, T < C);
    int blocks_needed = (L * G + P->wpb_b - 1) / P->wpb_b;
    P->grid_b = std::min(blocks_needed, c->n_sm * occ_b);
    P->grid_b = P->grid_b < 1 ? 1 : P->grid_b;
    return IDM_OK;
}

int run_fit_graph(idm_ctx *c, Prep &P, int n_iter, size_t N, const float *box_lo, const float *box_hi, float lr0,
                  float lr1, double *loss_hist, const void *extra_key, size_t extra_len, cudaStream_t st,
                  cudaError_t (*finalize)(idm_ctx *, const Prep &, int, double *, cudaStream_t),
                  const float *eval_targets, double *eval_hist)
{
    int rc;
    if ((rc = ensure(c, c->adam_m, sizeof(float) * 5 * N, "Adam m"))) return rc;
    if ((rc = ensure(c, c->adam_v, sizeof(float) * 5 * N, "Adam v"))) return rc;
    const bool eval = eval_targets && eval_hist;
    if (eval && (rc = ensure(c, c->eval_part, sizeof(double) * (size_t)c->seg.n / sizeof(Seg) * P.G_f + 8,
                             "eval loss partials")))
        return rc;

    SimArgs &a = P.a;
    a.adam_m = (float *)c->adam_m.p;
    a.adam_v = (float *)c->adam_v.p;
    a.n_iter = n_iter;
    a.lr0 = lr0;
    a.lr1 = lr1;
    for (int q = 0; q < 5; ++q) { a.lo[q] = box_lo[q]; a.hi[q] = box_hi[q]; }

    // The graph depends on every launch argument; reuse it when they repeat.
    struct Key {
        SimArgs a;
        int vpt, G, grid_f, grid_b, wpb, wpb_b, n_iter, profiling, loss_per_seg, fwd_once;
        const double *hist;
        const float *eval_targets;
        const double *eval_hist;
        unsigned char extra[64];
    } key;
    memset(&key, 0, sizeof key);
    key.a = a;
    key.vpt = P.vpt * 16 + P.vpt_f; key.G = P.G * 16 + P.G_f; key.grid_f = P.grid_f; key.grid_b = P.grid_b; key.wpb = P.wpb_f;
    key.wpb_b = P.wpb_b; key.n_iter = n_iter; key.profiling = c->profiling; key.loss_per_seg = P.loss_per_seg;
    // With every horizon within one checkpoint interval the only checkpoint
    // is the initial state, which no iteration changes: the forward runs in
    // the first iteration only (the adjoint recomputes the steps itself).
    const bool fwd_once = !eval && P.k_max <= P.a.C;
    key.fwd_once = fwd_once;
    key.hist = loss_hist;
    key.eval_targets = eval ? eval_targets : nullptr;
    key.eval_hist = eval ? eval_hist : nullptr;
    if (extra_len > sizeof key.extra) extra_len = sizeof key.extra;
    if (extra_key) memcpy(key.extra, extra_key, extra_len);
    static_assert(sizeof(Key) <= sizeof(((idm_ctx *)0)->fit_key), "fit key too large");
    const bool cached = c->fit_exec && c->fit_key_len == sizeof key && memcmp(c->fit_key, &key, sizeof key) == 0;

    if (!cached) {
        while (c->profiling && (int)c->ev.size() < 4 * n_iter) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev.push_back(e);
        }
        // capture the whole fit (n_iter unrolled iterations) on the context's stream
        cudaStream_t cs = c->cap_stream;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(c->adam_m.p, 0, sizeof(float) * 5 * N, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_v.p, 0, sizeof(float) * 5 * N, cs);
        for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
            a.iter = it;
            const bool run_fwd = !fwd_once || it == 0;
            e = cudaMemsetAsync((int *)c->ctl.p + (run_fwd ? CTL_WORK_F : CTL_WORK_B), 0,
                                sizeof(int) * (run_fwd ? 2 : 1), cs);
            if (e == cudaSuccess && c->profiling) e = cudaEventRecordWithFlags(c->ev[4 * it], cs, cudaEventRecordExternal);
            if (e == cudaSuccess && run_fwd) {
                SimArgs af = a;
                af.work = (int *)c->ctl.p + CTL_WORK_F;
                if (eval) {
                    af.eval_targets = eval_targets;
                    af.eval_part = (double *)c->eval_part.p;
                }
                e = idm::launch_forward(P.vpt_f, P.G_f, false, false, true, af, P.grid_f, P.wpb_f, cs);
            }
            if (e == cudaSuccess && c->profiling) e = cudaEventRecordWithFlags(c->ev[4 * it + 1], cs, cudaEventRecordExternal);
            if (e == cudaSuccess && c->profiling) e = cudaEventRecordWithFlags(c->ev[4 * it + 2], cs, cudaEventRecordExternal);
            if (e == cudaSuccess) {
                a.work = (int *)c->ctl.p + CTL_WORK_B;
                e = idm::launch_backward(P.vpt, P.G, false, true, false, a, P.grid_b, P.wpb_b, cs);
            }
            if (e == cudaSuccess && c->profiling) e = cudaEventRecordWithFlags(c->ev[4 * it + 3], cs, cudaEventRecordExternal);
            if (e == cudaSuccess) e = finalize(c, P, it, loss_hist, cs);  // loss of the parameters before update it
            if (e == cudaSuccess && eval)
                e = idm::launch_loss_finalize((const double *)c->eval_part.p, a.n_seg, P.G_f, eval_hist + it, cs);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(c, e, "capturing the fit"); }
        if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
        if (c->fit_exec) {
            CK(cudaDeviceSynchronize());
            cudaGraphExecDestroy(c->fit_exec);
            c->fit_exec = nullptr;
            c->fit_key_len = 0;
        }
        e = cudaGraphInstantiate(&c->fit_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
        memcpy(c->fit_key, &key, sizeof key);
        c->fit_key_len = sizeof key;
        c->ev_used = c->profiling ? n_iter : 0;
    }
    CK(cudaGraphLaunch(c->fit_exec, st));
    return IDM_OK;
}

// Loss partials per iteration of the single launch: one per warp of the
// most segments the packing can produce (see run_fit_single).
long long single_launch_stride(const Prep &P, size_t N, int n_lanes)
{
    const long long cap = 32LL * P.vpt * P.G;
    const long long seg_bound =
        std::min<long long>(n_lanes, 2 * (((long long)N + cap - 1) / cap) + idm::SEG_BUILD_CHUNKS);
    return std::max<long long>(1, seg_bound * P.G);
}

// The fit as one persistent launch (idm_fused.cuh) for a single scene:
// clear the Adam moments and the work counter, run every iteration of every
// segment, then reduce the loss partials of all iterations.  The partials
// are sized for the most segments the packing can produce: next-fit packing
// inside each of the builder's lane chunks closes a segment only when
// the next lane would overflow it, so two consecutive segments of a chunk
// hold more than `cap` vehicles and a chunk of n vehicles gives at most
// 2n/cap + 1 segments.
int launch_single_fit(idm_ctx *c, Prep &P, int n_iter, size_t N, const float *box_lo, const float *box_hi, float lr0,
                      float lr1, long long stride, cudaStream_t st)
{
    int rc;
    if ((rc = ensure(c, c->adam_m, sizeof(float) * 5 * N, "Adam m"))) return rc;
    if ((rc = ensure(c, c->adam_v, sizeof(float) * 5 * N, "Adam v"))) return rc;
    if ((rc = ensure(c, c->fit_part, sizeof(double) * (size_t)stride * (size_t)n_iter, "fit loss partials")))
        return rc;
    SimArgs &a = P.a;
    a.adam_m = (float *)c->adam_m.p;
    a.adam_v = (float *)c->adam_v.p;
    a.n_iter = n_iter;
    a.lr0 = lr0;
    a.lr1 = lr1;
    for (int q = 0; q < 5; ++q) { a.lo[q] = box_lo[q]; a.hi[q] = box_hi[q]; }
    a.loss_part = (double *)c->fit_part.p;
    a.work = (int *)c->ctl.p + CTL_WORK_B;
    CK(cudaMemsetAsync(c->adam_m.p, 0, sizeof(float) * 5 * N, st));
    CK(cudaMemsetAsync(c->adam_v.p, 0, sizeof(float) * 5 * N, st));
    CK(cudaMemsetAsync(a.work, 0, sizeof(int), st));
    CK(idm::launch_fit_fused(P.vpt, P.G, a, stride, P.grid_b, P.wpb_b, st));
    return IDM_OK;
}

int run_fit_single(idm_ctx *c, Prep &P, int n_iter, size_t N, int n_lanes, const float *box_lo, const float *box_hi,
                   float lr0, float lr1, double *loss_hist, cudaStream_t st)
{
    const long long stride = single_launch_stride(P, N, n_lanes);
    int rc;
    if ((rc = launch_single_fit(c, P, n_iter, N, box_lo, box_hi, lr0, lr1, stride, st))) return rc;
    if (loss_hist)
        CK(idm::launch_loss_finalize_iters(P.a.loss_part, stride, P.a.n_seg, P.loss_per_seg, n_iter, loss_hist, st));
    return IDM_OK;
}

}  // namespace abi
}  // namespace idm

namespace {

// Loss of a single-scene fit iteration: fixed-order sum of the per-warp partials.
cudaError_t single_finalize(idm_ctx *c, const Prep &P, int it, double *hist, cudaStream_t st)
{
    (void)c;
    return idm::launch_loss_finalize(P.a.loss_part, P.a.n_seg, P.loss_per_seg, hist ? hist + it : nullptr, st);
}

}  // namespace

extern "C" {

int idm_max_lane_supported(void) { return 2048; }

int idm_ctx_create(idm_ctx_t **ctx, size_t workspace_cap_bytes)
{
    if (!ctx) return IDM_ERR_ARG;
    *ctx = nullptr;
    idm_ctx *c = new (std::nothrow) idm_ctx();
    if (!c) return IDM_ERR_WORKSPACE;
    c->cap = workspace_cap_bytes;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return IDM_ERR_CUDA;
    }
    *ctx = c;
    return IDM_OK;
}

int idm_ctx_destroy(idm_ctx_t *c)
{
    if (!c) return IDM_OK;
    cudaDeviceSynchronize();
    if (c->fit_exec) cudaGraphExecDestroy(c->fit_exec);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    Buf *bufs[] = {&c->seg,      &c->ctl,        &c->status,       &c->g0,           &c->ckpt,
                   &c->loss_part, &c->loss_tmp,  &c->adam_m,       &c->adam_v,       &c->lay_counts,
                   &c->lay_cursor, &c->eval_part, &c->sub_ckpt,    &c->scen_tab,     &c->scen_seg_off,
                   &c->scen_seg_idx, &c->lane_off_dev, &c->rec_oyy, &c->rec_oyc,    &c->rec_tape,
                   &c->rec_mom,  &c->rec_thm,    &c->rec_acc,      &c->rec_kmax,     &c->rec_multi,
                   &c->fit_part, &c->gsum};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return IDM_OK;
}

const char *idm_last_error(const idm_ctx_t *c) { return c ? c->err : "no context"; }

int idm_set_tuning(idm_ctx_t *c, int vpt, int warps_per_segment, int ckpt_interval, int warps_per_block)
{
    if (!c) return IDM_ERR_ARG;
    if (!(vpt == 0 || vpt == 2 || vpt == 4 || vpt == 8))
        return fail(c, IDM_ERR_ARG, "vpt must be 0, 2, 4 or 8");
    if (!(warps_per_segment == 0 || warps_per_segment == 1 || warps_per_segment == 2 || warps_per_segment == 4 ||
          warps_per_segment == 8))
        return fail(c, IDM_ERR_ARG, "warps_per_segment must be 0, 1, 2, 4 or 8");
    if (ckpt_interval < 1 || ckpt_interval > 64) return fail(c, IDM_ERR_ARG, "ckpt_interval must be in [1, 64]");
    if (warps_per_block < 1 || warps_per_block > 16) return fail(c, IDM_ERR_ARG, "warps_per_block must be in [1, 16]");
    c->vpt_req = vpt;
    c->G_req = warps_per_segment;
    c->C = ckpt_interval;
    c->wpb = warps_per_block;
    return IDM_OK;
}

int idm_set_fit_mode(idm_ctx_t *c, int mode)
{
    if (!c) return IDM_ERR_ARG;
    if (mode != IDM_FIT_AUTO && mode != IDM_FIT_GRAPH && mode != IDM_FIT_SINGLE_LAUNCH)
        return fail(c, IDM_ERR_ARG, "fit mode must be IDM_FIT_AUTO, IDM_FIT_GRAPH or IDM_FIT_SINGLE_LAUNCH");
    c->fit_mode = mode;
    return IDM_OK;
}

int idm_last_fit_form(const idm_ctx_t *c) { return c ? c->last_fit_form : 0; }

size_t idm_workspace_bytes(const idm_ctx_t *c, const idm_scene_t *s, const idm_sim_t *sim)
{
    if (!c || !s || !sim || sim->K < 1) return 0;
    size_t N = (size_t)s->n_vehicles, L = (size_t)s->n_lanes;
    const int C = std::min(c->C, sim->K);
    size_t n_ck = (size_t)((sim->K + C - 1) / C);
    // sub-checkpoints when the adjoint's tape is shallower than the interval
    // (at most ceil(C/2) - 1 rows; typically none for C <= 8)
    const size_t sub = C > 8 ? (size_t)((C + 1) / 2 - 1) : 0;
    const size_t cap = 512;  // default segment capacity
    const size_t totals =
        sim->K > idm::GSUM_FOLD_STEPS ? idm::gsum_bytes(std::min(L, 2 * ((N + cap - 1) / cap) + 1024), (int)cap) : 0;
    const size_t sb = sizeof(float) * idm::STATE_ROWS;  // bytes of one stored state
    return sizeof(Seg) * L + sizeof(int) * CTL_N + 16 + 4 * N + 8 * 8 * L + 16 + sb * n_ck * N + sb * sub * N +
           totals;
}

int idm_status(idm_ctx_t *c, uint32_t *flags, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    unsigned h = 0;
    if (c->status.p) {
        CK(cudaMemcpy(&h, c->status.p, sizeof h, cudaMemcpyDeviceToHost));
        CK(cudaMemset(c->status.p, 0, sizeof(unsigned)));
    }
    if (flags) *flags = h;
    if (h & (IDM_STATUS_LANE_TOO_LONG | IDM_STATUS_BAD_LANE_OFF))
        return fail(c, IDM_ERR_LANE, "device status 0x%x: lane longer than the segment or malformed lanes", h);
    if (h & IDM_STATUS_NONFINITE) return fail(c, IDM_ERR_NONFINITE, "device status 0x%x: non-finite value", h);
    if (h & IDM_STATUS_BAD_OBS)
        return fail(c, IDM_ERR_OBS, "device status 0x%x: malformed observations or horizons", h);
    if (h & IDM_STATUS_BAD_LANES)
        return fail(c, IDM_ERR_LANES, "device status 0x%x: malformed lane polylines or lane index", h);
    return IDM_OK;
}

int idm_set_event_counting(idm_ctx_t *c, int on)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = ensure_status(c))) return rc;
    c->count_events = on ? 1 : 0;
    return IDM_OK;
}

int idm_event_counts(idm_ctx_t *c, void *stream, uint64_t *gap_floor_hits, uint64_t *kink_near)
{
    if (!c) return IDM_ERR_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long h[2] = {0, 0};
    if (c->status.p) {
        char *p = static_cast<char *>(c->status.p) + STATUS_EVENTS_OFF;
        CK(cudaMemcpy(h, p, sizeof h, cudaMemcpyDeviceToHost));
        CK(cudaMemset(p, 0, sizeof h));
    }
    if (gap_floor_hits) *gap_floor_hits = h[0];
    if (kink_near) *kink_near = h[1];
    return IDM_OK;
}

int idm_layout(idm_ctx_t *c, int32_t N, int32_t n_lanes, const int32_t *lane_id, const float *pos, int32_t *perm,
               int32_t *lane_off, int32_t *max_lane_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (N < 0 || n_lanes < 1) return fail(c, IDM_ERR_ARG, "need N >= 0 and n_lanes >= 1");
    if (N > 0 && (!lane_id || !pos || !perm)) return fail(c, IDM_ERR_ARG, "lane_id, pos and perm are required");
    if (!lane_off) return fail(c, IDM_ERR_ARG, "lane_off is required");
    int rc;
    if ((rc = ensure_status(c))) return rc;
    if ((rc = ensure(c, c->lay_counts, sizeof(int) * (size_t)n_lanes, "layout counts"))) return rc;
    if ((rc = ensure(c, c->lay_cursor, sizeof(int) * (size_t)n_lanes, "layout cursor"))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(idm::launch_layout(N, n_lanes, lane_id, pos, perm, lane_off, max_lane_out, (int *)c->lay_counts.p,
                          (int *)c->lay_cursor.p, (unsigned *)c->status.p, st));
    return IDM_OK;
}

int idm_gather(idm_ctx_t *c, int32_t N, const int32_t *perm, int count, const float *const *srcs,
               float *const *dsts, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (N < 0 || count < 0) return fail(c, IDM_ERR_ARG, "N and count must be >= 0");
    if (N > 0 && count > 0 && (!perm || !srcs || !dsts)) return fail(c, IDM_ERR_ARG, "perm, srcs, dsts required");
    for (int q = 0; q < count; ++q)
        if (!srcs[q] || !dsts[q]) return fail(c, IDM_ERR_ARG, "array %d is NULL", q);
    CK(idm::launch_gather(N, perm, count, srcs, dsts, (cudaStream_t)stream));
    return IDM_OK;
}

int idm_forward(idm_ctx_t *c, const idm_scene_t *scene, const idm_params_t *params, const float *p_init,
                const float *v_init, const idm_sim_t *sim, float *traj, float *vtraj, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_scene(c, scene)) || (rc = check_params(c, params, true, scene->n_vehicles)) || (rc = check_sim(c, sim))) return rc;
    if (scene->n_vehicles > 0 && (!p_init || !v_init)) return fail(c, IDM_ERR_ARG, "p_init and v_init are required");
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    if ((rc = prepare(c, scene, params, p_init, v_init, sim, false, false, 1, &P, st))) return rc;
    P.a.work = (int *)c->ctl.p + CTL_WORK_F;
    P.a.traj = traj;
    P.a.vtraj = vtraj;
    P.a.events = event_counters(c);
    CK(idm::launch_forward(P.vpt_f, P.G_f, traj != nullptr, vtraj != nullptr, false, P.a, P.grid_f, P.wpb_f, st));
    return IDM_OK;
}

int idm_backward(idm_ctx_t *c, const idm_scene_t *scene, const idm_params_t *params, const float *p_init,
                 const float *v_init, const idm_sim_t *sim, const float *gP, const float *gV, idm_params_t *grad,
                 float *grad_p_init, float *grad_v_init, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_scene(c, scene)) || (rc = check_params(c, params, true, scene->n_vehicles)) || (rc = check_sim(c, sim))) return rc;
    if (scene->n_vehicles > 0 && (!p_init || !v_init || !gP))
        return fail(c, IDM_ERR_ARG, "p_init, v_init and gP are required");
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    if ((rc = prepare(c, scene, params, p_init, v_init, sim, true, false, 1, &P, st))) return rc;
    if ((rc = backward_grid(c, &P, true, false, grad && grad->delta, scene->n_lanes))) return rc;
    P.a.work = (int *)c->ctl.p + CTL_WORK_F;
    CK(idm::launch_forward(P.vpt_f, P.G_f, false, false, true, P.a, P.grid_f, P.wpb_f, st));
    P.a.work = (int *)c->ctl.p + CTL_WORK_B;
    P.a.gP = gP;
    P.a.gV = gV;
    if (grad) {
        P.a.g_v0 = grad->v0; P.a.g_T = grad->T; P.a.g_s0 = grad->s0;
        P.a.g_am = grad->a_max; P.a.g_b = grad->b; P.a.g_delta = grad->delta;
    }
    P.a.g_p_init = grad_p_init;
    P.a.g_v_init = grad_v_init;
    CK(idm::launch_backward(P.vpt, P.G, true, false, grad && grad->delta, P.a, P.grid_b, P.wpb_b, st));
    return IDM_OK;
}

int idm_loss_grad(idm_ctx_t *c, const idm_scene_t *scene, const idm_params_t *params, const float *p_init,
                  const float *v_init, const idm_sim_t *sim, const float *targets, int32_t obs_stride,
                  double *loss_out, idm_params_t *grad, float *grad_p_init, float *grad_v_init, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_scene(c, scene)) || (rc = check_params(c, params, true, scene->n_vehicles)) || (rc = check_sim(c, sim))) return rc;
    if (obs_stride < 1) return fail(c, IDM_ERR_ARG, "obs_stride must be >= 1");
    if (scene->n_vehicles > 0 && (!p_init || !v_init)) return fail(c, IDM_ERR_ARG, "p_init and v_init are required");
    if (sim->K / obs_stride > 0 && scene->n_vehicles > 0 && !targets)
        return fail(c, IDM_ERR_ARG, "targets are required");
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    if ((rc = prepare(c, scene, params, p_init, v_init, sim, true, true, obs_stride, &P, st))) return rc;
    const bool want_delta = grad && grad->delta;
    if ((rc = backward_grid(c, &P, false, false, want_delta, scene->n_lanes))) return rc;
    P.a.targets = targets;
    P.a.work = (int *)c->ctl.p + CTL_WORK_F;
    CK(idm::launch_forward(P.vpt_f, P.G_f, false, false, true, P.a, P.grid_f, P.wpb_f, st));
    P.a.work = (int *)c->ctl.p + CTL_WORK_B;
    if (grad) {
        P.a.g_v0 = grad->v0; P.a.g_T = grad->T; P.a.g_s0 = grad->s0;
        P.a.g_am = grad->a_max; P.a.g_b = grad->b; P.a.g_delta = grad->delta;
    }
    P.a.g_p_init = grad_p_init;
    P.a.g_v_init = grad_v_init;
    CK(idm::launch_backward(P.vpt, P.G, false, false, want_delta, P.a, P.grid_b, P.wpb_b, st));
    CK(idm::launch_loss_finalize(P.a.loss_part, P.a.n_seg, P.G, loss_out ? loss_out : (double *)c->loss_tmp.p, st));
    return IDM_OK;
}

int idm_fit(idm_ctx_t *c, const idm_scene_t *scene, idm_params_t *params, const float *p_init, const float *v_init,
            const idm_sim_t *sim, const float *targets, int32_t obs_stride, int32_t n_iter, float lr0, float lr1,
            const float *box_lo, const float *box_hi, double *loss_hist, void *stream)
{
    return idm_fit_eval(c, scene, params, p_init, v_init, sim, targets, obs_stride, n_iter, lr0, lr1, box_lo, box_hi,
                        loss_hist, nullptr, nullptr, stream);
}

int idm_fit_eval(idm_ctx_t *c, const idm_scene_t *scene, idm_params_t *params, const float *p_init,
                 const float *v_init, const idm_sim_t *sim, const float *targets, int32_t obs_stride, int32_t n_iter,
                 float lr0, float lr1, const float *box_lo, const float *box_hi, double *loss_hist,
                 const float *eval_targets, double *eval_hist, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if ((eval_targets == nullptr) != (eval_hist == nullptr))
        return fail(c, IDM_ERR_ARG, "eval_targets and eval_hist must be given together");
    int rc;
    if ((rc = check_scene(c, scene)) || (rc = check_params(c, params, true, scene->n_vehicles)) || (rc = check_sim(c, sim))) return rc;
    if (obs_stride < 1) return fail(c, IDM_ERR_ARG, "obs_stride must be >= 1");
    if (n_iter < 0 || n_iter > 100000) return fail(c, IDM_ERR_ARG, "n_iter must be in [0, 100000]");
    if (!box_lo || !box_hi) return fail(c, IDM_ERR_ARG, "box_lo and box_hi (host) are required");
    for (int q = 0; q < 5; ++q)
        if (!(box_lo[q] <= box_hi[q])) return fail(c, IDM_ERR_ARG, "box_lo[%d] > box_hi[%d]", q, q);
    if (!(lr0 >= 0.0f) || !(lr1 >= 0.0f)) return fail(c, IDM_ERR_ARG, "learning rates must be >= 0");
    if (scene->n_vehicles > 0 && (!p_init || !v_init)) return fail(c, IDM_ERR_ARG, "p_init and v_init are required");
    if (sim->K / obs_stride > 0 && scene->n_vehicles > 0 && !targets)
        return fail(c, IDM_ERR_ARG, "targets are required");
    if (n_iter == 0) return IDM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    if ((rc = prepare(c, scene, params, p_init, v_init, sim, true, true, obs_stride, &P, st))) return rc;
    if ((rc = backward_grid(c, &P, false, true, false, scene->n_lanes))) return rc;
    P.a.targets = targets;
    const double vehicle_steps = (double)scene->n_vehicles * (double)sim->K;
    const double partial_bytes =
        8.0 * (double)n_iter * (double)single_launch_stride(P, (size_t)scene->n_vehicles, scene->n_lanes);
    const bool single = !eval_targets && !c->profiling &&
                        (c->fit_mode == IDM_FIT_SINGLE_LAUNCH ||
                         (c->fit_mode == IDM_FIT_AUTO && partial_bytes <= IDM_SINGLE_LAUNCH_MAX_PARTIAL_BYTES &&
                          (sim->K <= c->C || vehicle_steps <= IDM_SINGLE_LAUNCH_MAX_VEHICLE_STEPS)));
    c->last_fit_form = single ? IDM_FIT_SINGLE_LAUNCH : IDM_FIT_GRAPH;
    if (single)
        return run_fit_single(c, P, n_iter, (size_t)scene->n_vehicles, scene->n_lanes, box_lo, box_hi, lr0, lr1,
                              loss_hist, st);
    return run_fit_graph(c, P, n_iter, (size_t)scene->n_vehicles, box_lo, box_hi, lr0, lr1, loss_hist, nullptr, 0,
                         st, single_finalize, eval_targets, eval_hist);
}

int idm_set_profiling(idm_ctx_t *c, int on)
{
    if (!c) return IDM_ERR_ARG;
    c->profiling = on ? 1 : 0;
    return IDM_OK;
}

int idm_phase_times(idm_ctx_t *c, void *stream, double *fwd_ms, double *bwd_ms, int32_t *n_launches)
{
    if (!c) return IDM_ERR_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    double f = 0.0, b = 0.0;
    for (int it = 0; it < c->ev_used; ++it) {
        float x = 0.0f, y = 0.0f;
        CK(cudaEventElapsedTime(&x, c->ev[4 * it], c->ev[4 * it + 1]));
        CK(cudaEventElapsedTime(&y, c->ev[4 * it + 2], c->ev[4 * it + 3]));
        f += x;
        b += y;
    }
    if (fwd_ms) *fwd_ms = f;
    if (bwd_ms) *bwd_ms = b;
    if (n_launches) *n_launches = c->ev_used;
    return IDM_OK;
}

int idm_gather_rows(idm_ctx_t *c, int32_t N, int32_t n_rows, const int32_t *perm, const float *src, float *dst,
                    void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (N < 0 || n_rows < 0) return fail(c, IDM_ERR_ARG, "N and n_rows must be >= 0");
    if (N > 0 && n_rows > 0 && (!perm || !src || !dst)) return fail(c, IDM_ERR_ARG, "perm, src and dst are required");
    CK(idm::launch_gather_rows(N, n_rows, perm, src, dst, (cudaStream_t)stream));
    return IDM_OK;
}

}  // extern "C"
