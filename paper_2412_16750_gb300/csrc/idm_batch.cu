// Batched uneven scenarios (C-ABI, include/idm.h): many independent scenes,
// each with its own lanes, horizon K_s, step dt_s and observation stride,
// simulated and differentiated by ONE persistent launch of the same kernels
// as the single-scene path.  The host plans the launch: a scenario table
// (offsets of every scenario's trajectories, targets and checkpoints), the
// packing of each scenario's lanes into warp segments, and a
// longest-processing-time-first order of the segments (cost = K_s x slots).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/idm.h"
#include "idm_ctx.h"
#include "idm_internal.h"

using idm::ScenDesc;
using idm::Seg;
using idm::SimArgs;
using namespace idm::abi;

#define CK(call) IDM_CK(call)

namespace {

struct BatchPlan {
    std::vector<ScenDesc> scen;
    std::vector<Seg> seg;
    std::vector<int> scen_seg_off;  // CSR: segments of scenario s (indices into seg)
    std::vector<int> scen_seg_idx;
    long long traj_elems = 0, tgt_elems = 0, ckpt_elems = 0;
    int max_lane = 0;
    int max_K = 0;
};

int check_batch(idm_ctx *c, const idm_batch_t *b)
{
    if (!b) return fail(c, IDM_ERR_ARG, "batch is NULL");
    if (b->n_scen < 1) return fail(c, IDM_ERR_ARG, "n_scen must be >= 1");
    if (b->n_lanes < 1 || b->n_vehicles < 0) return fail(c, IDM_ERR_ARG, "need n_lanes >= 1, n_vehicles >= 0");
    if (!b->scen_lane_off || !b->K || !b->dt || !b->lane_off_host || !b->lane_off)
        return fail(c, IDM_ERR_ARG, "scen_lane_off, K, dt, lane_off_host and lane_off are required");
    if (b->n_vehicles > 0 && !b->length) return fail(c, IDM_ERR_ARG, "length is NULL");
    if (!(b->a_min < 0.0f) || !std::isfinite(b->a_min)) return fail(c, IDM_ERR_ARG, "a_min must be finite and < 0");
    if (b->scen_lane_off[0] != 0 || b->scen_lane_off[b->n_scen] != b->n_lanes)
        return fail(c, IDM_ERR_ARG, "scen_lane_off must run from 0 to n_lanes");
    if (b->lane_off_host[0] != 0 || b->lane_off_host[b->n_lanes] != b->n_vehicles)
        return fail(c, IDM_ERR_ARG, "lane_off must run from 0 to n_vehicles");
    for (int l = 0; l < b->n_lanes; ++l)
        if (b->lane_off_host[l + 1] < b->lane_off_host[l]) return fail(c, IDM_ERR_ARG, "lane_off not monotone at %d", l);
    for (int s = 0; s < b->n_scen; ++s) {
        if (b->scen_lane_off[s + 1] < b->scen_lane_off[s])
            return fail(c, IDM_ERR_ARG, "scen_lane_off not monotone at %d", s);
        if (b->K[s] < 1) return fail(c, IDM_ERR_ARG, "K[%d] must be >= 1", s);
        if (!(b->dt[s] > 0.0f) || !std::isfinite(b->dt[s])) return fail(c, IDM_ERR_ARG, "dt[%d] must be > 0", s);
        if (b->obs_stride && b->obs_stride[s] < 1) return fail(c, IDM_ERR_ARG, "obs_stride[%d] must be >= 1", s);
    }
    return IDM_OK;
}

// Scenario table, warp segments (packed per scenario, LPT order) and sizes.
void plan_batch(const idm_batch_t *b, int C, int cap, BatchPlan &P)
{
    const int S = b->n_scen;
    P.scen.resize(S);
    P.seg.clear();
    long long traj = 0, tgt = 0, ck = 0;
    std::vector<long long> cost;
    std::vector<int> seg_scen;
    for (int s = 0; s < S; ++s) {
        ScenDesc &d = P.scen[s];
        memset(&d, 0, sizeof d);
        const int l0 = b->scen_lane_off[s], l1 = b->scen_lane_off[s + 1];
        d.veh_begin = b->lane_off_host[l0];
        d.n_veh = b->lane_off_host[l1] - d.veh_begin;
        d.K = b->K[s];
        d.obs_stride = b->obs_stride ? b->obs_stride[s] : 1;
        d.n_obs = d.K / d.obs_stride;
        d.dt = b->dt[s];
        d.inv_dt = 1.0f / d.dt;
        d.a_min = b->a_min;
        d.inv_nobs = d.n_obs > 0 ? 1.0f / (float)d.n_obs : 0.0f;
        d.traj_off = traj;
        d.tgt_off = tgt;
        d.ckpt_off = ck;
        traj += (long long)(d.K + 1) * d.n_veh;
        tgt += (long long)d.n_obs * d.n_veh;
        ck += (long long)idm::STATE_ROWS * ((d.K + C - 1) / C) * d.n_veh;
        P.max_K = std::max(P.max_K, d.K);
        // greedy packing of this scenario's lanes
        int fill = 0, begin = 0;
        for (int l = l0; l < l1; ++l) {
            const int a = b->lane_off_host[l], n = b->lane_off_host[l + 1] - a;
            P.max_lane = std::max(P.max_lane, n);
            if (n == 0) continue;
            if (fill > 0 && fill + n > cap) {
                P.seg.push_back(Seg{begin, fill, s, 0});
                fill = 0;
            }
            if (fill == 0) begin = a;
            fill += n;
        }
        if (fill > 0) P.seg.push_back(Seg{begin, fill, s, 0});
    }
    P.traj_elems = traj;
    P.tgt_elems = tgt;
    P.ckpt_elems = ck;
    // longest first: cost = steps x occupied slots
    std::vector<int> order(P.seg.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const long long cx = (long long)P.scen[P.seg[x].scen].K * P.seg[x].n_veh;
        const long long cy = (long long)P.scen[P.seg[y].scen].K * P.seg[y].n_veh;
        return cx > cy;
    });
    std::vector<Seg> sorted(P.seg.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = P.seg[order[i]];
    P.seg.swap(sorted);
    // CSR of segment indices per scenario (fixed order -> deterministic loss)
    P.scen_seg_off.assign(S + 1, 0);
    for (const Seg &g : P.seg) P.scen_seg_off[g.scen + 1] += 1;
    for (int s = 0; s < S; ++s) P.scen_seg_off[s + 1] += P.scen_seg_off[s];
    P.scen_seg_idx.assign(P.seg.size(), 0);
    std::vector<int> cur(P.scen_seg_off.begin(), P.scen_seg_off.end() - 1);
    for (int i = 0; i < (int)P.seg.size(); ++i) P.scen_seg_idx[cur[P.seg[i].scen]++] = i;
}

// Upload the plan and build the launch arguments of a batched call.
int prepare_batch(idm_ctx *c, const idm_batch_t *b, const idm_params_t *pr, const float *p_init, const float *v_init,
                  bool need_ckpt, Prep *Pp, BatchPlan &BP, cudaStream_t st)
{
    int rc;
    // shape from the longest lane (needs a host pass over the lanes first)
    int max_lane = 0;
    for (int l = 0; l < b->n_lanes; ++l) max_lane = std::max(max_lane, b->lane_off_host[l + 1] - b->lane_off_host[l]);
    if (max_lane > idm_max_lane_supported())
        return fail(c, IDM_ERR_ARG, "a lane has %d vehicles, more than %d", max_lane, idm_max_lane_supported());
    if ((rc = pick_shape(c, max_lane, b->n_vehicles, b->n_lanes, &Pp->vpt, &Pp->G))) return rc;
    const int G = Pp->G;
    // the checkpoint interval, at most the longest horizon (same segments,
    // shallower adjoint tape)
    int max_K = 1;
    for (int s = 0; s < b->n_scen; ++s) max_K = std::max(max_K, b->K[s]);
    const int C = std::min(c->C, max_K);
    plan_batch(b, C, 32 * Pp->vpt * G, BP);
    const int N = b->n_vehicles, L = b->n_lanes, S = b->n_scen;
    const size_t n_seg = BP.seg.size();
    if ((rc = ensure(c, c->seg, sizeof(Seg) * std::max<size_t>(n_seg, 1), "segments"))) return rc;
    if ((rc = ensure(c, c->ctl, sizeof(int) * CTL_N, "control"))) return rc;
    if ((rc = ensure_status(c))) return rc;
    if ((rc = ensure(c, c->g0, sizeof(float) * (size_t)N, "initial gaps"))) return rc;
    if ((rc = ensure(c, c->loss_part, sizeof(double) * std::max<size_t>(n_seg, 1) * G, "loss partials"))) return rc;
    if ((rc = ensure(c, c->loss_tmp, sizeof(double) * 2, "loss scalar"))) return rc;
    if ((rc = ensure(c, c->scen_tab, sizeof(ScenDesc) * S, "scenario table"))) return rc;
    if ((rc = ensure(c, c->scen_seg_off, sizeof(int) * (S + 1), "scenario segments"))) return rc;
    if ((rc = ensure(c, c->scen_seg_idx, sizeof(int) * std::max<size_t>(n_seg, 1), "scenario segment list"))) return rc;
    if (need_ckpt && (rc = ensure(c, c->ckpt, sizeof(float) * (size_t)BP.ckpt_elems, "checkpoints"))) return rc;

    // pageable host -> device copies complete before returning
    CK(cudaMemcpyAsync(c->scen_tab.p, BP.scen.data(), sizeof(ScenDesc) * S, cudaMemcpyHostToDevice, st));
    if (n_seg) CK(cudaMemcpyAsync(c->seg.p, BP.seg.data(), sizeof(Seg) * n_seg, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->scen_seg_off.p, BP.scen_seg_off.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice, st));
    if (n_seg)
        CK(cudaMemcpyAsync(c->scen_seg_idx.p, BP.scen_seg_idx.data(), sizeof(int) * n_seg, cudaMemcpyHostToDevice, st));
    int ctl0[3] = {(int)n_seg, 0, 0};
    CK(cudaMemcpyAsync(c->ctl.p, ctl0, sizeof ctl0, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // the host plan may be released after return

    SimArgs &a = Pp->a;
    memset(&a, 0, sizeof a);
    a.seg = (const Seg *)c->seg.p;
    a.n_seg = (const int *)c->ctl.p + CTL_NSEG;
    a.scen_tab = (const ScenDesc *)c->scen_tab.p;
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
    Pp->loss_per_seg = G;
    Pp->k_max = max_K;
    CK(idm::launch_prep_gap(b->lane_off, L, p_init, b->length, N, (float *)c->g0.p, a.status, st));
    return forward_grid(c, Pp, (int)std::max<size_t>(n_seg, 1));
}

// Per-scenario losses: one thread per scenario sums its segments' per-warp
// partials in a fixed order.  The batch total is the sum of every segment's
// partials (each segment belongs to one scenario), reduced in parallel by
// launch_loss_finalize as for a single scene.
__global__ void scen_loss_kernel(const double *part, int per_seg, const int *seg_off, const int *seg_idx, int S,
                                 double *scen_loss)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = seg_off[s]; i < seg_off[s + 1]; ++i)
            for (int w = 0; w < per_seg; ++w) acc += part[(size_t)seg_idx[i] * per_seg + w];
        scen_loss[s] = acc;
    }
}

struct BatchFinalize {
    int S;
    double *scen_loss;  // per-scenario output of the last iteration (may be NULL)
};
thread_local BatchFinalize g_bfin;

cudaError_t batch_finalize(idm_ctx *c, const Prep &P, int it, double *hist, cudaStream_t st)
{
    const int S = g_bfin.S;
    if (g_bfin.scen_loss)
        scen_loss_kernel<<<(S + 255) / 256, 256, 0, st>>>(P.a.loss_part, P.loss_per_seg, (const int *)c->scen_seg_off.p,
                                                          (const int *)c->scen_seg_idx.p, S, g_bfin.scen_loss);
    if (hist) return idm::launch_loss_finalize(P.a.loss_part, P.a.n_seg, P.loss_per_seg, hist + it, st);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int idm_batch_sizes(const idm_batch_t *b, int ckpt_interval, int64_t *traj_elems, int64_t *target_elems,
                    int64_t *ckpt_elems)
{
    if (!b || b->n_scen < 1 || !b->scen_lane_off || !b->K || !b->lane_off_host || ckpt_interval < 1) return IDM_ERR_ARG;
    BatchPlan P;
    for (int s = 0; s < b->n_scen; ++s)
        if (b->K[s] < 1 || (b->obs_stride && b->obs_stride[s] < 1)) return IDM_ERR_ARG;
    plan_batch(b, ckpt_interval, 1 << 30, P);
    if (traj_elems) *traj_elems = P.traj_elems;
    if (target_elems) *target_elems = P.tgt_elems;
    if (ckpt_elems) *ckpt_elems = P.ckpt_elems;
    return IDM_OK;
}

int idm_batch_forward(idm_ctx_t *c, const idm_batch_t *b, const idm_params_t *params, const float *p_init,
                      const float *v_init, float *traj, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(c, b)) || (rc = check_params(c, params, true, b->n_vehicles))) return rc;
    if (b->n_vehicles > 0 && (!p_init || !v_init || !traj))
        return fail(c, IDM_ERR_ARG, "p_init, v_init and traj are required");
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    BatchPlan BP;
    if ((rc = prepare_batch(c, b, params, p_init, v_init, false, &P, BP, st))) return rc;
    P.a.work = (int *)c->ctl.p + CTL_WORK_F;
    P.a.traj = traj;
    P.a.events = event_counters(c);
    CK(idm::launch_forward(P.vpt_f, P.G_f, true, false, false, P.a, P.grid_f, P.wpb_f, st));
    return IDM_OK;
}

int idm_batch_loss_grad(idm_ctx_t *c, const idm_batch_t *b, const idm_params_t *params, const float *p_init,
                        const float *v_init, const float *targets, double *scen_loss, double *loss_total,
                        idm_params_t *grad, float *grad_p_init, float *grad_v_init, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(c, b)) || (rc = check_params(c, params, true, b->n_vehicles))) return rc;
    if (b->n_vehicles > 0 && (!p_init || !v_init || !targets))
        return fail(c, IDM_ERR_ARG, "p_init, v_init and targets are required");
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    BatchPlan BP;
    if ((rc = prepare_batch(c, b, params, p_init, v_init, true, &P, BP, st))) return rc;
    const bool want_delta = grad && grad->delta;
    if ((rc = backward_grid(c, &P, false, false, want_delta, (int)std::max<size_t>(BP.seg.size(), 1)))) return rc;
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
    g_bfin = BatchFinalize{b->n_scen, scen_loss};
    CK(batch_finalize(c, P, 0, loss_total, st));
    return IDM_OK;
}

int idm_batch_fit(idm_ctx_t *c, const idm_batch_t *b, idm_params_t *params, const float *p_init, const float *v_init,
                  const float *targets, int32_t n_iter, float lr0, float lr1, const float *box_lo, const float *box_hi,
                  double *loss_hist, double *scen_loss, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(c, b)) || (rc = check_params(c, params, true, b->n_vehicles))) return rc;
    if (n_iter < 0 || n_iter > 100000) return fail(c, IDM_ERR_ARG, "n_iter must be in [0, 100000]");
    if (!box_lo || !box_hi) return fail(c, IDM_ERR_ARG, "box_lo and box_hi (host) are required");
    for (int q = 0; q < 5; ++q)
        if (!(box_lo[q] <= box_hi[q])) return fail(c, IDM_ERR_ARG, "box_lo[%d] > box_hi[%d]", q, q);
    if (!(lr0 >= 0.0f) || !(lr1 >= 0.0f)) return fail(c, IDM_ERR_ARG, "learning rates must be >= 0");
    if (b->n_vehicles > 0 && (!p_init || !v_init || !targets))
        return fail(c, IDM_ERR_ARG, "p_init, v_init and targets are required");
    if (n_iter == 0) return IDM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Prep P;
    BatchPlan BP;
    if ((rc = prepare_batch(c, b, params, p_init, v_init, true, &P, BP, st))) return rc;
    if ((rc = backward_grid(c, &P, false, true, false, (int)std::max<size_t>(BP.seg.size(), 1)))) return rc;
    P.a.targets = targets;
    P.k_max = BP.max_K;
    // the form (see idm_set_fit_mode): the single launch needs the partials
    // of every iteration, one per warp of every segment (their number is
    // known here)
    const int S = b->n_scen;
    const long long stride = std::max<long long>(1, (long long)BP.seg.size() * P.G);
    double vehicle_steps = 0.0;
    for (int q = 0; q < S; ++q) vehicle_steps += (double)BP.scen[q].n_veh * (double)BP.scen[q].K;
    const bool single = !c->profiling &&
                        (c->fit_mode == IDM_FIT_SINGLE_LAUNCH ||
                         (c->fit_mode == IDM_FIT_AUTO &&
                          8.0 * (double)stride * (double)n_iter <= IDM_SINGLE_LAUNCH_MAX_PARTIAL_BYTES &&
                          (BP.max_K <= c->C || vehicle_steps <= IDM_SINGLE_LAUNCH_MAX_VEHICLE_STEPS)));
    c->last_fit_form = single ? IDM_FIT_SINGLE_LAUNCH : IDM_FIT_GRAPH;
    if (single) {
        if ((rc = launch_single_fit(c, P, n_iter, (size_t)b->n_vehicles, box_lo, box_hi, lr0, lr1, stride, st)))
            return rc;
        const SimArgs &a = P.a;
        const int *seg_off = (const int *)c->scen_seg_off.p, *seg_idx = (const int *)c->scen_seg_idx.p;
        if (loss_hist) CK(idm::launch_loss_finalize_iters(a.loss_part, stride, a.n_seg, P.loss_per_seg, n_iter, loss_hist, st));
        if (scen_loss)
            scen_loss_kernel<<<(S + 255) / 256, 256, 0, st>>>(a.loss_part + (size_t)(n_iter - 1) * (size_t)stride,
                                                              P.loss_per_seg, seg_off, seg_idx, S, scen_loss);
        CK(cudaGetLastError());
        return IDM_OK;
    }
    g_bfin = BatchFinalize{b->n_scen, scen_loss};
    struct {
        int S;
        double *scen_loss;
    } extra = {b->n_scen, scen_loss};
    return run_fit_graph(c, P, n_iter, (size_t)b->n_vehicles, box_lo, box_hi, lr0, lr1, loss_hist, &extra,
                         sizeof extra, st, batch_finalize);
}

}  // extern "C"
