// The whole Adam fit (arXiv 2412.16750, Sec. IV-A and V-B) in one persistent
// launch.  Lane segments are independent (whole lanes, per-vehicle
// parameters), so a warp group can carry one segment through every
// iteration without waiting for the rest of the scene: per iteration it
// reloads the segment's vehicles (the parameters the previous update wrote),
// runs the forward with checkpoints (idm_forward.cuh; only in the first
// iteration when K fits one checkpoint interval, since the one checkpoint is
// then the unchanging initial state), then the adjoint with the fused Adam
// update (idm_adjoint.cuh).  The arithmetic is that of one
// forward launch plus one adjoint launch per iteration, so parameters and
// loss history match the per-iteration graph bit for bit; what goes away is
// the per-iteration launch boundary (drain, launch, segment pickup), which
// dominates when K is short or the scene small.
//
// Every slot's checkpoints, sub-checkpoints, parameters and Adam moments are
// written and read back by the thread that owns the slot (the forward and
// the adjoint use the same slot mapping), so program order orders them; the
// membar after the forward also covers the adjoint's cp.async reads of the
// checkpoints.  The loss partial of iteration it goes to
// loss_part[it * part_stride + s_idx * G + w].
#pragma once
#include "idm_adjoint.cuh"
#include "idm_forward.cuh"

namespace idm {

template <int VPT, int GW, bool SUB>
__global__ void __launch_bounds__(BwdBounds<VPT, GW>::threads, BwdBounds<VPT, GW>::blocks)
fit_fused_kernel(SimArgs a, long long part_stride)
{
    constexpr int NP = VPT / 2;
    constexpr int G = GW;
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5;
    const int gf = bwd_group_floats(VPT, false, a.tape_T, G, a.bwd_pf != 0);
    float *gbase = smem + (warp / G) * gf;
    float *ctrl = gbase + gf - grp_ctrl_floats(G);
    Grp g = make_grp(G, ctrl);
    const int n_seg = *a.n_seg;
    // more segments than the partials were sized for: only possible when a
    // lane exceeds the segment capacity or lane_off is malformed, both
    // already flagged by the segment builder
    if ((long long)n_seg * G > part_stride) {
        if (threadIdx.x == 0) atomicOr(a.status, IDM_STATUS_LANE_TOO_LONG);
        return;
    }
    double *const part0 = a.loss_part;
    const FwdFlags ff{false, false, true, false};
    int par = 0;
    for (;;) {
        const int s_idx = grp_next(g, a.work, par);
        if (s_idx >= n_seg) break;
        const Seg sg = a.seg[s_idx];
        const ScenDesc sc = a.scen_tab ? a.scen_tab[sg.scen] : a.scen0;
        const int lb = sg.veh_begin - sc.veh_begin;
        for (int it = 0; it < a.n_iter; ++it) {
            a.iter = it;
            a.loss_part = part0 + (size_t)it * (size_t)part_stride;
            VehConst2 kc[NP];
            State2 st[NP], sf[NP];
            bool vx[NP], vy[NP];
            load_vehicles<NP>(a, sg, g.lane, g.w * 64 * NP, kc, st, vx, vy);
            const bool d4 = segment_is_d4<NP>(kc, vx, vy);
#pragma unroll
            for (int p = 0; p < NP; ++p) sf[p] = st[p];
            // with K within one checkpoint interval the only checkpoint is the
            // initial state: written in the first iteration, unchanged after
            if (it == 0 || sc.K > a.C) {
                if (d4)
                    forward_segment<NP, true>(a, sc, s_idx, lb, g, kc, sf, vx, vy, ff);
                else
                    forward_segment<NP, false>(a, sc, s_idx, lb, g, kc, sf, vx, vy, ff);
                __threadfence_block();
                grp_sync(g);  // the group's exchange cells: the forward's last reads before the adjoint's first writes
            }
            if constexpr (SUB) {
                if (d4)
                    backward_segment_blocks<NP, false, true, false, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
                else
                    backward_segment_blocks<NP, false, true, false, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx,
                                                                           vy);
            } else {
                if (d4)
                    backward_segment<NP, false, true, false, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
                else
                    backward_segment<NP, false, true, false, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
            }
            grp_sync(g);  // and the adjoint's last reads before the next forward's first writes
        }
    }
}

template <int VPT, int GW>
inline void *fused_fn_t(bool sub)
{
    return sub ? (void *)fit_fused_kernel<VPT, GW, true> : (void *)fit_fused_kernel<VPT, GW, false>;
}

// The forward, adjoint and single-launch fit kernels of one shape, as the
// entry points declared in idm_internal.h (one translation unit per shape, so
// the shapes compile in parallel).
#define IDM_DEFINE_SHAPE_KERNELS(V, GW)                                                  \
    void *forward_fn_v##V##_g##GW(bool count) { return forward_fn_t<V, GW>(count); }     \
    void *backward_fn_v##V##_g##GW(bool dense, bool adam, bool wd, bool sub)              \
    {                                                                                    \
        return sub ? backward_fn_t<V, GW, true>(dense, adam, wd) : backward_fn_t<V, GW, false>(dense, adam, wd); \
    }                                                                                    \
    void *fused_fn_v##V##_g##GW(bool sub) { return fused_fn_t<V, GW>(sub); }

}  // namespace idm
