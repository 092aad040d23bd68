// Device helpers shared by the forward kernel (idm_sim.cu) and the adjoint
// kernels (idm_adjoint.cuh): work distribution, compensated sums, cp.async,
// warp groups (segments run by several warps of one block), vehicle loads.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idm_device.cuh"
#include "idm_internal.h"

namespace idm {

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int next_segment(int *work, int lane)
{
    int s = 0;
    if (lane == 0) s = atomicAdd(work, 1);
    return __shfl_sync(FULL, s, 0);
}

// Kahan-compensated float accumulation.
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    float y = __fsub_rn(x, comp);
    float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

__device__ __forceinline__ double warp_sum_double(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Asynchronous 4-byte global->shared copies (cp.async, completion tracked
// per thread in commit groups).
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Slots of a warp: pair p of lane l holds slots 64p + 2l and 64p + 2l + 1.
// dst/src_row already point at this warp's first slot.
template <int NP>
__device__ __forceinline__ void prefetch_row(float *dst, const float *src_row, int lane, const bool (&vx)[NP],
                                             const bool (&vy)[NP])
{
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int q = 64 * p + 2 * lane;
        if (vx[p]) cp_async4(dst + q, src_row + q);
        if (vy[p]) cp_async4(dst + q + 1, src_row + q + 1);
    }
}

// ---------------------------------------------------------------------------
// Warp groups.  A segment of up to 32*VPT*G vehicles is run by G warps of
// one block (G = 1: a single warp, no barrier).  Warp w of the group holds
// slots [w*32*VPT, (w+1)*32*VPT).  Per step, the leader value of each warp's
// first slot and (in the adjoint) the follower terms of each warp's last
// slot cross warp boundaries through double-buffered shared cells and one
// named barrier (bar.sync id, 32*G) per exchange.
// ---------------------------------------------------------------------------
struct Grp {
    int G;       // warps per segment
    int w;       // warp index in the group
    int lane;
    int bar;     // named barrier id (1 + group index in the block)
    int *cell;   // [2] work-item broadcast
    float *xl;   // [2][G][2] leader exchange (speed, speed compensation)
    float *xf;   // [2][2][G] follower exchange
};

// Shared floats of one group's control area (cells + exchange cells).
__host__ __device__ __forceinline__ int grp_ctrl_floats(int G) { return ((2 + 8 * G) + 3) & ~3; }

__device__ __forceinline__ void grp_sync(const Grp &g)
{
    if (g.G > 1)
        asm volatile("bar.sync %0, %1;" ::"r"(g.bar), "r"(32 * g.G) : "memory");
    else
        __syncwarp();
}

__device__ __forceinline__ Grp make_grp(int G, float *ctrl)
{
    Grp g;
    g.G = G;
    const int warp = threadIdx.x >> 5;
    g.w = warp % G;
    g.lane = threadIdx.x & 31;
    g.bar = 1 + warp / G;
    g.cell = reinterpret_cast<int *>(ctrl);
    g.xl = ctrl + 2;
    g.xf = ctrl + 2 + 4 * G;
    return g;
}

__device__ __forceinline__ int grp_next(const Grp &g, int *work, int &par)
{
    if (g.G == 1) return next_segment(work, g.lane);
    if (g.w == 0 && g.lane == 0) g.cell[par] = atomicAdd(work, 1);
    grp_sync(g);
    const int s = g.cell[par];
    par ^= 1;
    return s;
}

// Leader speed and speed compensation of this warp's first slot (0 for the
// group's first warp); last is this lane's pair of the warp's last slot
// (used by lane 31).
__device__ __forceinline__ float2 grp_lead_in(const Grp &g, float2 last, int &xp)
{
    if (g.G == 1) return make_float2(0.0f, 0.0f);
    float2 *c = reinterpret_cast<float2 *>(g.xl);
    if (g.lane == 31) c[xp * g.G + g.w] = last;
    grp_sync(g);
    const float2 r = g.w > 0 ? c[xp * g.G + g.w - 1] : make_float2(0.0f, 0.0f);
    xp ^= 1;
    return r;
}

// Follower terms arriving at this warp's last slot (0 for the last warp).
__device__ __forceinline__ void grp_follow_in(const Grp &g, float p_first, float v_first, float &in_p, float &in_v,
                                              int &xp)
{
    in_p = 0.0f;
    in_v = 0.0f;
    if (g.G == 1) return;
    float *c = g.xf + xp * 2 * g.G;
    if (g.lane == 0) {
        c[g.w] = p_first;
        c[g.G + g.w] = v_first;
    }
    grp_sync(g);
    if (g.w + 1 < g.G) {
        in_p = c[g.w + 1];
        in_v = c[g.G + g.w + 1];
    }
    xp ^= 1;
}

// One Euler step (Eq. 1-3 with the Sec. III-C bounds) of this thread's
// vehicle pairs: the leaders' speeds and speed compensations by shuffle
// (across warps through the group's cells), then a* and the state update.
template <int NP, bool D4>
__device__ __forceinline__ void step_pairs(const Grp &g, State2 (&st)[NP], const VehConst2 (&kc)[NP],
                                           const ScenDesc &sc, int &xp)
{
    f2 vcur[NP], ccur[NP], vh[NP], ch[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        vcur[p] = st[p].v;
        ccur[p] = st[p].vc;
    }
    const float2 lead_in = grp_lead_in(g, make_float2(vcur[NP - 1].y, ccur[NP - 1].y), xp);
    leader_vals2<NP>(vcur, vh, g.lane, lead_in.x);
    leader_vals2<NP>(ccur, ch, g.lane, lead_in.y);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const f2 as = accel_star2<D4>(st[p].v, st[p].gap, vh[p], kc[p], sc.inv_dt, sc.a_min);
        euler2(st[p], as, vh[p], ch[p], sc.dt);
    }
}

template <int NP>
__device__ __forceinline__ void load_vehicles(const SimArgs &a, const Seg &sg, int lane, int wb, VehConst2 (&kc)[NP],
                                              State2 (&st)[NP], bool (&vx)[NP], bool (&vy)[NP])
{
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int q = wb + 64 * p + 2 * lane + c;
            const bool ok = q < sg.n_veh;
            float inv_v0 = 1.0f, T = 0.0f, s0 = 0.0f, am = 1.0f, cc = 0.5f, dl = 4.0f;  // ghost slot
            float ph = 0.0f, v = 0.0f, gap = INFINITY;
            if (ok) {
                const int gi = sg.veh_begin + q;
                inv_v0 = __frcp_rn(a.v0[gi]);
                T = a.T[gi];
                s0 = a.s0[gi];
                am = a.am[gi];
                cc = c_of(am, a.b[gi]);
                dl = a.delta[gi];
                ph = a.p_init[gi];
                v = a.v_init[gi];
                gap = a.g0[gi];
            }
            if (c == 0) {
                vx[p] = ok;
                kc[p].inv_v0.x = inv_v0; kc[p].T.x = T; kc[p].s0.x = s0; kc[p].am.x = am; kc[p].c.x = cc;
                kc[p].delta.x = dl;
                st[p].ph.x = ph; st[p].pl.x = 0.0f; st[p].v.x = v; st[p].gap.x = gap; st[p].vc.x = 0.0f;
            } else {
                vy[p] = ok;
                kc[p].inv_v0.y = inv_v0; kc[p].T.y = T; kc[p].s0.y = s0; kc[p].am.y = am; kc[p].c.y = cc;
                kc[p].delta.y = dl;
                st[p].ph.y = ph; st[p].pl.y = 0.0f; st[p].v.y = v; st[p].gap.y = gap; st[p].vc.y = 0.0f;
            }
        }
    }
}

// True when every occupied slot of the warp has delta == 4, so the step body
// can use the squaring form of (v/v0)^delta with no branch.  (Both variants
// execute the same sequence of group barriers.)
template <int NP>
__device__ __forceinline__ bool segment_is_d4(const VehConst2 (&kc)[NP], const bool (&vx)[NP], const bool (&vy)[NP])
{
    bool ok = true;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (vx[p] && kc[p].delta.x != 4.0f) ok = false;
        if (vy[p] && kc[p].delta.y != 4.0f) ok = false;
    }
    return __all_sync(FULL, ok);
}

// Store one pair to a scalar array at slot offset q (two 4-byte stores:
// the pair's global index need not be 8-byte aligned).
__device__ __forceinline__ void store_pair(float *base, int q, f2 x, bool vx, bool vy)
{
    if (vx) base[q] = x.x;
    if (vy) base[q + 1] = x.y;
}

__device__ __forceinline__ f2 load_pair(const float *base, int q, bool vx, bool vy)
{
    return make_float2(vx ? base[q] : 0.0f, vy ? base[q + 1] : 0.0f);
}


__device__ __forceinline__ f2 lds2(const float *p) { return *reinterpret_cast<const f2 *>(p); }
__device__ __forceinline__ void sts2(float *p, f2 x) { *reinterpret_cast<f2 *>(p) = x; }

// Shared floats of one adjoint group: tape v/gap [T][G*SL], target/seed
// tapes [T][G*SL] (MSE only), state stages [STATE_ROWS][G*SL], control area; T is the tape depth (the checkpoint interval, or less when
// blocks restart from sub-checkpoints).  With prefetch the target tape and
// the state stage are doubled and the next block's targets and starting
// state are copied (cp.async) into the idle pair while the current block
// runs.
__host__ __device__ __forceinline__ int bwd_group_floats(int vpt, bool dense, int T, int G, bool pf)
{
    const int nb = pf ? 2 : 1;
    return ((dense ? 2 : 2 + nb) * T + STATE_ROWS * nb) * 32 * vpt * G + grp_ctrl_floats(G);
}

}  // namespace idm
