// The forward pass over one warp segment (Eq. 1-3 with the Sec. III-C
// bounds, arXiv 2412.16750): K Euler steps with checkpoints every C steps,
// optional trajectory / speed output and an optional squared error against
// a second target set.  Used by the forward kernel (idm_sim.cu) and by the
// single-launch fit (idm_fused.cuh).
#pragma once
#include "idm_sim_common.cuh"

namespace idm {

// ---------------------------------------------------------------------------
// Forward: K steps per segment, optional trajectory / speed output,
// checkpoints every C steps.  (The squared-error loss is accumulated by the
// adjoint's recompute, which evaluates the residuals anyway.)
// ---------------------------------------------------------------------------
struct FwdFlags {
    bool traj, vtraj, ckpt, eval;
};

// COUNT: also count the vehicle-steps with the raw gap below the floor and
// those within IDM_KINK_BAND of the kink of the lower bound into a.events
// (a separate instantiation, so the plain forward carries no cost of it).
template <int NP, bool D4, bool COUNT = false>
__device__ __forceinline__ void forward_segment(const SimArgs &a, const ScenDesc &sc, int s_idx, int lb, Grp &g,
                                                const VehConst2 (&kc)[NP], State2 (&st)[NP], const bool (&vx)[NP],
                                                const bool (&vy)[NP], FwdFlags f)
{
    const int lane = g.lane;
    const int Ns = sc.n_veh;
    const int wl = lb + g.w * 64 * NP;  // scenario-local index of this warp's first slot
    int next_ck = 0, ck_idx = 0;
    int xp = 0;
    int obs_k = sc.obs_stride, obs_row = 0;  // next observed step and its target row (eval)
    float esum = 0.0f, ecomp = 0.0f;         // squared residuals (eval), Kahan over observed steps
    int n_floor = 0, n_kink = 0;             // event counts of this thread's slots (count)
    for (int k = 0;; ++k) {
        if (f.ckpt && k == next_ck && k < sc.K) {
            float *base = a.ckpt + sc.ckpt_off + (size_t)ck_idx * STATE_ROWS * Ns + wl;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                store_pair(base, q, st[p].ph, vx[p], vy[p]);
                store_pair(base + (size_t)Ns, q, st[p].pl, vx[p], vy[p]);
                store_pair(base + 2 * (size_t)Ns, q, st[p].v, vx[p], vy[p]);
                store_pair(base + 3 * (size_t)Ns, q, st[p].gap, vx[p], vy[p]);
                store_pair(base + 4 * (size_t)Ns, q, st[p].vc, vx[p], vy[p]);
            }
            next_ck += a.C;
            ++ck_idx;
        }
        if (f.traj || f.vtraj) {
            const size_t row = sc.traj_off + (size_t)k * Ns + wl;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                if (f.traj) store_pair(a.traj + row, q, position2(st[p]), vx[p], vy[p]);
                if (f.vtraj) store_pair(a.vtraj + row, q, speed2(st[p]), vx[p], vy[p]);
            }
        }
        if (f.eval && k == obs_k) {
            if (obs_row < sc.n_obs) {
                const float *y = a.eval_targets + sc.tgt_off + (size_t)obs_row * Ns + wl;
                f2 e = F2(0.0f);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    f2 r = residual2(st[p], load_pair(y, 64 * p + 2 * lane, vx[p], vy[p]));
                    r.x = vx[p] ? r.x : 0.0f;
                    r.y = vy[p] ? r.y : 0.0f;
                    e = fma2(r, r, e);
                }
                kahan_add(esum, ecomp, __fadd_rn(e.x, e.y));
            }
            obs_k += sc.obs_stride;
            ++obs_row;
        }
        if (k == sc.K) break;
        if (COUNT) {
            // the step's raw gap below the floor (derivative 0 there), and -v/dt
            // within IDM_KINK_BAND of a_min, as the step below evaluates it
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const f2 lbv = mul2(st[p].v, F2(-sc.inv_dt));
                n_floor += (vx[p] && st[p].gap.x < IDM_GAP_FLOOR) + (vy[p] && st[p].gap.y < IDM_GAP_FLOOR);
                n_kink += (vx[p] && fabsf(__fsub_rn(lbv.x, sc.a_min)) < IDM_KINK_BAND) +
                          (vy[p] && fabsf(__fsub_rn(lbv.y, sc.a_min)) < IDM_KINK_BAND);
            }
        }

        step_pairs<NP, D4>(g, st, kc, sc, xp);
    }
    bool bad = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (vx[p] && !(isfinite(st[p].v.x) && isfinite(st[p].ph.x))) bad = true;
        if (vy[p] && !(isfinite(st[p].v.y) && isfinite(st[p].ph.y))) bad = true;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, IDM_STATUS_NONFINITE);
    if (COUNT) {
        const int cf = __reduce_add_sync(FULL, (unsigned)n_floor), ck = __reduce_add_sync(FULL, (unsigned)n_kink);
        if (lane == 0 && cf) atomicAdd(a.events, (unsigned long long)cf);
        if (lane == 0 && ck) atomicAdd(a.events + 1, (unsigned long long)ck);
    }
    if (f.eval) {
        const double part = warp_sum_double((double)esum - (double)ecomp) * (double)sc.inv_nobs;
        if (lane == 0) a.eval_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

// Register budgets: 8 vehicles per thread (four pairs of state and constants)
// need more than the 128 registers of 16 warps per SM: their blocks are
// capped at 12 warps (one block per SM, up to 168 registers).
template <int VPT>
struct FwdBounds {
    static constexpr int threads = VPT == 8 ? 384 : 512;
};

template <int VPT, int GW, bool COUNT>
__global__ void __launch_bounds__(FwdBounds<VPT>::threads)
forward_kernel(SimArgs a, FwdFlags f)
{
    constexpr int NP = VPT / 2;
    constexpr int G = GW;  // a compile-time constant, as in the adjoint
    extern __shared__ float fsmem[];
    const int warp = threadIdx.x >> 5;
    float *ctrl = fsmem + (warp / G) * grp_ctrl_floats(G);
    Grp g = make_grp(G, ctrl);
    int par = 0;
    for (;;) {
        const int s_idx = grp_next(g, a.work, par);
        if (s_idx >= *a.n_seg) break;
        const Seg sg = a.seg[s_idx];
        const ScenDesc sc = a.scen_tab ? a.scen_tab[sg.scen] : a.scen0;
        const int lb = sg.veh_begin - sc.veh_begin;  // scenario-local index of slot 0
        VehConst2 kc[NP];
        State2 st[NP];
        bool vx[NP], vy[NP];
        load_vehicles<NP>(a, sg, g.lane, g.w * 64 * NP, kc, st, vx, vy);
        if (segment_is_d4<NP>(kc, vx, vy))
            forward_segment<NP, true, COUNT>(a, sc, s_idx, lb, g, kc, st, vx, vy, f);
        else
            forward_segment<NP, false, COUNT>(a, sc, s_idx, lb, g, kc, st, vx, vy, f);
    }
}

template <int VPT, int GW>
inline void *forward_fn_t(bool count)
{
    return count ? (void *)forward_kernel<VPT, GW, true> : (void *)forward_kernel<VPT, GW, false>;
}

}  // namespace idm
