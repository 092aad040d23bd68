// Adjoint kernel templates; each idm_adjoint<VPT>.cu instantiates the
// variants of one vehicles-per-thread value (so they compile in parallel).
#pragma once
#include "idm_sim_common.cuh"

namespace idm {

// ---------------------------------------------------------------------------
// Adjoint.  Per segment of C steps (last first): cp.async the observed
// targets of the C steps into the seed tape, reload the checkpoint,
// recompute the C steps into the group's shared tape of (v, raw gap, seed),
// then run the reverse recurrences
//   lp_k = seed_k + lp_{k+1} + mu A_p + mu_f A_ph(f)
//   lv_k = dt lp_{k+1} + lv_{k+1} + mu A_v + mu_f A_vh(f)
// with mu = dt lv_{k+1}; the follower's terms arrive by one warp shuffle
// (and across warps through the group's exchange cells).  The coefficients
// of step k-1 are evaluated while the dependent chain of step k runs.
// The six factored gradient sums of each slot accumulate in registers and
// are folded into compensated totals about every FOLD_STEPS steps.
// ---------------------------------------------------------------------------
// Compensated gradient sums.  Within a fold window of max(1, FOLD_STEPS / C)
// checkpoint segments (counted from the last) the six factored sums of a slot
// accumulate in FP32 registers; at the end of each window they are added to
// the slot's running totals, kept in a.gsum as unevaluated float pairs
// hi + lo, by Knuth's TwoSum, which returns the rounding error of the
// addition exactly.  The error of a slot's sum then stays that of one
// window's FP32 accumulation, whatever the horizon.  The totals of segment
// s_idx occupy 6 x (capacity / 2) float4 (hi.x, hi.y, lo.x, lo.y) per vehicle
// pair, each written and read back by the thread that owns the pair.
// ---------------------------------------------------------------------------
constexpr int FOLD_STEPS = GSUM_FOLD_STEPS;

// A compile-time flag passed as a value (to a generic lambda).
template <bool B>
struct BoolC {
    static constexpr bool value = B;
};

template <int NP, bool WD>
__device__ __forceinline__ void fold_sums(const SimArgs &a, int s_idx, const Grp &g, f2 (&sacc)[6][NP], bool have,
                                          bool last)
{
    const int pairs = 32 * NP * g.G;  // vehicle pairs of a segment
    float4 *base = reinterpret_cast<float4 *>(a.gsum) + (size_t)s_idx * 6 * pairs + g.w * 32 * NP + g.lane;
#pragma unroll
    for (int q = 0; q < (WD ? 6 : 5); ++q) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float4 *t = base + (size_t)q * pairs + 32 * p;
            f2 hi = F2(0.0f), lo = F2(0.0f);
            if (have) {
                const float4 v = *t;
                hi = make_float2(v.x, v.y);
                lo = make_float2(v.z, v.w);
            }
            const f2 x = sacc[q][p];
            const f2 sum = add2(hi, x);  // TwoSum: sum + e == hi + x exactly
            const f2 bb = sub2(sum, hi);
            const f2 e = add2(sub2(hi, sub2(sum, bb)), sub2(x, bb));
            lo = add2(lo, e);
            if (last) {
                sacc[q][p] = add2(sum, lo);
            } else {
                *t = make_float4(sum.x, sum.y, lo.x, lo.y);
                sacc[q][p] = F2(0.0f);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Epilogue of a segment: the parameter gradients from the six factored
// sums, then either their output or (fit) the Adam update with the box
// projection in place.  Adam is taken in the reordered form of Kingma & Ba
// (2015, Sec. 2): with alpha_t = lr sqrt(1 - beta2^t) / (1 - beta1^t) and
// eps_t = eps sqrt(1 - beta2^t), theta -= alpha_t m / (sqrt(v) + eps_t) is
// the bias-corrected step with its per-iteration factors computed once per
// thread.  Every load of a slot is issued before the slot's stores: the
// parameter and moment arrays may alias as far as the compiler knows, so a
// store would otherwise hold back each later load for a full memory round
// trip (this epilogue was half of a short-horizon fit iteration).
template <int NP, bool ADAM, bool WD, bool D4>
__device__ __forceinline__ void segment_epilogue(const SimArgs &a, const Seg &sg, int lane, int wb,
                                                 const VehConst2 (&kc)[NP], const f2 (&sacc)[6][NP],
                                                 const f2 (&lp)[NP], const f2 (&lv)[NP], const bool (&vx)[NP],
                                                 const bool (&vy)[NP])
{
    float step_t = 0.0f, eps_t = 0.0f;
    if (ADAM) {
        const int it = a.iter;
        const float lr = a.n_iter > 1 ? a.lr0 + (a.lr1 - a.lr0) * (float)it / (float)(a.n_iter - 1) : a.lr0;
        const float bc1 = 1.0f - powf(0.9f, (float)(it + 1)), bc2 = 1.0f - powf(0.999f, (float)(it + 1));
        const float sb2 = sqrtf(bc2);
        step_t = lr * sb2 / bc1;
        eps_t = 1e-8f * sb2;
    }
    float *const th[5] = {const_cast<float *>(a.v0), const_cast<float *>(a.T), const_cast<float *>(a.s0),
                          const_cast<float *>(a.am), const_cast<float *>(a.b)};
    bool bad = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(c ? vy[p] : vx[p])) continue;
            const int gi = sg.veh_begin + wb + 64 * p + 2 * lane + c;
            // this slot's loads, all ahead of its stores
            float tv[5], mm[5], vm[5];
            if (ADAM) {
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const size_t mi = (size_t)r * a.N_total + gi;
                    tv[r] = th[r][gi];
                    mm[r] = a.adam_m[mi];
                    vm[r] = a.adam_v[mi];
                }
            } else {
                tv[0] = a.v0[gi];
                tv[4] = a.b[gi];
            }
            const float v0 = tv[0], b = tv[4];
            const float am = c ? kc[p].am.y : kc[p].am.x, cc = c ? kc[p].c.y : kc[p].c.x;
            const float dl = D4 ? 4.0f : (c ? kc[p].delta.y : kc[p].delta.x);
            const float A0 = c ? sacc[0][p].y : sacc[0][p].x, A1 = c ? sacc[1][p].y : sacc[1][p].x;
            const float A2 = c ? sacc[2][p].y : sacc[2][p].x, A3 = c ? sacc[3][p].y : sacc[3][p].x;
            const float A4 = c ? sacc[4][p].y : sacc[4][p].x, A5 = c ? sacc[5][p].y : sacc[5][p].x;
            float gr[6];
            gr[0] = am * dl * A4 / v0;                 // v0
            gr[1] = -A1;                               // T
            gr[2] = -A0;                               // s0
            gr[3] = A3 + A2 * cc / (2.0f * am);        // a_max
            gr[4] = A2 * cc / (2.0f * b);              // b
            gr[5] = -am * A5;                          // delta
#pragma unroll
            for (int r = 0; r < 6; ++r) bad |= !isfinite(gr[r]);
            if (ADAM) {
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const size_t mi = (size_t)r * a.N_total + gi;
                    const float m = 0.9f * mm[r] + 0.1f * gr[r];
                    const float vv = 0.999f * vm[r] + 0.001f * gr[r] * gr[r];
                    a.adam_m[mi] = m;
                    a.adam_v[mi] = vv;
                    const float x = tv[r] - step_t * m / (sqrtf(vv) + eps_t);
                    th[r][gi] = fminf(fmaxf(x, a.lo[r]), a.hi[r]);
                }
            } else {
                if (a.g_v0) a.g_v0[gi] = gr[0];
                if (a.g_T) a.g_T[gi] = gr[1];
                if (a.g_s0) a.g_s0[gi] = gr[2];
                if (a.g_am) a.g_am[gi] = gr[3];
                if (a.g_b) a.g_b[gi] = gr[4];
                if (a.g_delta) a.g_delta[gi] = WD ? gr[5] : 0.0f;
                if (a.g_p_init) a.g_p_init[gi] = c ? lp[p].y : lp[p].x;
                if (a.g_v_init) a.g_v_init[gi] = c ? lv[p].y : lv[p].x;
            }
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, IDM_STATUS_NONFINITE);
}

template <int NP, bool DENSE, bool ADAM, bool WD, bool D4>
__device__ __forceinline__ void backward_segment(const SimArgs &a, const ScenDesc &sc, const Seg &sg, int s_idx, int lb,
                                                 Grp &g, float *tv, const VehConst2 (&kc)[NP], State2 (&st)[NP],
                                                 const bool (&vx)[NP], const bool (&vy)[NP])
{
    constexpr int SL = 64 * NP;
    const int SLG = SL * g.G;
    const int lane = g.lane;
    const int wb = g.w * SL;                        // this warp's first slot in the group
    const int nb = a.bwd_pf ? 2 : 1;                // stages (double-buffered with prefetch)
    float *tg = tv + a.C * SLG;                     // (tape depth = checkpoint interval here)
    float *trb = tg + a.C * SLG;                    // nb tapes: targets, then seeds (MSE only)
    float *ckb = tv + (DENSE ? 2 : 2 + nb) * a.C * SLG;  // nb checkpoint stages [STATE_ROWS][SLG]
    const int Ns = sc.n_veh;
    const int wl = lb + wb;                         // scenario-local index of this warp's first slot
    const float dt = sc.dt;
    const f2 seed_scale = F2(2.0f * sc.inv_nobs);
    int xp = 0, fp = 0;
    float lsum = 0.0f, lcomp = 0.0f;  // squared residuals (MSE): Kahan across checkpoint segments

    // lp, lv: adjoints of position and speed; sacc: the six factored
    // gradient sums of every slot, accumulated in registers over all steps
    f2 lp[NP], lv[NP], sacc[6][NP], qc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        qc[p] = D4 ? mul2(mul2(kc[p].am, F2(4.0f)), kc[p].inv_v0) : F2(0.0f);  // 4 a_max / v0
        lp[p] = F2(0.0f);
        lv[p] = F2(0.0f);
#pragma unroll
        for (int q = 0; q < 6; ++q) sacc[q][p] = F2(0.0f);
    }

    // first observed step >= max(c0, 1) of a checkpoint segment and its
    // target row (one division per segment; the step loops count instead)
    auto first_obs = [&](int c0, int &obs_k, int &obs_row) {
        obs_row = (c0 + sc.obs_stride - 1) / sc.obs_stride;
        if (obs_row == 0) obs_row = 1;
        obs_k = obs_row * sc.obs_stride;
        obs_row -= 1;
    };
    // cp.async of segment cs's observed targets and checkpoint into the
    // stage of its parity (each thread copies only its own slots)
    auto prefetch_segment = [&](int cs) {
        const int c0 = cs * a.C;
        const int n = min(a.C, sc.K - c0);
        const int par = a.bwd_pf ? (cs & 1) : 0;
        if (!DENSE) {
            float *tr = trb + par * a.C * SLG;
            int obs_k, obs_row;
            first_obs(c0, obs_k, obs_row);
            const float *yrow = a.targets + sc.tgt_off + (size_t)obs_row * Ns + wl;
            for (int k = obs_k, r = obs_row; k < c0 + n && r < sc.n_obs; k += sc.obs_stride, ++r, yrow += Ns)
                prefetch_row<NP>(tr + (k - c0) * SLG + wb, yrow, lane, vx, vy);
        }
        float *ck = ckb + par * STATE_ROWS * SLG;
        const float *base = a.ckpt + sc.ckpt_off + (size_t)cs * STATE_ROWS * Ns + wl;
#pragma unroll
        for (int f = 0; f < STATE_ROWS; ++f)
            prefetch_row<NP>(ck + f * SLG + wb, base + (size_t)f * Ns, lane, vx, vy);
        cp_async_commit();
    };

    const int n_ck = (sc.K + a.C - 1) / a.C;
    const int fold_every = max(1, FOLD_STEPS / a.C);  // checkpoint segments per fold of the gradient sums
    if (a.bwd_pf) prefetch_segment(n_ck - 1);
    for (int cs = n_ck - 1; cs >= 0; --cs) {
        const int c0 = cs * a.C;
        const int n = min(a.C, sc.K - c0);
        int obs_k, obs_row;
        first_obs(c0, obs_k, obs_row);
        const int par = a.bwd_pf ? (cs & 1) : 0;
        float *tr = trb + par * a.C * SLG;
        if (!a.bwd_pf) prefetch_segment(cs);
        cp_async_wait<0>();  // this segment's targets and checkpoint (this thread's own slots)
        {
            const float *ck = ckb + par * STATE_ROWS * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                const f2 ph = lds2(ck + q), pl = lds2(ck + SLG + q), v = lds2(ck + 2 * SLG + q);
                const f2 gp = lds2(ck + 3 * SLG + q), vc = lds2(ck + 4 * SLG + q);
                st[p].ph = make_float2(vx[p] ? ph.x : 0.0f, vy[p] ? ph.y : 0.0f);
                st[p].pl = make_float2(vx[p] ? pl.x : 0.0f, vy[p] ? pl.y : 0.0f);
                st[p].v = make_float2(vx[p] ? v.x : 0.0f, vy[p] ? v.y : 0.0f);
                st[p].gap = make_float2(vx[p] ? gp.x : INFINITY, vy[p] ? gp.y : INFINITY);
                st[p].vc = make_float2(vx[p] ? vc.x : 0.0f, vy[p] ? vc.y : 0.0f);
            }
        }
        if (a.bwd_pf && cs > 0) prefetch_segment(cs - 1);  // lands while this segment runs
        f2 lseg = F2(0.0f);
        // recompute the segment into the tape.  The observation handling has no
        // branch (an unobserved step's residual, read from a row the copies
        // did not fill, is selected to 0), and the last step is peeled off:
        // the state after it is needed only at the end of the horizon (the
        // seed of step K)
        auto recompute_step = [&](const int s, const bool advance) {
            const int k = c0 + s;
            float *rv = tv + s * SLG + wb, *rg = tg + s * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                sts2(rv + q, st[p].v);
                sts2(rg + q, st[p].gap);
            }
            if constexpr (!DENSE) {
                const bool hit = k == obs_k;
                const bool obs = hit && obs_row < sc.n_obs;
                float *rr = tr + s * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    f2 r = residual2(st[p], lds2(rr + q));
                    r.x = obs && vx[p] ? r.x : 0.0f;
                    r.y = obs && vy[p] ? r.y : 0.0f;
                    sts2(rr + q, mul2(seed_scale, r));
                    lseg = fma2(r, r, lseg);
                }
                obs_k += hit ? sc.obs_stride : 0;
                obs_row += hit ? 1 : 0;
            }
            if (advance) step_pairs<NP, D4>(g, st, kc, sc, xp);
        };
        for (int s = 0; s + 1 < n; ++s) recompute_step(s, true);
        recompute_step(n - 1, cs == n_ck - 1);
        if (cs == n_ck - 1) {  // state is now at step K: seed of the final step
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)sc.K * Ns + wl;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    lp[p] = load_pair(a.gP + row, q, vx[p], vy[p]);
                    lv[p] = a.gV ? load_pair(a.gV + row, q, vx[p], vy[p]) : F2(0.0f);
                }
            } else {
                const int k = sc.K;
                const bool obs = sc.n_obs > 0 && (k % sc.obs_stride) == 0 && k / sc.obs_stride <= sc.n_obs;
                if (obs) {
                    const float *y = a.targets + sc.tgt_off + (size_t)(k / sc.obs_stride - 1) * Ns + wl;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const int q = 64 * p + 2 * lane;
                        f2 r = residual2(st[p], load_pair(y, q, vx[p], vy[p]));
                        r.x = vx[p] ? r.x : 0.0f;
                        r.y = vy[p] ? r.y : 0.0f;
                        lp[p] = mul2(seed_scale, r);
                        lseg = fma2(r, r, lseg);
                    }
                }
            }
        }
        kahan_add(lsum, lcomp, __fadd_rn(lseg.x, lseg.y));
        grp_sync(g);  // the whole group's tape is written

        // last observed step <= c0 + n - 1 (for the MSE seeds of the sweep)
        int row_hi = (c0 + n - 1) / sc.obs_stride;  // target row + 1 of obs_hi
        int obs_hi = row_hi * sc.obs_stride;
        AdjJac2 J[NP];
        {
            const float *rv = tv + (n - 1) * SLG + wb, *rg = tg + (n - 1) * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                const f2 v = lds2(rv + q);
                const f2 vh = make_float2(wb + q > 0 ? rv[q - 1] : 0.0f, v.x);
                J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min, qc[p]);
            }
        }
        // one reverse step; the coefficients of step s - 1 are evaluated inside
        // it (next_j) for every step but the last, which is peeled off so that
        // the loop body has no branch around them
        auto reverse_step = [&](const int s, auto next_j) {
            const int k = c0 + s;
            f2 to_lp[NP], to_lv[NP], t1[NP], nlv[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const f2 mu = mul2(F2(dt), lv[p]);
                to_lp[p] = mul2(mu, J[p].Aph);
                to_lv[p] = mul2(mu, J[p].Avh);
                t1[p] = sub2(lp[p], to_lp[p]);                          // lp + mu A_p
                nlv[p] = fma2(mu, J[p].Av, fma2(F2(dt), lp[p], lv[p]));  // dt lp + lv + mu A_v
                sacc[0][p] = fma2(mu, J[p].w0n, sacc[0][p]);
                sacc[1][p] = fma2(mu, J[p].w0nv, sacc[1][p]);
                sacc[2][p] = fma2(mu, J[p].w0nvdv, sacc[2][p]);
                sacc[3][p] = fma2(mu, J[p].fa, sacc[3][p]);
                sacc[4][p] = fma2(mu, J[p].frd, sacc[4][p]);
                if (WD) sacc[5][p] = fma2(mu, J[p].frdl, sacc[5][p]);
            }
            if constexpr (decltype(next_j)::value) {
                const float *rv = tv + (s - 1) * SLG + wb, *rg = tg + (s - 1) * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    const f2 v = lds2(rv + q);
                    const f2 vh = make_float2(wb + q > 0 ? rv[q - 1] : 0.0f, v.x);
                    J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min, qc[p]);
                }
            }
            float in_p, in_v;
            grp_follow_in(g, to_lp[0].x, to_lv[0].x, in_p, in_v, fp);
            f2 from_p[NP], from_v[NP];
            follower_vals2<NP>(to_lp, from_p, lane, in_p);
            follower_vals2<NP>(to_lv, from_v, lane, in_v);
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)k * Ns + wl;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    lp[p] = add2(add2(t1[p], from_p[p]), load_pair(a.gP + row, q, vx[p], vy[p]));
                    lv[p] = add2(nlv[p], from_v[p]);
                    if (a.gV) lv[p] = add2(lv[p], load_pair(a.gV + row, q, vx[p], vy[p]));
                }
            } else {
                // the step's seed, selected to 0 where the step is not observed
                const bool hit = k == obs_hi;
                const bool on = hit && k >= 1 && row_hi <= sc.n_obs;
                const float *rr = tr + s * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    f2 sd = lds2(rr + 64 * p + 2 * lane);
                    sd.x = on ? sd.x : 0.0f;
                    sd.y = on ? sd.y : 0.0f;
                    lp[p] = add2(add2(t1[p], from_p[p]), sd);
                    lv[p] = add2(nlv[p], from_v[p]);
                }
                obs_hi -= hit ? sc.obs_stride : 0;
                row_hi -= hit ? 1 : 0;
            }
        };
        for (int s = n - 1; s >= 1; --s) reverse_step(s, BoolC<true>{});
        reverse_step(0, BoolC<false>{});
        // a fold window is fold_every checkpoint segments, counted from the last
        if (cs > 0 && (n_ck - cs) % fold_every == 0)
            fold_sums<NP, WD>(a, s_idx, g, sacc, n_ck - cs > fold_every, false);
        grp_sync(g);  // the tape may be overwritten by the next segment
    }
    if (n_ck > fold_every) fold_sums<NP, WD>(a, s_idx, g, sacc, true, true);

    segment_epilogue<NP, ADAM, WD, D4>(a, sg, lane, wb, kc, sacc, lp, lv, vx, vy);
    if (!DENSE) {
        const double part = warp_sum_double((double)lsum - (double)lcomp) * (double)sc.inv_nobs;
        if (lane == 0) a.loss_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

// The same adjoint when the tape is shallower than the checkpoint interval:
// each checkpoint segment is first run forward once writing sub-checkpoints
// every T steps (global scratch, this thread's own slots), then processed as
// tape blocks of T steps, last first.
template <int NP, bool DENSE, bool ADAM, bool WD, bool D4>
__device__ __forceinline__ void backward_segment_blocks(const SimArgs &a, const ScenDesc &sc, const Seg &sg, int s_idx, int lb,
                                                 Grp &g, float *tv, const VehConst2 (&kc)[NP], State2 (&st)[NP],
                                                 const bool (&vx)[NP], const bool (&vy)[NP])
{
    constexpr int SL = 64 * NP;
    const int SLG = SL * g.G;
    const int lane = g.lane;
    const int wb = g.w * SL;                        // this warp's first slot in the group
    const int nb = a.bwd_pf ? 2 : 1;                // stages (double-buffered with prefetch)
    const int T = a.tape_T;                         // tape depth (steps per block)
    float *tg = tv + T * SLG;
    float *trb = tg + T * SLG;                      // nb tapes: targets, then seeds (MSE only)
    float *ckb = tv + (DENSE ? 2 : 2 + nb) * T * SLG;  // nb state stages [STATE_ROWS][SLG]
    const int Ns = sc.n_veh;
    const int wl = lb + wb;                         // scenario-local index of this warp's first slot
    const float dt = sc.dt;
    const f2 seed_scale = F2(2.0f * sc.inv_nobs);
    int xp = 0, fp = 0;
    float lsum = 0.0f, lcomp = 0.0f;  // squared residuals (MSE): Kahan across checkpoint segments

    // lp, lv: adjoints of position and speed; sacc: the six factored
    // gradient sums of every slot, accumulated in registers over all steps
    f2 lp[NP], lv[NP], sacc[6][NP], qc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        qc[p] = D4 ? mul2(mul2(kc[p].am, F2(4.0f)), kc[p].inv_v0) : F2(0.0f);  // 4 a_max / v0
        lp[p] = F2(0.0f);
        lv[p] = F2(0.0f);
#pragma unroll
        for (int q = 0; q < 6; ++q) sacc[q][p] = F2(0.0f);
    }

    // first observed step >= max(c0, 1) of a checkpoint segment and its
    // target row (one division per segment; the step loops count instead)
    auto first_obs = [&](int c0, int &obs_k, int &obs_row) {
        obs_row = (c0 + sc.obs_stride - 1) / sc.obs_stride;
        if (obs_row == 0) obs_row = 1;
        obs_k = obs_row * sc.obs_stride;
        obs_row -= 1;
    };
    // Blocks.  Checkpoint segment cs (steps [cs C, cs C + len)) is processed
    // as ceil(len / T) tape blocks of at most T steps, last first.  Block j > 0
    // starts from sub-checkpoint row j - 1, written by a forward pass over
    // the segment; block 0 starts from the checkpoint.
    auto seg_len = [&](int cs) { return min(a.C, sc.K - cs * a.C); };
    auto n_sub = [&](int cs) { return (seg_len(cs) + T - 1) / T; };
    auto block_src = [&](int cs, int j, const float *&base, size_t &stride) {
        if (j == 0) {
            base = a.ckpt + sc.ckpt_off + (size_t)cs * STATE_ROWS * Ns + wl;
            stride = (size_t)Ns;
        } else {
            base = a.sub_ckpt + (size_t)(j - 1) * STATE_ROWS * a.N_total + sg.veh_begin + wb;
            stride = (size_t)a.N_total;
        }
    };
    // cp.async of block (cs, j)'s observed targets and starting state into
    // stage par (each thread copies only its own slots)
    auto prefetch_block = [&](int cs, int j, int par) {
        const int b0 = cs * a.C + j * T;
        const int bn = min(T, seg_len(cs) - j * T);
        if (!DENSE) {
            float *tr = trb + par * T * SLG;
            int obs_k, obs_row;
            first_obs(b0, obs_k, obs_row);
            const float *yrow = a.targets + sc.tgt_off + (size_t)obs_row * Ns + wl;
            for (int k = obs_k, r = obs_row; k < b0 + bn && r < sc.n_obs; k += sc.obs_stride, ++r, yrow += Ns)
                prefetch_row<NP>(tr + (k - b0) * SLG + wb, yrow, lane, vx, vy);
        }
        float *ck = ckb + par * STATE_ROWS * SLG;
        const float *base;
        size_t stride;
        block_src(cs, j, base, stride);
#pragma unroll
        for (int f = 0; f < STATE_ROWS; ++f)
            prefetch_row<NP>(ck + f * SLG + wb, base + (size_t)f * stride, lane, vx, vy);
        cp_async_commit();
    };
    // one forward step of the pair state (the leader's speed by shuffle)
    auto fwd_step = [&]() { step_pairs<NP, D4>(g, st, kc, sc, xp); };

    const int n_ck = (sc.K + a.C - 1) / a.C;
    const int fold_every = max(1, FOLD_STEPS / a.C);  // checkpoint segments per fold of the gradient sums
    int par = 0;
    bool have_next = false;  // the next block's stage is already being filled
    if (a.bwd_pf && n_sub(n_ck - 1) == 1) {
        prefetch_block(n_ck - 1, 0, 0);
        have_next = true;
    }
    for (int cs = n_ck - 1; cs >= 0; --cs) {
      const int nsub = n_sub(cs);
      if (nsub > 1) {  // forward pass over the segment writing the sub-checkpoints
        {
            const float *base = a.ckpt + sc.ckpt_off + (size_t)cs * STATE_ROWS * Ns + wl;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                st[p].ph = load_pair(base, q, vx[p], vy[p]);
                st[p].pl = load_pair(base + (size_t)Ns, q, vx[p], vy[p]);
                st[p].v = load_pair(base + 2 * (size_t)Ns, q, vx[p], vy[p]);
                const f2 gp = load_pair(base + 3 * (size_t)Ns, q, vx[p], vy[p]);
                st[p].gap = make_float2(vx[p] ? gp.x : INFINITY, vy[p] ? gp.y : INFINITY);
                st[p].vc = load_pair(base + 4 * (size_t)Ns, q, vx[p], vy[p]);
            }
        }
        for (int j = 1; j < nsub; ++j) {
            for (int s = 0; s < T; ++s) fwd_step();
            float *row = a.sub_ckpt + (size_t)(j - 1) * STATE_ROWS * a.N_total + sg.veh_begin + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                store_pair(row, q, st[p].ph, vx[p], vy[p]);
                store_pair(row + (size_t)a.N_total, q, st[p].pl, vx[p], vy[p]);
                store_pair(row + 2 * (size_t)a.N_total, q, st[p].v, vx[p], vy[p]);
                store_pair(row + 3 * (size_t)a.N_total, q, st[p].gap, vx[p], vy[p]);
                store_pair(row + 4 * (size_t)a.N_total, q, st[p].vc, vx[p], vy[p]);
            }
        }
        __threadfence_block();  // the rows are read back below (this thread's own slots)
      }
      for (int j = nsub - 1; j >= 0; --j) {
        const int c0 = cs * a.C + j * T;
        const int n = min(T, seg_len(cs) - j * T);
        int obs_k, obs_row;
        first_obs(c0, obs_k, obs_row);
        if (!have_next) prefetch_block(cs, j, par);
        float *tr = trb + par * T * SLG;
        cp_async_wait<0>();  // this block's targets and starting state (this thread's own slots)
        {
            const float *ck = ckb + par * STATE_ROWS * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                const f2 ph = lds2(ck + q), pl = lds2(ck + SLG + q), v = lds2(ck + 2 * SLG + q);
                const f2 gp = lds2(ck + 3 * SLG + q), vc = lds2(ck + 4 * SLG + q);
                st[p].ph = make_float2(vx[p] ? ph.x : 0.0f, vy[p] ? ph.y : 0.0f);
                st[p].pl = make_float2(vx[p] ? pl.x : 0.0f, vy[p] ? pl.y : 0.0f);
                st[p].v = make_float2(vx[p] ? v.x : 0.0f, vy[p] ? v.y : 0.0f);
                st[p].gap = make_float2(vx[p] ? gp.x : INFINITY, vy[p] ? gp.y : INFINITY);
                st[p].vc = make_float2(vx[p] ? vc.x : 0.0f, vy[p] ? vc.y : 0.0f);
            }
        }
        // start filling the other stage with the next block when its state exists
        have_next = false;
        if (a.bwd_pf) {
            if (j > 0) {
                prefetch_block(cs, j - 1, par ^ 1);
                have_next = true;
            } else if (cs > 0 && n_sub(cs - 1) == 1) {
                prefetch_block(cs - 1, 0, par ^ 1);
                have_next = true;
            }
        }
        f2 lseg = F2(0.0f);
        // recompute the segment into the tape.  The observation handling has no
        // branch (an unobserved step's residual, read from a row the copies
        // did not fill, is selected to 0), and the last step is peeled off:
        // the state after it is needed only at the end of the horizon (the
        // seed of step K)
        auto recompute_step = [&](const int s, const bool advance) {
            const int k = c0 + s;
            float *rv = tv + s * SLG + wb, *rg = tg + s * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                sts2(rv + q, st[p].v);
                sts2(rg + q, st[p].gap);
            }
            if constexpr (!DENSE) {
                const bool hit = k == obs_k;
                const bool obs = hit && obs_row < sc.n_obs;
                float *rr = tr + s * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    f2 r = residual2(st[p], lds2(rr + q));
                    r.x = obs && vx[p] ? r.x : 0.0f;
                    r.y = obs && vy[p] ? r.y : 0.0f;
                    sts2(rr + q, mul2(seed_scale, r));
                    lseg = fma2(r, r, lseg);
                }
                obs_k += hit ? sc.obs_stride : 0;
                obs_row += hit ? 1 : 0;
            }
            if (advance) step_pairs<NP, D4>(g, st, kc, sc, xp);
        };
        for (int s = 0; s + 1 < n; ++s) recompute_step(s, true);
        recompute_step(n - 1, c0 + n == sc.K);
        if (c0 + n == sc.K) {  // state is now at step K: seed of the final step
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)sc.K * Ns + wl;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    lp[p] = load_pair(a.gP + row, q, vx[p], vy[p]);
                    lv[p] = a.gV ? load_pair(a.gV + row, q, vx[p], vy[p]) : F2(0.0f);
                }
            } else {
                const int k = sc.K;
                const bool obs = sc.n_obs > 0 && (k % sc.obs_stride) == 0 && k / sc.obs_stride <= sc.n_obs;
                if (obs) {
                    const float *y = a.targets + sc.tgt_off + (size_t)(k / sc.obs_stride - 1) * Ns + wl;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const int q = 64 * p + 2 * lane;
                        f2 r = residual2(st[p], load_pair(y, q, vx[p], vy[p]));
                        r.x = vx[p] ? r.x : 0.0f;
                        r.y = vy[p] ? r.y : 0.0f;
                        lp[p] = mul2(seed_scale, r);
                        lseg = fma2(r, r, lseg);
                    }
                }
            }
        }
        kahan_add(lsum, lcomp, __fadd_rn(lseg.x, lseg.y));
        grp_sync(g);  // the whole group's tape is written

        // last observed step <= c0 + n - 1 (for the MSE seeds of the sweep)
        int row_hi = (c0 + n - 1) / sc.obs_stride;  // target row + 1 of obs_hi
        int obs_hi = row_hi * sc.obs_stride;
        AdjJac2 J[NP];
        {
            const float *rv = tv + (n - 1) * SLG + wb, *rg = tg + (n - 1) * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                const f2 v = lds2(rv + q);
                const f2 vh = make_float2(wb + q > 0 ? rv[q - 1] : 0.0f, v.x);
                J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min, qc[p]);
            }
        }
        // one reverse step; the coefficients of step s - 1 are evaluated inside
        // it (next_j) for every step but the last, which is peeled off so that
        // the loop body has no branch around them
        auto reverse_step = [&](const int s, auto next_j) {
            const int k = c0 + s;
            f2 to_lp[NP], to_lv[NP], t1[NP], nlv[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const f2 mu = mul2(F2(dt), lv[p]);
                to_lp[p] = mul2(mu, J[p].Aph);
                to_lv[p] = mul2(mu, J[p].Avh);
                t1[p] = sub2(lp[p], to_lp[p]);                          // lp + mu A_p
                nlv[p] = fma2(mu, J[p].Av, fma2(F2(dt), lp[p], lv[p]));  // dt lp + lv + mu A_v
                sacc[0][p] = fma2(mu, J[p].w0n, sacc[0][p]);
                sacc[1][p] = fma2(mu, J[p].w0nv, sacc[1][p]);
                sacc[2][p] = fma2(mu, J[p].w0nvdv, sacc[2][p]);
                sacc[3][p] = fma2(mu, J[p].fa, sacc[3][p]);
                sacc[4][p] = fma2(mu, J[p].frd, sacc[4][p]);
                if (WD) sacc[5][p] = fma2(mu, J[p].frdl, sacc[5][p]);
            }
            if constexpr (decltype(next_j)::value) {
                const float *rv = tv + (s - 1) * SLG + wb, *rg = tg + (s - 1) * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    const f2 v = lds2(rv + q);
                    const f2 vh = make_float2(wb + q > 0 ? rv[q - 1] : 0.0f, v.x);
                    J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min, qc[p]);
                }
            }
            float in_p, in_v;
            grp_follow_in(g, to_lp[0].x, to_lv[0].x, in_p, in_v, fp);
            f2 from_p[NP], from_v[NP];
            follower_vals2<NP>(to_lp, from_p, lane, in_p);
            follower_vals2<NP>(to_lv, from_v, lane, in_v);
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)k * Ns + wl;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    lp[p] = add2(add2(t1[p], from_p[p]), load_pair(a.gP + row, q, vx[p], vy[p]));
                    lv[p] = add2(nlv[p], from_v[p]);
                    if (a.gV) lv[p] = add2(lv[p], load_pair(a.gV + row, q, vx[p], vy[p]));
                }
            } else {
                // the step's seed, selected to 0 where the step is not observed
                const bool hit = k == obs_hi;
                const bool on = hit && k >= 1 && row_hi <= sc.n_obs;
                const float *rr = tr + s * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    f2 sd = lds2(rr + 64 * p + 2 * lane);
                    sd.x = on ? sd.x : 0.0f;
                    sd.y = on ? sd.y : 0.0f;
                    lp[p] = add2(add2(t1[p], from_p[p]), sd);
                    lv[p] = add2(nlv[p], from_v[p]);
                }
                obs_hi -= hit ? sc.obs_stride : 0;
                row_hi -= hit ? 1 : 0;
            }
        };
        for (int s = n - 1; s >= 1; --s) reverse_step(s, BoolC<true>{});
        reverse_step(0, BoolC<false>{});
        grp_sync(g);  // the tape may be overwritten by the next block
        if (a.bwd_pf) par ^= 1;
      }
      if (cs > 0 && (n_ck - cs) % fold_every == 0)
          fold_sums<NP, WD>(a, s_idx, g, sacc, n_ck - cs > fold_every, false);
    }
    if (n_ck > fold_every) fold_sums<NP, WD>(a, s_idx, g, sacc, true, true);

    segment_epilogue<NP, ADAM, WD, D4>(a, sg, lane, wb, kc, sacc, lp, lv, vx, vy);
    if (!DENSE) {
        const double part = warp_sum_double((double)lsum - (double)lcomp) * (double)sc.inv_nobs;
        if (lane == 0) a.loss_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

// Register budgets: 2 vehicles per thread fit 128 registers (2 blocks of 8
// warps per SM); 4 per thread need ~168 without spilling, so their blocks
// are 4 warps (3 blocks per SM) unless the segment has 8 warps (256 threads,
// one block per SM); 8 per thread use up to 255.
template <int VPT, int GW>
struct BwdBounds {
    static constexpr bool narrow = VPT == 4 && GW < 8;
    static constexpr int threads = narrow ? 128 : 256;
    static constexpr int blocks = VPT == 2 ? 2 : (narrow ? 3 : 1);
};

// The warps per segment GW are a compile-time constant of each kernel: the
// group exchange, its barriers and every slot offset of the shared tape then
// fold into immediates (measured on GB300 at 4 vehicles x 4 warps: 7 % fewer
// instructions and an 11 % shorter adjoint than with GW read from SimArgs).
template <int VPT, int GW, bool DENSE, bool ADAM, bool WD, bool SUB>
__global__ void __launch_bounds__(BwdBounds<VPT, GW>::threads, BwdBounds<VPT, GW>::blocks)
backward_kernel(SimArgs a)
{
    constexpr int NP = VPT / 2;
    constexpr int G = GW;
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5;
    float *gbase = smem + (warp / G) * bwd_group_floats(VPT, DENSE, a.tape_T, G, a.bwd_pf != 0);
    float *ctrl = gbase + bwd_group_floats(VPT, DENSE, a.tape_T, G, a.bwd_pf != 0) - grp_ctrl_floats(G);
    Grp g = make_grp(G, ctrl);
    int par = 0;
    for (;;) {
        const int s_idx = grp_next(g, a.work, par);
        if (s_idx >= *a.n_seg) break;
        const Seg sg = a.seg[s_idx];
        const ScenDesc sc = a.scen_tab ? a.scen_tab[sg.scen] : a.scen0;
        const int lb = sg.veh_begin - sc.veh_begin;
        VehConst2 kc[NP];
        State2 st[NP];
        bool vx[NP], vy[NP];
        load_vehicles<NP>(a, sg, g.lane, g.w * 64 * NP, kc, st, vx, vy);
        if constexpr (SUB) {
            if (segment_is_d4<NP>(kc, vx, vy))
                backward_segment_blocks<NP, DENSE, ADAM, WD, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
            else
                backward_segment_blocks<NP, DENSE, ADAM, WD, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
        } else {
            if (segment_is_d4<NP>(kc, vx, vy))
                backward_segment<NP, DENSE, ADAM, WD, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
            else
                backward_segment<NP, DENSE, ADAM, WD, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
        }
    }
}

// Kernel variants of one (vehicles per thread, warps per segment) shape:
// seeds from dense gradients or from targets, fused Adam or gradient output,
// with or without the delta gradient, and tape blocks (SUB).
template <int VPT, int GW, bool SUB>
inline void *backward_fn_t(bool dense, bool adam, bool wd)
{
    if (dense)
        return wd ? (void *)backward_kernel<VPT, GW, true, false, true, SUB>
                  : (void *)backward_kernel<VPT, GW, true, false, false, SUB>;
    if (adam) return (void *)backward_kernel<VPT, GW, false, true, false, SUB>;
    return wd ? (void *)backward_kernel<VPT, GW, false, false, true, SUB>
              : (void *)backward_kernel<VPT, GW, false, false, false, SUB>;
}

}  // namespace idm
