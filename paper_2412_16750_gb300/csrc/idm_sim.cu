// Simulation kernels of libidm for sm_103a: initial gaps, lane packing into
// warp segments, the fused forward (Eq. 1-3 with the Sec. III-C bounds,
// squared-error loss, checkpoints) and the reverse-time adjoint with
// checkpoint recompute (arXiv 2412.16750, Sec. III and IV-A).
//
// Mapping.  Vehicles are ordered lane by lane, head first.  Whole lanes are
// packed into warp segments of at most 32*VPT vehicles; slot q of a segment
// lives in register j = q / 32 of thread q % 32, so every per-step load or
// store of a segment is one contiguous 128-byte row per register.  The
// leader of slot q is slot q-1, fetched by one warp shuffle; lanes never
// cross a segment, so a warp runs all K steps of its lanes with no
// inter-warp synchronisation.  Warps take segments from a global atomic
// counter (persistent grid).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idm_device.cuh"
#include "idm_internal.h"

namespace idm {

// ---------------------------------------------------------------------------
// Initial gaps g0[i] = p_init[i-1] - p_init[i] - length[i-1] (Sec. III-A),
// +inf for lane heads.
// ---------------------------------------------------------------------------
__global__ void gap_kernel(const float *p_init, const float *length, int N, float *g0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (i == 0) { g0[0] = INFINITY; return; }
    double g = (double)p_init[i - 1] - (double)p_init[i] - (double)length[i - 1];
    g0[i] = (float)g;
}

__global__ void head_kernel(const int *lane_off, int n_lanes, int N, float *g0, unsigned *status)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lanes) return;
    int a = lane_off[l], e = lane_off[l + 1];
    bool bad = e < a || a < 0 || e > N || (l == 0 && a != 0) || (l == n_lanes - 1 && e != N);
    if (bad) { atomicOr(status, IDM_STATUS_BAD_LANE_OFF); return; }
    if (a < e) g0[a] = INFINITY;
}

cudaError_t launch_prep_gap(const int *lane_off, int n_lanes, const float *p_init, const float *length,
                            int N, float *g0, unsigned *status, cudaStream_t st)
{
    if (N > 0) gap_kernel<<<(N + 255) / 256, 256, 0, st>>>(p_init, length, N, g0);
    if (n_lanes > 0) head_kernel<<<(n_lanes + 255) / 256, 256, 0, st>>>(lane_off, n_lanes, N, g0, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lane packing: each of 1024 threads packs a contiguous chunk of lanes
// greedily into segments of at most `cap` vehicles (never across a scenario
// boundary); a block scan places the chunks' segments.  A lane longer than
// cap is skipped and flagged.
// ---------------------------------------------------------------------------
constexpr int BUILD_THREADS = 1024;

template <bool EMIT>
__device__ int pack_lanes(const int *lane_off, int l0, int l1, const int *scen_lane_off, int n_scen, int cap,
                          int N, Seg *out, unsigned *status)
{
    int cnt = 0, fill = 0, seg_begin = 0, cur_scen = -1;
    int s = 0;
    if (scen_lane_off) {  // scenario of lane l0
        int lo = 0, hi = n_scen - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (scen_lane_off[mid] <= l0) lo = mid; else hi = mid - 1;
        }
        s = lo;
    }
    for (int l = l0; l < l1; ++l) {
        if (scen_lane_off)
            while (s + 1 < n_scen && scen_lane_off[s + 1] <= l) ++s;
        int a = lane_off[l], e = lane_off[l + 1], n = e - a;
        if (a < 0 || e > N || n < 0) {  // malformed: never read outside [0, N)
            if (EMIT) atomicOr(status, IDM_STATUS_BAD_LANE_OFF);
            if (fill > 0) {
                if (EMIT) out[cnt] = Seg{seg_begin, fill, cur_scen < 0 ? 0 : cur_scen, 0};
                ++cnt;
                fill = 0;
            }
            continue;
        }
        if (n == 0) continue;
        bool close = fill > 0 && (fill + n > cap || s != cur_scen);
        if (n > cap) {
            if (EMIT) atomicOr(status, IDM_STATUS_LANE_TOO_LONG);
            close = fill > 0;
        }
        if (close) {
            if (EMIT) out[cnt] = Seg{seg_begin, fill, cur_scen < 0 ? 0 : cur_scen, 0};
            ++cnt;
            fill = 0;
        }
        if (n > cap) continue;
        if (fill == 0) { seg_begin = a; cur_scen = s; }
        fill += n;
    }
    if (fill > 0) {
        if (EMIT) out[cnt] = Seg{seg_begin, fill, cur_scen < 0 ? 0 : cur_scen, 0};
        ++cnt;
    }
    return cnt;
}

__global__ void __launch_bounds__(BUILD_THREADS)
build_segments_kernel(const int *lane_off, int n_lanes, const int *scen_lane_off, int n_scen, int cap, int N,
                      Seg *seg, int *n_seg, unsigned *status)
{
    __shared__ int sc[BUILD_THREADS];
    const int t = threadIdx.x;
    const int per = (n_lanes + BUILD_THREADS - 1) / BUILD_THREADS;
    const int l0 = min(n_lanes, t * per), l1 = min(n_lanes, l0 + per);
    int cnt = pack_lanes<false>(lane_off, l0, l1, scen_lane_off, n_scen, cap, N, nullptr, status);
    sc[t] = cnt;
    __syncthreads();
    for (int off = 1; off < BUILD_THREADS; off <<= 1) {  // inclusive Hillis-Steele scan
        int v = t >= off ? sc[t - off] : 0;
        __syncthreads();
        sc[t] += v;
        __syncthreads();
    }
    int base = sc[t] - cnt;
    pack_lanes<true>(lane_off, l0, l1, scen_lane_off, n_scen, cap, N, seg + base, status);
    if (t == BUILD_THREADS - 1) *n_seg = sc[t];
}

cudaError_t launch_build_segments(const int *lane_off, int n_lanes, const int *scen_lane_off, int n_scen,
                                  int cap, int N, Seg *seg, int *n_seg, unsigned *status, cudaStream_t st)
{
    build_segments_kernel<<<1, BUILD_THREADS, 0, st>>>(lane_off, n_lanes, scen_lane_off, n_scen, cap, N, seg,
                                                       n_seg, status);
    return cudaGetLastError();
}

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
    float *xl;   // [2][G] leader exchange
    float *xf;   // [2][2][G] follower exchange
};

// Shared floats of one group's control area (cells + exchange cells).
__host__ __device__ __forceinline__ int grp_ctrl_floats(int G) { return ((2 + 6 * G) + 3) & ~3; }

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
    g.xf = ctrl + 2 + 2 * G;
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

// Leader speed of this warp's first slot (0 for the group's first warp);
// last_v is this lane's value of the warp's last slot (used by lane 31).
__device__ __forceinline__ float grp_lead_in(const Grp &g, float last_v, int &xp)
{
    if (g.G == 1) return 0.0f;
    if (g.lane == 31) g.xl[xp * g.G + g.w] = last_v;
    grp_sync(g);
    const float r = g.w > 0 ? g.xl[xp * g.G + g.w - 1] : 0.0f;
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
                st[p].ph.x = ph; st[p].pl.x = 0.0f; st[p].v.x = v; st[p].gap.x = gap;
            } else {
                vy[p] = ok;
                kc[p].inv_v0.y = inv_v0; kc[p].T.y = T; kc[p].s0.y = s0; kc[p].am.y = am; kc[p].c.y = cc;
                kc[p].delta.y = dl;
                st[p].ph.y = ph; st[p].pl.y = 0.0f; st[p].v.y = v; st[p].gap.y = gap;
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

// ---------------------------------------------------------------------------
// Forward: K steps per segment, optional trajectory / speed output,
// checkpoints every C steps.  (The squared-error loss is accumulated by the
// adjoint's recompute, which evaluates the residuals anyway.)
// ---------------------------------------------------------------------------
struct FwdFlags {
    bool traj, vtraj, ckpt, eval;
};

template <int NP, bool D4>
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
    for (int k = 0;; ++k) {
        if (f.ckpt && k == next_ck && k < sc.K) {
            float *base = a.ckpt + sc.ckpt_off + (size_t)ck_idx * 4 * Ns + wl;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                store_pair(base, q, st[p].ph, vx[p], vy[p]);
                store_pair(base + (size_t)Ns, q, st[p].pl, vx[p], vy[p]);
                store_pair(base + 2 * (size_t)Ns, q, st[p].v, vx[p], vy[p]);
                store_pair(base + 3 * (size_t)Ns, q, st[p].gap, vx[p], vy[p]);
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
                if (f.vtraj) store_pair(a.vtraj + row, q, st[p].v, vx[p], vy[p]);
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

        f2 vcur[NP], vh[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) vcur[p] = st[p].v;
        const float lead_in = grp_lead_in(g, vcur[NP - 1].y, xp);
        leader_vals2<NP>(vcur, vh, lane, lead_in);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const f2 as = accel_star2<D4>(st[p].v, st[p].gap, vh[p], kc[p], sc.inv_dt, sc.a_min);
            euler2(st[p], as, vh[p], sc.dt);
        }
    }
    bool bad = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (vx[p] && !(isfinite(st[p].v.x) && isfinite(st[p].ph.x))) bad = true;
        if (vy[p] && !(isfinite(st[p].v.y) && isfinite(st[p].ph.y))) bad = true;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, IDM_STATUS_NONFINITE);
    if (f.eval) {
        const double part = warp_sum_double((double)esum - (double)ecomp) * (double)sc.inv_nobs;
        if (lane == 0) a.eval_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

template <int VPT>
__global__ void __launch_bounds__(512)
forward_kernel(SimArgs a, FwdFlags f)
{
    constexpr int NP = VPT / 2;
    extern __shared__ float fsmem[];
    const int G = a.G;
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
            forward_segment<NP, true>(a, sc, s_idx, lb, g, kc, st, vx, vy, f);
        else
            forward_segment<NP, false>(a, sc, s_idx, lb, g, kc, st, vx, vy, f);
    }
}

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
// Gradient increments accumulate in registers per checkpoint segment and
// are added to per-slot totals in shared memory.
// ---------------------------------------------------------------------------
// Shared floats of one group: tape v/gap [C][G*SL], target/seed tapes
// [C][G*SL] (MSE only), checkpoint stages [4][G*SL], totals [6][G*SL],
// control area.  With prefetch the target tape and the checkpoint stage are
// doubled and the next checkpoint segment's targets and checkpoint are
// copied (cp.async) into the idle pair while the current segment runs.
__host__ __device__ __forceinline__ int bwd_group_floats(int vpt, bool dense, int C, int G, bool pf)
{
    const int nb = pf ? 2 : 1;
    return ((dense ? 2 : 2 + nb) * C + 4 * nb + 6) * 32 * vpt * G + grp_ctrl_floats(G);
}

__device__ __forceinline__ f2 lds2(const float *p) { return *reinterpret_cast<const f2 *>(p); }
__device__ __forceinline__ void sts2(float *p, f2 x) { *reinterpret_cast<f2 *>(p) = x; }

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
    float *tg = tv + a.C * SLG;
    float *trb = tg + a.C * SLG;                    // nb tapes: targets, then seeds (MSE only)
    float *ckb = tv + (DENSE ? 2 : 2 + nb) * a.C * SLG;  // nb checkpoint stages [4][SLG]
    float *acc = ckb + nb * 4 * SLG;                // gradient totals [6][SLG]
    const int Ns = sc.n_veh;
    const int wl = lb + wb;                         // scenario-local index of this warp's first slot
    const float dt = sc.dt;
    const f2 seed_scale = F2(2.0f * sc.inv_nobs);
    int xp = 0, fp = 0;
    float lsum = 0.0f, lcomp = 0.0f;  // squared residuals (MSE): Kahan across checkpoint segments

    f2 lp[NP], lv[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        lp[p] = F2(0.0f);
        lv[p] = F2(0.0f);
#pragma unroll
        for (int q = 0; q < 6; ++q) sts2(acc + q * SLG + wb + 64 * p + 2 * lane, F2(0.0f));
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
        float *ck = ckb + par * 4 * SLG;
        const float *base = a.ckpt + sc.ckpt_off + (size_t)cs * 4 * Ns + wl;
#pragma unroll
        for (int f = 0; f < 4; ++f) prefetch_row<NP>(ck + f * SLG + wb, base + (size_t)f * Ns, lane, vx, vy);
        cp_async_commit();
    };

    const int n_ck = (sc.K + a.C - 1) / a.C;
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
            const float *ck = ckb + par * 4 * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                const f2 ph = lds2(ck + q), pl = lds2(ck + SLG + q), v = lds2(ck + 2 * SLG + q);
                const f2 gp = lds2(ck + 3 * SLG + q);
                st[p].ph = make_float2(vx[p] ? ph.x : 0.0f, vy[p] ? ph.y : 0.0f);
                st[p].pl = make_float2(vx[p] ? pl.x : 0.0f, vy[p] ? pl.y : 0.0f);
                st[p].v = make_float2(vx[p] ? v.x : 0.0f, vy[p] ? v.y : 0.0f);
                st[p].gap = make_float2(vx[p] ? gp.x : INFINITY, vy[p] ? gp.y : INFINITY);
            }
        }
        if (a.bwd_pf && cs > 0) prefetch_segment(cs - 1);  // lands while this segment runs
        f2 lseg = F2(0.0f);
        // recompute the segment into the tape
        for (int s = 0; s < n; ++s) {
            const int k = c0 + s;
            float *rv = tv + s * SLG + wb, *rg = tg + s * SLG + wb;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q = 64 * p + 2 * lane;
                sts2(rv + q, st[p].v);
                sts2(rg + q, st[p].gap);
            }
            if (!DENSE && k == obs_k) {
                if (obs_row < sc.n_obs) {
                    float *rr = tr + s * SLG + wb;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const int q = 64 * p + 2 * lane;
                        f2 r = residual2(st[p], lds2(rr + q));
                        r.x = vx[p] ? r.x : 0.0f;
                        r.y = vy[p] ? r.y : 0.0f;
                        sts2(rr + q, mul2(seed_scale, r));
                        lseg = fma2(r, r, lseg);
                    }
                }
                obs_k += sc.obs_stride;
                ++obs_row;
            }
            f2 vcur[NP], vh[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) vcur[p] = st[p].v;
            const float lead_in = grp_lead_in(g, vcur[NP - 1].y, xp);
            leader_vals2<NP>(vcur, vh, lane, lead_in);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const f2 as = accel_star2<D4>(st[p].v, st[p].gap, vh[p], kc[p], sc.inv_dt, sc.a_min);
                euler2(st[p], as, vh[p], dt);
            }
        }
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

        f2 sacc[6][NP];
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
            for (int p = 0; p < NP; ++p) sacc[q][p] = F2(0.0f);

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
                J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min);
            }
        }
        for (int s = n - 1; s >= 0; --s) {
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
            if (s > 0) {
                const float *rv = tv + (s - 1) * SLG + wb, *rg = tg + (s - 1) * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int q = 64 * p + 2 * lane;
                    const f2 v = lds2(rv + q);
                    const f2 vh = make_float2(wb + q > 0 ? rv[q - 1] : 0.0f, v.x);
                    J[p] = adjoint_jac2<WD, D4>(v, lds2(rg + q), vh, kc[p], sc.inv_dt, sc.a_min);
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
            } else if (k == obs_hi && k >= 1 && row_hi <= sc.n_obs) {
                const float *rr = tr + s * SLG + wb;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    lp[p] = add2(add2(t1[p], from_p[p]), lds2(rr + 64 * p + 2 * lane));
                    lv[p] = add2(nlv[p], from_v[p]);
                }
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    lp[p] = add2(t1[p], from_p[p]);
                    lv[p] = add2(nlv[p], from_v[p]);
                }
            }
            if (!DENSE && k == obs_hi) {
                obs_hi -= sc.obs_stride;
                --row_hi;
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float *ap = acc + q * SLG + wb + 64 * p + 2 * lane;
                sts2(ap, add2(lds2(ap), sacc[q][p]));
            }
        grp_sync(g);  // the tape may be overwritten by the next segment
    }

    // epilogue: parameter gradients from the factored sums
    bool bad = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(c ? vy[p] : vx[p])) continue;
            const int q = wb + 64 * p + 2 * lane + c;
            const int gi = sg.veh_begin + q;
            const float v0 = a.v0[gi], b = a.b[gi];
            const float am = c ? kc[p].am.y : kc[p].am.x, cc = c ? kc[p].c.y : kc[p].c.x;
            const float dl = c ? kc[p].delta.y : kc[p].delta.x;
            const float A0 = acc[0 * SLG + q], A1 = acc[1 * SLG + q], A2 = acc[2 * SLG + q];
            const float A3 = acc[3 * SLG + q], A4 = acc[4 * SLG + q], A5 = acc[5 * SLG + q];
            float gr[6];
            gr[0] = am * dl * A4 / v0;                 // v0
            gr[1] = -A1;                               // T
            gr[2] = -A0;                               // s0
            gr[3] = A3 + A2 * cc / (2.0f * am);        // a_max
            gr[4] = A2 * cc / (2.0f * b);              // b
            gr[5] = -am * A5;                          // delta
            for (int r = 0; r < 6; ++r) bad |= !isfinite(gr[r]);
            if (ADAM) {
                const int it = a.iter;
                const int t = it + 1;
                const float lr = a.n_iter > 1 ? a.lr0 + (a.lr1 - a.lr0) * (float)it / (float)(a.n_iter - 1) : a.lr0;
                const float bc1 = 1.0f - powf(0.9f, (float)t), bc2 = 1.0f - powf(0.999f, (float)t);
                float *th[5] = {const_cast<float *>(a.v0), const_cast<float *>(a.T), const_cast<float *>(a.s0),
                                const_cast<float *>(a.am), const_cast<float *>(a.b)};
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const size_t mi = (size_t)r * a.N_total + gi;
                    float m = 0.9f * a.adam_m[mi] + 0.1f * gr[r];
                    float vv = 0.999f * a.adam_v[mi] + 0.001f * gr[r] * gr[r];
                    a.adam_m[mi] = m;
                    a.adam_v[mi] = vv;
                    float x = th[r][gi] - lr * (m / bc1) / (sqrtf(vv / bc2) + 1e-8f);
                    x = fminf(fmaxf(x, a.lo[r]), a.hi[r]);
                    th[r][gi] = x;
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
    if (!DENSE) {
        const double part = warp_sum_double((double)lsum - (double)lcomp) * (double)sc.inv_nobs;
        if (lane == 0) a.loss_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

// Register budgets: 2 vehicles per thread fit 128 registers (2 blocks of 8
// warps per SM); 4 per thread need ~168 without spilling, so their blocks
// are 4 warps (3 blocks per SM) unless the segment has 8 warps (BIG, 256
// threads, one block per SM); 8 per thread use up to 255.
template <int VPT, bool BIG>
struct BwdBounds {
    static constexpr int threads = (VPT == 4 && !BIG) ? 128 : 256;
    static constexpr int blocks = VPT == 2 ? 2 : ((VPT == 4 && !BIG) ? 3 : 1);
};

template <int VPT, bool DENSE, bool ADAM, bool WD, bool BIG>
__global__ void __launch_bounds__(BwdBounds<VPT, BIG>::threads, BwdBounds<VPT, BIG>::blocks)
backward_kernel(SimArgs a)
{
    constexpr int NP = VPT / 2;
    extern __shared__ float smem[];
    const int G = a.G;
    const int warp = threadIdx.x >> 5;
    float *gbase = smem + (warp / G) * bwd_group_floats(VPT, DENSE, a.C, G, a.bwd_pf != 0);
    float *ctrl = gbase + bwd_group_floats(VPT, DENSE, a.C, G, a.bwd_pf != 0) - grp_ctrl_floats(G);
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
        if (segment_is_d4<NP>(kc, vx, vy))
            backward_segment<NP, DENSE, ADAM, WD, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
        else
            backward_segment<NP, DENSE, ADAM, WD, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, vx, vy);
    }
}

// ---------------------------------------------------------------------------
// Deterministic loss reduction over segments (fixed order).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
loss_finalize_kernel(const double *part, const int *n_seg, int per_seg, double *out)
{
    __shared__ double sh[1024];
    const int n = *n_seg * per_seg;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && out) *out = sh[0];
}

cudaError_t launch_loss_finalize(const double *loss_part, const int *n_seg, int per_seg, double *out, cudaStream_t st)
{
    loss_finalize_kernel<<<1, 1024, 0, st>>>(loss_part, n_seg, per_seg, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
cudaError_t launch_forward(int vpt, int G, bool traj, bool vtraj, bool ckpt, const SimArgs &a, int grid, int wpb,
                           cudaStream_t st)
{
    FwdFlags f{traj, vtraj, ckpt, a.eval_targets != nullptr && a.eval_part != nullptr};
    void *fn = nullptr;
    switch (vpt) {
    case 2: fn = (void *)forward_kernel<2>; break;
    case 4: fn = (void *)forward_kernel<4>; break;
    case 8: fn = (void *)forward_kernel<8>; break;
    default: return cudaErrorInvalidValue;
    }
    const size_t smem = forward_smem_bytes(vpt, G, wpb);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SimArgs args = a;
    args.G = G;
    void *params[] = {&args, &f};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * wpb), params, smem, st);
}

size_t backward_smem_bytes(int vpt, bool dense_seed, int C, int G, int wpb, bool prefetch)
{
    return (size_t)bwd_group_floats(vpt, dense_seed, C, G, prefetch) * (wpb / G) * sizeof(float);
}

size_t forward_smem_bytes(int vpt, int G, int wpb)
{
    (void)vpt;
    return (size_t)grp_ctrl_floats(G) * (wpb / G) * sizeof(float);
}

// Kernel variants of the adjoint: seeds from dense gradients or from targets,
// fused Adam or gradient output, with or without the delta gradient; for 4
// vehicles per thread a 4-warp and an 8-warp block form.
template <int VPT, bool BIG>
static void *backward_fn(bool dense, bool adam, bool wd)
{
    if (dense)
        return wd ? (void *)backward_kernel<VPT, true, false, true, BIG>
                  : (void *)backward_kernel<VPT, true, false, false, BIG>;
    if (adam) return (void *)backward_kernel<VPT, false, true, false, BIG>;
    return wd ? (void *)backward_kernel<VPT, false, false, true, BIG>
              : (void *)backward_kernel<VPT, false, false, false, BIG>;
}

static void *backward_fn_v(int vpt, bool dense, bool adam, bool wd, int wpb)
{
    switch (vpt) {
    case 2: return backward_fn<2, false>(dense, adam, wd);
    case 4: return wpb > 4 ? backward_fn<4, true>(dense, adam, wd) : backward_fn<4, false>(dense, adam, wd);
    case 8: return backward_fn<8, false>(dense, adam, wd);
    }
    return nullptr;
}

int backward_max_warps(int vpt, int G) { return (vpt == 4 && G <= 4) ? 4 : 8; }

int backward_resident_warps(int vpt, int G)
{
    if (vpt == 2) return 16;
    if (vpt == 4 && G <= 4) return 12;
    return 8;
}

cudaError_t launch_backward(int vpt, int G, bool dense_seed, bool adam, bool want_delta, const SimArgs &a, int grid,
                            int wpb, cudaStream_t st)
{
    if (dense_seed && adam) return cudaErrorInvalidValue;
    if (wpb > backward_max_warps(vpt, G) || wpb % G) return cudaErrorInvalidValue;
    void *fn = backward_fn_v(vpt, dense_seed, adam, want_delta && !adam, wpb);
    if (!fn) return cudaErrorInvalidValue;
    size_t smem = backward_smem_bytes(vpt, dense_seed, a.C, G, wpb, a.bwd_pf != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SimArgs args = a;
    args.G = G;
    void *params[] = {&args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * wpb), params, smem, st);
}

int occupancy_blocks(int vpt, int G, bool backward, bool dense, bool adam, bool want_delta, int wpb, size_t smem)
{
    void *fn = nullptr;
    if (!backward) {
        switch (vpt) {
        case 2: fn = (void *)forward_kernel<2>; break;
        case 4: fn = (void *)forward_kernel<4>; break;
        case 8: fn = (void *)forward_kernel<8>; break;
        }
        smem = forward_smem_bytes(vpt, G, wpb);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
        fn = backward_fn_v(vpt, dense, adam, want_delta && !adam, wpb);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (!fn) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * wpb, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace idm
