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

// dst/src_row already point at this warp's first slot.
template <int VPT>
__device__ __forceinline__ void prefetch_row(float *dst, const float *src_row, int lane, const bool (&valid)[VPT])
{
#pragma unroll
    for (int j = 0; j < VPT; ++j)
        if (valid[j]) cp_async4(dst + lane + 32 * j, src_row + lane + 32 * j);
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

// Leader speed of this warp's first slot (0 for the group's first warp).
template <int VPT>
__device__ __forceinline__ float grp_lead_in(const Grp &g, const float (&v)[VPT], int &xp)
{
    if (g.G == 1) return 0.0f;
    if (g.lane == 31) g.xl[xp * g.G + g.w] = v[VPT - 1];
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

template <int VPT>
__device__ __forceinline__ void load_vehicles(const SimArgs &a, const Seg &sg, int lane, int wb, VehConst (&kc)[VPT],
                                              State (&st)[VPT], bool (&valid)[VPT])
{
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        const int q = wb + lane + 32 * j;
        valid[j] = q < sg.n_veh;
        if (valid[j]) {
            const int gi = sg.veh_begin + q;
            kc[j] = make_const(a.v0[gi], a.T[gi], a.s0[gi], a.am[gi], a.b[gi], a.delta[gi]);
            st[j] = State{a.p_init[gi], 0.0f, a.v_init[gi], a.g0[gi]};
        } else {
            kc[j] = ghost_const();
            st[j] = State{0.0f, 0.0f, 0.0f, INFINITY};
        }
    }
}


// True when every occupied slot of the warp has delta == 4, so the step body
// can use the squaring form of (v/v0)^delta with no branch.  (Both variants
// execute the same sequence of group barriers.)
template <int VPT>
__device__ __forceinline__ bool segment_is_d4(const VehConst (&kc)[VPT], const bool (&valid)[VPT])
{
    bool ok = true;
#pragma unroll
    for (int j = 0; j < VPT; ++j)
        if (valid[j] && kc[j].delta != 4.0f) ok = false;
    return __all_sync(FULL, ok);
}

// ---------------------------------------------------------------------------
// Forward: K steps per segment, optional trajectory / speed output,
// checkpoints every C steps.  (The squared-error loss is accumulated by the
// adjoint's recompute, which evaluates the residuals anyway.)
// ---------------------------------------------------------------------------
struct FwdFlags {
    bool traj, vtraj, ckpt;
};

template <int VPT, bool D4>
__device__ __forceinline__ void forward_segment(const SimArgs &a, const ScenDesc &sc, int lb, Grp &g,
                                                const VehConst (&kc)[VPT], State (&st)[VPT],
                                                const bool (&valid)[VPT], FwdFlags f)
{
    const int lane = g.lane;
    const int Ns = sc.n_veh;
    const int wl = lb + g.w * 32 * VPT;  // scenario-local index of this warp's first slot
    int next_ck = 0, ck_idx = 0;
    int xp = 0;
    for (int k = 0;; ++k) {
        if (f.ckpt && k == next_ck && k < sc.K) {
            float *base = a.ckpt + sc.ckpt_off + (size_t)ck_idx * 4 * Ns + wl;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if (!valid[j]) continue;
                const int q = lane + 32 * j;
                base[q] = st[j].ph;
                base[(size_t)Ns + q] = st[j].pl;
                base[2 * (size_t)Ns + q] = st[j].v;
                base[3 * (size_t)Ns + q] = st[j].gap;
            }
            next_ck += a.C;
            ++ck_idx;
        }
        if (f.traj || f.vtraj) {
            const size_t row = sc.traj_off + (size_t)k * Ns + wl;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if (!valid[j]) continue;
                const int q = lane + 32 * j;
                if (f.traj) a.traj[row + q] = position(st[j]);
                if (f.vtraj) a.vtraj[row + q] = st[j].v;
            }
        }
        if (k == sc.K) break;

        float vcur[VPT], vh[VPT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) vcur[j] = st[j].v;
        const float lead_in = grp_lead_in<VPT>(g, vcur, xp);
        leader_vals<VPT>(vcur, vh, lane, lead_in);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            float as = accel_star<D4>(st[j].v, st[j].gap, vh[j], kc[j], sc.inv_dt, sc.a_min);
            euler(st[j], as, vh[j], sc.dt);
        }
    }
    bool bad = false;
#pragma unroll
    for (int j = 0; j < VPT; ++j)
        if (valid[j] && !(isfinite(st[j].v) && isfinite(st[j].ph))) bad = true;
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, IDM_STATUS_NONFINITE);
}

template <int VPT>
__global__ void __launch_bounds__(512)
forward_kernel(SimArgs a, FwdFlags f)
{
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
        VehConst kc[VPT];
        State st[VPT];
        bool valid[VPT];
        load_vehicles<VPT>(a, sg, g.lane, g.w * 32 * VPT, kc, st, valid);
        if (segment_is_d4<VPT>(kc, valid))
            forward_segment<VPT, true>(a, sc, lb, g, kc, st, valid, f);
        else
            forward_segment<VPT, false>(a, sc, lb, g, kc, st, valid, f);
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
// (and across warps through the group's exchange cells).  Gradient
// increments accumulate in registers per checkpoint segment and are added
// to per-slot totals in shared memory.
// ---------------------------------------------------------------------------
// Shared floats of one group: tape v/gap[/seed] [C][G*SL], totals [6][G*SL],
// control area.
__host__ __device__ __forceinline__ int bwd_group_floats(int vpt, bool dense, int C, int G)
{
    return ((dense ? 2 : 3) * C + 6) * 32 * vpt * G + grp_ctrl_floats(G);
}

template <int VPT, bool DENSE, bool ADAM, bool WD, bool D4>
__device__ __forceinline__ void backward_segment(const SimArgs &a, const ScenDesc &sc, const Seg &sg, int s_idx, int lb,
                                                 Grp &g, float *tv, const VehConst (&kc)[VPT], State (&st)[VPT],
                                                 const bool (&valid)[VPT])
{
    constexpr int SL = 32 * VPT;
    const int SLG = SL * g.G;
    const int lane = g.lane;
    const int wb = g.w * SL;                      // this warp's first slot in the group
    float *tg = tv + a.C * SLG;
    float *tr = tg + a.C * SLG;                   // targets, then seeds (MSE only)
    float *acc = tv + (DENSE ? 2 : 3) * a.C * SLG;  // gradient totals [6][SLG]
    const int Ns = sc.n_veh;
    const int wl = lb + wb;                       // scenario-local index of this warp's first slot
    const float dt = sc.dt;
    const float seed_scale = 2.0f * sc.inv_nobs;
    int xp = 0, fp = 0;
    float lsum = 0.0f, lcomp = 0.0f;  // squared residuals (MSE): Kahan across checkpoint segments

    float lp[VPT], lv[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        lp[j] = 0.0f;
        lv[j] = 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q * SLG + wb + lane + 32 * j] = 0.0f;
    }

    const int n_ck = (sc.K + a.C - 1) / a.C;
    for (int cs = n_ck - 1; cs >= 0; --cs) {
        const int c0 = cs * a.C;
        const int n = min(a.C, sc.K - c0);
        // first observed step >= max(c0, 1) and its target row (one division
        // per checkpoint segment; the step loops count instead of dividing)
        int obs_row = (c0 + sc.obs_stride - 1) / sc.obs_stride;
        if (obs_row == 0) obs_row = 1;
        int obs_k = obs_row * sc.obs_stride;
        obs_row -= 1;
        if (!DENSE) {  // fetch the segment's observed targets into the seed tape
            const float *yrow = a.targets + sc.tgt_off + (size_t)obs_row * Ns + wl;
            for (int k = obs_k, r = obs_row; k < c0 + n && r < sc.n_obs; k += sc.obs_stride, ++r, yrow += Ns)
                prefetch_row<VPT>(tr + (k - c0) * SLG + wb, yrow, lane, valid);
            cp_async_commit();
        }
        {
            const float *base = a.ckpt + sc.ckpt_off + (size_t)cs * 4 * Ns + wl;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if (!valid[j]) continue;
                const int q = lane + 32 * j;
                st[j] = State{base[q], base[(size_t)Ns + q], base[2 * (size_t)Ns + q], base[3 * (size_t)Ns + q]};
            }
        }
        if (!DENSE) cp_async_wait<0>();
        float lseg = 0.0f;
        // recompute the segment into the tape
        for (int s = 0; s < n; ++s) {
            const int k = c0 + s;
            float *rv = tv + s * SLG + wb, *rg = tg + s * SLG + wb;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                rv[lane + 32 * j] = st[j].v;
                rg[lane + 32 * j] = st[j].gap;
            }
            if (!DENSE && k == obs_k) {
                if (obs_row < sc.n_obs) {
                    float *rr = tr + s * SLG + wb;
#pragma unroll
                    for (int j = 0; j < VPT; ++j) {
                        float r = valid[j] ? residual(st[j], rr[lane + 32 * j]) : 0.0f;
                        rr[lane + 32 * j] = __fmul_rn(seed_scale, r);
                        lseg = __fmaf_rn(r, r, lseg);
                    }
                }
                obs_k += sc.obs_stride;
                ++obs_row;
            }
            float vcur[VPT], vh[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j) vcur[j] = st[j].v;
            const float lead_in = grp_lead_in<VPT>(g, vcur, xp);
            leader_vals<VPT>(vcur, vh, lane, lead_in);
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                float as = accel_star<D4>(st[j].v, st[j].gap, vh[j], kc[j], sc.inv_dt, sc.a_min);
                euler(st[j], as, vh[j], dt);
            }
        }
        if (cs == n_ck - 1) {  // state is now at step K: seed of the final step
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)sc.K * Ns + wl;
#pragma unroll
                for (int j = 0; j < VPT; ++j) {
                    if (!valid[j]) continue;
                    lp[j] = a.gP[row + lane + 32 * j];
                    lv[j] = a.gV ? a.gV[row + lane + 32 * j] : 0.0f;
                }
            } else {
                const int k = sc.K;
                const bool obs = sc.n_obs > 0 && (k % sc.obs_stride) == 0 && k / sc.obs_stride <= sc.n_obs;
                if (obs) {
                    const float *y = a.targets + sc.tgt_off + (size_t)(k / sc.obs_stride - 1) * Ns + wl;
#pragma unroll
                    for (int j = 0; j < VPT; ++j)
                        if (valid[j]) {
                            const float r = residual(st[j], __ldg(y + lane + 32 * j));
                            lp[j] = __fmul_rn(seed_scale, r);
                            kahan_add(lsum, lcomp, __fmul_rn(r, r));
                        }
                }
            }
        }
        kahan_add(lsum, lcomp, lseg);
        grp_sync(g);  // the whole group's tape is written

        float sacc[6][VPT];
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
            for (int j = 0; j < VPT; ++j) sacc[q][j] = 0.0f;

        // last observed step <= c0 + n - 1 (for the MSE seeds of the sweep)
        int row_hi = (c0 + n - 1) / sc.obs_stride;  // target row + 1 of obs_hi
        int obs_hi = row_hi * sc.obs_stride;
        // The step-k coefficients do not depend on the adjoint, so those of
        // step k-1 are evaluated while the dependent chain of step k runs.
        AdjJac J[VPT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            const int q = wb + lane + 32 * j;
            const float *rv = tv + (n - 1) * SLG, *rg = tg + (n - 1) * SLG;
            J[j] = adjoint_jac<WD, D4>(rv[q], rg[q], q > 0 ? rv[q - 1] : 0.0f, kc[j], sc.inv_dt, sc.a_min);
        }
        for (int s = n - 1; s >= 0; --s) {
            const int k = c0 + s;
            float own_p[VPT], own_v[VPT], to_lp[VPT], to_lv[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                const float mu = __fmul_rn(dt, lv[j]);
                own_p[j] = mu * J[j].Ap;
                own_v[j] = mu * J[j].Av;
                to_lp[j] = -own_p[j];
                to_lv[j] = mu * J[j].Avh;
                sacc[0][j] += mu * J[j].w0;
                sacc[1][j] += mu * J[j].w0v;
                sacc[2][j] += mu * J[j].w0vdv;
                sacc[3][j] += mu * J[j].fa;
                sacc[4][j] += mu * J[j].frd;
                if (WD) sacc[5][j] += mu * J[j].frdl;
            }
            if (s > 0) {
                const float *rv = tv + (s - 1) * SLG, *rg = tg + (s - 1) * SLG;
#pragma unroll
                for (int j = 0; j < VPT; ++j) {
                    const int q = wb + lane + 32 * j;
                    J[j] = adjoint_jac<WD, D4>(rv[q], rg[q], q > 0 ? rv[q - 1] : 0.0f, kc[j], sc.inv_dt, sc.a_min);
                }
            }
            float in_p, in_v;
            grp_follow_in(g, to_lp[0], to_lv[0], in_p, in_v, fp);
            float from_p[VPT], from_v[VPT];
            follower_vals<VPT>(to_lp, from_p, lane, in_p);
            follower_vals<VPT>(to_lv, from_v, lane, in_v);
            float seed_p[VPT], seed_v[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j) { seed_p[j] = 0.0f; seed_v[j] = 0.0f; }
            if (DENSE) {
                const size_t row = sc.traj_off + (size_t)k * Ns + wl;
#pragma unroll
                for (int j = 0; j < VPT; ++j) {
                    if (!valid[j]) continue;
                    seed_p[j] = a.gP[row + lane + 32 * j];
                    if (a.gV) seed_v[j] = a.gV[row + lane + 32 * j];
                }
            } else if (k == obs_hi) {
                if (k >= 1 && row_hi <= sc.n_obs) {
                    const float *rr = tr + s * SLG + wb;
#pragma unroll
                    for (int j = 0; j < VPT; ++j) seed_p[j] = rr[lane + 32 * j];
                }
                obs_hi -= sc.obs_stride;
                --row_hi;
            }
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                float nlp = lp[j] + own_p[j] + from_p[j] + seed_p[j];
                float nlv = dt * lp[j] + lv[j] + own_v[j] + from_v[j] + seed_v[j];
                lp[j] = nlp;
                lv[j] = nlv;
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
            for (int j = 0; j < VPT; ++j) acc[q * SLG + wb + lane + 32 * j] += sacc[q][j];
        grp_sync(g);  // the tape may be overwritten by the next segment
    }

    // epilogue: parameter gradients from the factored sums
    bool bad = false;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        if (!valid[j]) continue;
        const int q = wb + lane + 32 * j;
        const int gi = sg.veh_begin + q;
        const float v0 = a.v0[gi], b = a.b[gi];
        const float am = kc[j].am, c = kc[j].c, dl = kc[j].delta;
        const float A0 = acc[0 * SLG + q], A1 = acc[1 * SLG + q], A2 = acc[2 * SLG + q];
        const float A3 = acc[3 * SLG + q], A4 = acc[4 * SLG + q], A5 = acc[5 * SLG + q];
        float gr[6];
        gr[0] = am * dl * A4 / v0;                 // v0
        gr[1] = A1;                                // T
        gr[2] = A0;                                // s0
        gr[3] = A3 - A2 * c / (2.0f * am);         // a_max
        gr[4] = -A2 * c / (2.0f * b);              // b
        gr[5] = -am * A5;                          // delta
        for (int p = 0; p < 6; ++p) bad |= !isfinite(gr[p]);
        if (ADAM) {
            const int it = a.iter;
            const int t = it + 1;
            const float lr = a.n_iter > 1 ? a.lr0 + (a.lr1 - a.lr0) * (float)it / (float)(a.n_iter - 1) : a.lr0;
            const float bc1 = 1.0f - powf(0.9f, (float)t), bc2 = 1.0f - powf(0.999f, (float)t);
            float *th[5] = {const_cast<float *>(a.v0), const_cast<float *>(a.T), const_cast<float *>(a.s0),
                            const_cast<float *>(a.am), const_cast<float *>(a.b)};
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                const size_t mi = (size_t)p * a.N_total + gi;
                float m = 0.9f * a.adam_m[mi] + 0.1f * gr[p];
                float vv = 0.999f * a.adam_v[mi] + 0.001f * gr[p] * gr[p];
                a.adam_m[mi] = m;
                a.adam_v[mi] = vv;
                float x = th[p][gi] - lr * (m / bc1) / (sqrtf(vv / bc2) + 1e-8f);
                x = fminf(fmaxf(x, a.lo[p]), a.hi[p]);
                th[p][gi] = x;
            }
        } else {
            if (a.g_v0) a.g_v0[gi] = gr[0];
            if (a.g_T) a.g_T[gi] = gr[1];
            if (a.g_s0) a.g_s0[gi] = gr[2];
            if (a.g_am) a.g_am[gi] = gr[3];
            if (a.g_b) a.g_b[gi] = gr[4];
            if (a.g_delta) a.g_delta[gi] = WD ? gr[5] : 0.0f;
            if (a.g_p_init) a.g_p_init[gi] = lp[j];
            if (a.g_v_init) a.g_v_init[gi] = lv[j];
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, IDM_STATUS_NONFINITE);
    if (!DENSE) {
        const double part = warp_sum_double((double)lsum - (double)lcomp) * (double)sc.inv_nobs;
        if (lane == 0) a.loss_part[(size_t)s_idx * g.G + g.w] = part;
    }
}

template <int VPT, bool DENSE, bool ADAM, bool WD>
__global__ void __launch_bounds__(256, (VPT <= 4 ? 2 : 1))
backward_kernel(SimArgs a)
{
    extern __shared__ float smem[];
    const int G = a.G;
    const int warp = threadIdx.x >> 5;
    float *gbase = smem + (warp / G) * bwd_group_floats(VPT, DENSE, a.C, G);
    float *ctrl = gbase + bwd_group_floats(VPT, DENSE, a.C, G) - grp_ctrl_floats(G);
    Grp g = make_grp(G, ctrl);
    int par = 0;
    for (;;) {
        const int s_idx = grp_next(g, a.work, par);
        if (s_idx >= *a.n_seg) break;
        const Seg sg = a.seg[s_idx];
        const ScenDesc sc = a.scen_tab ? a.scen_tab[sg.scen] : a.scen0;
        const int lb = sg.veh_begin - sc.veh_begin;
        VehConst kc[VPT];
        State st[VPT];
        bool valid[VPT];
        load_vehicles<VPT>(a, sg, g.lane, g.w * 32 * VPT, kc, st, valid);
        if (segment_is_d4<VPT>(kc, valid))
            backward_segment<VPT, DENSE, ADAM, WD, true>(a, sc, sg, s_idx, lb, g, gbase, kc, st, valid);
        else
            backward_segment<VPT, DENSE, ADAM, WD, false>(a, sc, sg, s_idx, lb, g, gbase, kc, st, valid);
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
    FwdFlags f{traj, vtraj, ckpt};
    void *fn = nullptr;
    switch (vpt) {
    case 1: fn = (void *)forward_kernel<1>; break;
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

size_t backward_smem_bytes(int vpt, bool dense_seed, int C, int G, int wpb)
{
    return (size_t)bwd_group_floats(vpt, dense_seed, C, G) * (wpb / G) * sizeof(float);
}

size_t forward_smem_bytes(int vpt, int G, int wpb)
{
    (void)vpt;
    return (size_t)grp_ctrl_floats(G) * (wpb / G) * sizeof(float);
}

// Kernel variants of the adjoint: seeds from dense gradients or from targets,
// fused Adam or gradient output, with or without the delta gradient.
template <int VPT>
static void *backward_fn(bool dense, bool adam, bool wd)
{
    if (dense) return wd ? (void *)backward_kernel<VPT, true, false, true> : (void *)backward_kernel<VPT, true, false, false>;
    if (adam) return (void *)backward_kernel<VPT, false, true, false>;
    return wd ? (void *)backward_kernel<VPT, false, false, true> : (void *)backward_kernel<VPT, false, false, false>;
}

static void *backward_fn_v(int vpt, bool dense, bool adam, bool wd)
{
    switch (vpt) {
    case 1: return backward_fn<1>(dense, adam, wd);
    case 2: return backward_fn<2>(dense, adam, wd);
    case 4: return backward_fn<4>(dense, adam, wd);
    case 8: return backward_fn<8>(dense, adam, wd);
    }
    return nullptr;
}

cudaError_t launch_backward(int vpt, int G, bool dense_seed, bool adam, bool want_delta, const SimArgs &a, int grid,
                            int wpb, cudaStream_t st)
{
    if (dense_seed && adam) return cudaErrorInvalidValue;
    void *fn = backward_fn_v(vpt, dense_seed, adam, want_delta && !adam);
    if (!fn) return cudaErrorInvalidValue;
    size_t smem = backward_smem_bytes(vpt, dense_seed, a.C, G, wpb);
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
        case 1: fn = (void *)forward_kernel<1>; break;
        case 2: fn = (void *)forward_kernel<2>; break;
        case 4: fn = (void *)forward_kernel<4>; break;
        case 8: fn = (void *)forward_kernel<8>; break;
        }
        smem = forward_smem_bytes(vpt, G, wpb);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
        fn = backward_fn_v(vpt, dense, adam, want_delta && !adam);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (!fn) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * wpb, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace idm
