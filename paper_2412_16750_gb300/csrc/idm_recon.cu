// Single-trajectory filtering and reconstruction mode of arXiv 2412.16750
// (Sec. IV-A; optimisation settings and metrics of Sec. V-B): one ego
// vehicle per trajectory, simulated with the modified IDM (Eq. 1-3, bounds of
// Sec. III-C) behind a virtual leader whose gap dp_k and speed difference
// dv_k at every step are free variables.
//
// One thread per trajectory, one warp per block.  Every per-step array is
// time-major, so at step k a warp touches one 128-byte row segment per array.
// Rows are staged into shared memory with cp.async, S - 1 chunks of U steps
// ahead of use, so the forward's serial chain (the speed of step k+1 needs the
// whole model evaluation of step k) does not wait on memory: rows of the
// caller's arrays with 16-byte copies shared by the warp (then __syncwarp), or
// with 4-byte copies of each lane's own column when the row stride is not a
// multiple of four; the tape and the Adam moments with one 16-byte copy per
// lane of its own data.
//
// Forward: integrates the state and, while its serial chain (one model
// evaluation per step) leaves most issue slots idle, evaluates the adjoint's
// partials of every step (they depend only on the step's speed, dp_k and dv_k)
// and writes them with the loss seed of step k+1 as the tape; or writes the
// requested P/V/A, or the metric sums.  Adjoint: walks the tape backwards; its
// only serial chain is the adjoint recursion (two FMAs per step), the rest
// (gradient sums, Adam on dp_k and dv_k) is independent across steps.  The fit
// runs every iteration of its trajectory inside one launch (trajectories are
// independent), with Adam for dp_k and dv_k fused into the adjoint and Adam
// for the parameters at its end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "../../include/idm.h"
#include "../../include/idm_recon.h"
#include "idm_ctx.h"
#include "idm_device.cuh"

namespace idm {
namespace rec {

constexpr int U = 8;                       // steps per staged chunk
constexpr int S = 3;                       // chunks in flight
// A stage holds, per step and lane: three float4 slots (forward: the rows of
// dp, dv, the observed position and the observation code, overlaid as four
// float rows; adjoint: the two tape halves and the Adam moments or the delta
// factor) and two float rows (adjoint: dp, dv).
constexpr int STAGE = (3 * 4 + 2) * U * 32;   // floats per chunk
constexpr int SMEM = (int)sizeof(float) * S * STAGE;

enum Mode { FWD_OUT = 0, LOSS_GRAD = 1, FIT = 2, METRICS = 3 };

struct Args {
    int N, k_max, ld, n_obs;
    const int32_t *K;
    const float *p_init, *v_init;
    float dt, inv_dt, a_min;
    float *th[6];                    // v0, T, s0, a_max, b, delta (the fit updates the first five)
    float *dp, *dv;
    const float *oyy;                // [k_max][ld]: first observed position of step k+1
    const int32_t *oyc;              // [k_max][ld]: 8 j + min(count, 7) of that observation, -1 = none
    const int32_t *multi;            // [N]: 1 if some step of the trajectory has several observations
    int wide_ok;                     // dp, dv and the observation rows allow 16-byte row copies (ld % 4 == 0, aligned)
    const int32_t *obs_off, *obs_k;
    const float *obs_p;
    float4 *tape_a, *tape_b;         // tape [k_max][ld]: (Av, Adp, Adv, w0n), (w0n v, fa, frd, seed of step k+1)
    float *tape_d;                   // [k_max][ld]: frdl (delta gradient only)
    float4 *mom;                     // [k_max][ld]: Adam moments (m_dp, v_dp, m_dv, v_dv)
    float *thm, *thv;                // Adam moments of the parameters, [5][N]
    float *P, *V, *A;
    double *loss;                    // loss_out (LOSS_GRAD) or loss_hist (FIT)
    float *g6[6];
    float *g_dp, *g_dv, *g_p0, *g_v0;
    double *acc;                     // METRICS: pos sum, n_pos, sum |a|, sum a^2, n_a, n_imp
    unsigned *status;
    int n_iter;
    float lr0, lr1;
    float lo[5], hi[5];
};

// Per-trajectory constants of Eq. 1-2.
struct Par {
    float v0, inv_v0, T, s0, am, b, c, delta;
};

__device__ __forceinline__ Par make_par(float v0, float T, float s0, float am, float b, float delta)
{
    Par q;
    q.v0 = v0;
    q.inv_v0 = 1.0f / v0;
    q.T = T;
    q.s0 = s0;
    q.am = am;
    q.b = b;
    q.c = c_of(am, b);   // 1 / (2 sqrt(a_max b)), Eq. 1
    q.delta = delta;
    return q;
}

__device__ __forceinline__ float softplus1(float x, float &e)
{
    e = ex2_approx(fabsf(x) * -LOG2E);
    return fmaf(lg2_approx(1.0f + e), LN2, fmaxf(x, 0.0f));
}

// sigma(x) and sigma(-x) from e = exp(-|x|).
__device__ __forceinline__ void sigmoid1(float x, float e, float &sig, float &sig_neg)
{
    const float d = rcp_approx(1.0f + e);
    const float ed = e * d;
    sig = x >= 0.0f ? d : ed;
    sig_neg = x >= 0.0f ? ed : d;
}

template <bool D4>
__device__ __forceinline__ float pow_delta1(float r, float delta)
{
    if (D4) {
        const float r2 = r * r;
        return r2 * r2;
    }
    return r > 0.0f ? __powf(r, delta) : 0.0f;
}

// Partials of a* at (v, dp, dv) for the reverse step; with sigma2 = d a*/d a,
// sigma1 = d s*/d s_opt, Sn = 2 a_max z / gap = -d a/d s* and w0n = sigma2
// Sn sigma1:
//   Av  = d a*/d v  = -(sigma2 a_max delta r^(delta-1) / v0 + w0n (T + c dv)
//                       + [a_lb = -v/dt] (1 - sigma2) / dt)
//   Adp = d a*/d dp = sigma2 Sn z  (0 below the gap floor)
//   Adv = d a*/d dv = -w0n c v
// and the parameter factors w0n, w0n v, w0n v dv, sigma2 (1 - r^delta -
// z^2), sigma2 r^delta, sigma2 r^delta ln r.
struct Jac1 {
    float Av, Adp, Adv, w0n, fa, frd, frdl;
};

template <bool D4, bool WD>
__device__ __forceinline__ Jac1 jac1(float v, float dp, float dv, const Par &q, float inv_dt, float a_min)
{
    Jac1 J;
    const bool floored = dp < IDM_GAP_FLOOR;
    const float ig = rcp_approx(fmaxf(dp, IDM_GAP_FLOOR));
    const float u = fmaf(dv, q.c, q.T);                                 // d s_opt / d v (dv is free)
    const float s_opt = fmaf(v, u, q.s0);
    float e1, sig1, sig1n;
    const float sp1 = softplus1(s_opt, e1);
    sigmoid1(s_opt, e1, sig1, sig1n);
    const float z = sp1 * ig;
    const float r = v * q.inv_v0;
    float rd, rdm1;
    if (D4) {
        const float r2 = r * r;
        rd = r2 * r2;
        rdm1 = r2 * r;
    } else {
        rd = pow_delta1<false>(r, q.delta);
        rdm1 = r > 0.0f ? __powf(r, q.delta - 1.0f) : (q.delta > 1.0f ? 0.0f : (q.delta == 1.0f ? 1.0f : INFINITY));
    }
    const float fa0 = (1.0f - rd) - z * z;
    const float a = q.am * fa0;
    const float lbv = v * -inv_dt;
    const bool beta = lbv > a_min;
    const float a_lb = fmaxf(lbv, a_min);
    const float x2 = a - a_lb;
    const float e2 = ex2_approx(fabsf(x2) * -LOG2E);
    float sig2, one_m_sig2;
    sigmoid1(x2, e2, sig2, one_m_sig2);
    const float Sn = (q.am + q.am) * z * ig;
    const float G = floored ? 0.0f : Sn * z;
    const float w0n = sig2 * Sn * sig1;
    const float qv = q.am * (D4 ? 4.0f : q.delta) * rdm1 * q.inv_v0;
    const float bt = beta ? one_m_sig2 * inv_dt : 0.0f;
    J.Av = -fmaf(sig2, qv, fmaf(w0n, u, bt));
    J.Adp = sig2 * G;
    J.Adv = -(w0n * q.c) * v;
    J.w0n = w0n;
    J.fa = sig2 * fa0;
    J.frd = sig2 * rd;
    if (WD) {
        const float t = J.frd * (lg2_approx(r) * LN2);
        J.frdl = r > 0.0f && rd > 0.0f ? t : 0.0f;   // the r -> 0+ limit (also for a speed rounded to <= 0 or a denormal)
    } else {
        J.frdl = 0.0f;
    }
    return J;
}

// The speed update of one explicit Euler step (Eq. 3) with a* of Eq. 1-2
// and Sec. III-C, arranged so that the serial chain v -> v' has a single FMA
// after each softplus: with sp(x) = max(x, 0) + ln 2 log2(1 + exp(-|x|)),
//   z  = s* / gap = fma(ln2 / gap, log2(1 + e1), max(s_opt, 0) / gap),
//   v' = v + dt a* = fma(dt ln2, log2(1 + e2), v + dt max(a, a_lb)),
// everything else (1 - r^delta, a_lb, the max terms) runs beside the chain.
// a_star receives a* = max(a, a_lb) + ln 2 log2(1 + e2).
template <bool D4>
__device__ __forceinline__ float speed_step(float v, float gap_inv, float u, const Par &q, float dt, float inv_dt,
                                            float a_min, float &a_star)
{
    const float s_opt = fmaf(v, u, q.s0);                                       // Eq. 1
    const float e1 = ex2_approx(fabsf(s_opt) * -LOG2E);
    const float z = fmaf(LN2 * gap_inv, lg2_approx(1.0f + e1), fmaxf(s_opt, 0.0f) * gap_inv);
    const float rd = pow_delta1<D4>(v * q.inv_v0, q.delta);
    const float a = fmaf(-q.am, z * z, q.am * (1.0f - rd));                    // Eq. 2
    const float a_lb = fmaxf(v * -inv_dt, a_min);                               // Sec. III-C
    const float l2 = lg2_approx(1.0f + ex2_approx(fabsf(a - a_lb) * -LOG2E));
    const float m = fmaxf(a, a_lb);
    a_star = fmaf(LN2, l2, m);
    return fmaf(dt * LN2, l2, fmaf(dt, m, v));
}

// The position update of the Euler step (Eq. 3, old speed) on an FP32 pair:
// TwoSum plus the exact rounding error of dt v.
__device__ __forceinline__ void euler_pos(float &ph, float &pl, float v, float dt)
{
    const float d = dt * v;
    const float en = fmaf(-dt, v, d);
    const float t = ph + d;
    const float bb = t - ph;
    const float err = (ph - (t - bb)) + (d - bb);
    ph = t;
    pl = pl + (err - en);
}

__device__ __forceinline__ void kahan(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ float sgn(float r) { return (float)((r > 0.0f) - (r < 0.0f)); }

__device__ __forceinline__ void cp4(float *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}

// Slot of (chunk c, step u, lane) in float4 region r (0..2) of the chunk's
// stage, and the row-major float rows of the stage: row (r, u) holds the 32
// columns of array r at step u.  Float region 0 overlays float4 region 0
// (forward: dp, dv, observed position, observation code); float region 1
// lies after the three float4 regions (adjoint: dp, dv).
__device__ __forceinline__ float4 *slot4(float *sm, int c, int r, int u, int lane)
{
    return reinterpret_cast<float4 *>(sm + (size_t)(c % S) * STAGE) + ((size_t)r * U + u) * 32 + lane;
}
__device__ __forceinline__ float *rows_fwd(float *sm, int c) { return sm + (size_t)(c % S) * STAGE; }
__device__ __forceinline__ float *rows_adj(float *sm, int c) { return sm + (size_t)(c % S) * STAGE + 3 * 4 * U * 32; }

// Stage NR time-major rows per step (arrays src[0..NR), steps k(u), u < U)
// of the warp's 32 columns starting at column i0 into rows[(r U + u) 32 +
// col].  wide: 16-byte copies shared by the warp (eight per 128-byte row
// segment; needs ld % 4 == 0, 16-byte aligned arrays and i0 + 32 <= ld);
// otherwise each lane copies its own column.  Rows with k(u) < 0, or k(u) >=
// k_lim_lane (the lane's horizon, own-column copies) or k_lim (the warp's
// largest horizon, wide copies) are skipped.
template <int NR, typename KOF>
__device__ __forceinline__ void stage_rows(float *rows, const float *const (&src)[NR], size_t ld, int i0, int lane,
                                           bool wide, int k_lim, int k_lim_lane, KOF k_of)
{
    if (wide) {
#pragma unroll
        for (int m = 0; m < NR * U * 8 / 32; ++m) {
            const int q = lane + 32 * m;               // segment: 8 per row
            const int row = q >> 3, seg = q & 7;
            const int r = row / U, u = row % U;
            const int k = k_of(u);
            if (k >= 0 && k < k_lim) cp16(rows + (size_t)row * 32 + seg * 4, src[r] + (size_t)k * ld + i0 + seg * 4);
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k_of(u);
            if (k >= 0 && k < k_lim_lane) {
#pragma unroll
                for (int r = 0; r < NR; ++r) cp4(rows + (size_t)(r * U + u) * 32 + lane, src[r] + (size_t)k * ld + i0 + lane);
            }
        }
    }
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

struct MetricAcc {
    double pos = 0.0, s1 = 0.0, s2 = 0.0;
    int n_pos = 0, n_a = 0, imp = 0;
};

// Forward over the Ki steps of trajectory i (Kw = the warp's largest Ki).
// Returns the loss sum (LOSS_GRAD, FIT), which also write the tape.
template <int MODE, bool D4, bool WD>
__device__ __forceinline__ double fwd_phase(const Args &a, const Par &q, int i, bool act, int Ki, int Kw, float *sm,
                                            int lane, MetricAcc &ma, float len_inv)
{
    constexpr bool TAPE = MODE == LOSS_GRAD || MODE == FIT;
    const int nch = (Kw + U - 1) / U;
    const size_t ld = (size_t)a.ld;
    const int i0 = i - lane;
    const bool wide = a.wide_ok && i0 + 32 <= a.ld;   // warp-uniform
    auto issue = [&](int c) {
        if (c < nch) {
            auto k_of = [c](int u) { return c * U + u; };
            if (MODE == FWD_OUT) {
                const float *const src[2] = {a.dp, a.dv};
                stage_rows<2>(rows_fwd(sm, c), src, ld, i0, lane, wide, Kw, Ki, k_of);
            } else {
                const float *const src[4] = {a.dp, a.dv, a.oyy, reinterpret_cast<const float *>(a.oyc)};
                stage_rows<4>(rows_fwd(sm, c), src, ld, i0, lane, wide, Kw, Ki, k_of);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int c = 0; c < S - 1; ++c) issue(c);

    const float dt = a.dt, inv_dt = a.inv_dt, a_min = a.a_min;
    float v = act ? a.v_init[i] : 0.0f;
    float ph = act ? a.p_init[i] : 0.0f, pl = 0.0f;
    float Ls = 0.0f, Lcomp = 0.0f;   // loss: per-thread Kahan sum of the chunk sums
    const int j_end =
        (MODE == LOSS_GRAD || MODE == FIT || MODE == METRICS) && Ki > 0 ? min(a.obs_off[i + 1], a.n_obs) : 0;
    // One chunk of U steps.  MULTI: some step of the chunk has several
    // observations (rare); without it the chunk is one branch-free block, so
    // the compiler can overlap a step's partials, position and observation
    // work with the next step's serial chain.
    auto chunk = [&](int c, auto multi_tag) {
        constexpr bool MULTI = decltype(multi_tag)::value;
        float Lc = 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = c * U + u;
            const bool valid = k < Ki;
            const float *rw = rows_fwd(sm, c) + u * 32 + lane;
            const float dp = rw[0], dv = rw[U * 32];
            const float y_obs = MODE != FWD_OUT ? rw[2 * U * 32] : 0.0f;
            const float code_f = MODE != FWD_OUT ? rw[3 * U * 32] : 0.0f;
            const float gap_inv = rcp_approx(fmaxf(dp, IDM_GAP_FLOOR));
            const float uu = fmaf(dv, q.c, q.T);
            float as;
            const float vn = speed_step<D4>(v, gap_inv, uu, q, dt, inv_dt, a_min, as);
            // the adjoint's partials at this step, beside the serial chain
            Jac1 J;
            if (TAPE) J = jac1<D4, WD>(v, dp, dv, q, inv_dt, a_min);
            float phn = ph, pln = pl;
            euler_pos(phn, pln, v, dt);
            const float v_k = v;
            v = valid ? vn : v;
            ph = valid ? phn : ph;
            pl = valid ? pln : pl;
            const size_t o = (size_t)k * ld + i;
            if (MODE == FWD_OUT) {
                if (valid) {
                    if (a.P) a.P[o + ld] = ph + pl;
                    if (a.V) a.V[o + ld] = v;
                    if (a.A) a.A[o] = as;
                }
            } else {
                // observations at step k+1: the staged first one, then (MULTI)
                // any further ones from the CSR
                const int code = valid ? __float_as_int(code_f) : -1;
                const bool has = code >= 0;
                float r = (ph - y_obs) + pl;
                float seed = has ? sgn(r) : 0.0f;
                Lc += has ? fabsf(r) : 0.0f;
                if (MODE == METRICS && has) {
                    ma.pos += fabs((double)r) * len_inv;
                    ++ma.n_pos;
                }
                if (MULTI && has && (code & 7) > 1) {
                    const int cnt = code & 7, j0 = code >> 3;
                    for (int j = j0 + 1; j < j_end; ++j) {
                        if (cnt < 7 ? j >= j0 + cnt : a.obs_k[j] != k + 1) break;
                        r = (ph - a.obs_p[j]) + pl;
                        seed += sgn(r);
                        Lc += fabsf(r);
                        if (MODE == METRICS) {
                            ma.pos += fabs((double)r) * len_inv;
                            ++ma.n_pos;
                        }
                    }
                }
                if (TAPE && valid) {
                    a.tape_a[o] = make_float4(J.Av, J.Adp, J.Adv, J.w0n);
                    a.tape_b[o] = make_float4(J.w0n * v_k, J.fa, J.frd, seed);
                    if (WD) a.tape_d[o] = J.frdl;
                }
                if (MODE == METRICS && valid) {
                    const double aa = fabs((double)as);
                    ma.s1 += aa;
                    ma.s2 += aa * aa;
                    ++ma.n_a;
                    ma.imp |= aa > 10.0;
                }
            }
        }
        return Lc;
    };
    // several observations at one step: decided once per warp
    const bool multi = MODE != FWD_OUT && __any_sync(FULL, act && Ki > 0 && a.multi[i] != 0);
    for (int c = 0; c < nch; ++c) {
        issue(c + S - 1);
        cp_wait<S - 1>();
        if (wide) __syncwarp();   // rows copied by other lanes
        // Branch-free over the chunk: a lane past its horizon computes on
        // stale staged values and keeps its state (selects, predicated stores).
        const float Lc = multi ? chunk(c, std::true_type{}) : chunk(c, std::false_type{});
        kahan(Ls, Lcomp, Lc);
    }
    const double L = (double)Ls - (double)Lcomp;
    cp_wait<0>();
    if (MODE == FWD_OUT && act) {
        // rows beyond the trajectory's horizon hold its final state
        const float pf = ph + pl;
        for (int k = Ki; k < a.k_max; ++k) {
            const size_t o = (size_t)k * ld + i;
            if (a.P) a.P[o + ld] = pf;
            if (a.V) a.V[o + ld] = v;
            if (a.A) a.A[o] = 0.0f;
        }
    }
    if (!isfinite(v) || !isfinite(ph + pl)) atomicOr(a.status, IDM_STATUS_NONFINITE);
    return L;
}

// Adam update of one unconstrained variable (moments m, w), with a1 = lr /
// (1 - beta1^t) and isb2 = 1 / sqrt(1 - beta2^t).
__device__ __forceinline__ float adam1(float x, float g, float &m, float &w, float a1, float isb2)
{
    m = fmaf(0.9f, m, 0.1f * g);
    w = fmaf(0.999f, w, 0.001f * g * g);
    float sw;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sw) : "f"(w));
    return fmaf(-a1 * m, rcp_approx(fmaf(sw, isb2, 1e-8f)), x);
}

// Reverse pass over the Ki steps of trajectory i on the tape of the forward.
// lambda_p and lambda_v are the adjoints of the position and speed; the seed
// of step k+1 enters lambda_p before step k is reversed.  Returns the
// parameter sums A[6] (gradients assembled by the caller), lambda_p(0) and
// lambda_v(0).
template <int MODE, bool WD>
__device__ __forceinline__ void adj_phase(const Args &a, int i, int Ki, int Kw, float *sm, int lane, float a1,
                                          float isb2, float (&Acc)[6], float &lp_out, float &lv_out)
{
    const int nch = (Kw + U - 1) / U;
    const size_t ld = (size_t)a.ld;
    const int i0 = i - lane;
    const bool wide = a.wide_ok && i0 + 32 <= a.ld;   // warp-uniform
    auto issue = [&](int c) {
        if (c < nch) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = Kw - 1 - (c * U + u);
                if (k >= 0 && k < Ki) {
                    const size_t o = (size_t)k * ld + i;
                    cp16(slot4(sm, c, 0, u, lane), a.tape_a + o);
                    cp16(slot4(sm, c, 1, u, lane), a.tape_b + o);
                    if (MODE == FIT) cp16(slot4(sm, c, 2, u, lane), a.mom + o);
                    if (WD) cp4(reinterpret_cast<float *>(slot4(sm, c, 2, u, lane)), a.tape_d + o);
                }
            }
            const float *const src[2] = {a.dp, a.dv};
            stage_rows<2>(rows_adj(sm, c), src, ld, i0, lane, wide, Kw, Ki, [c, Kw](int u) { return Kw - 1 - (c * U + u); });
        }
        cp_commit();
    };
#pragma unroll
    for (int c = 0; c < S - 1; ++c) issue(c);

    const float dt = a.dt;
    float lp = 0.0f, lv = 0.0f;
#pragma unroll
    for (int r = 0; r < 6; ++r) Acc[r] = 0.0f;
    for (int c = 0; c < nch; ++c) {
        issue(c + S - 1);
        cp_wait<S - 1>();
        if (wide) __syncwarp();   // rows copied by other lanes
        // Branch-free: a lane past its horizon reads stale staged values and
        // keeps its state (selects, predicated stores).
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = Kw - 1 - (c * U + u);
            const bool valid = k >= 0 && k < Ki;
            const float4 ta = *slot4(sm, c, 0, u, lane);     // Av, Adp, Adv, w0n
            const float4 tb = *slot4(sm, c, 1, u, lane);     // w0n v, fa, frd, seed of step k+1
            const float2 pv = make_float2(rows_adj(sm, c)[u * 32 + lane], rows_adj(sm, c)[(U + u) * 32 + lane]);   // dp, dv
            const float lpn = lp + tb.w;                     // lambda_p(k+1)
            const float mu = dt * lv;                        // dt lambda_v(k+1)
            const float lvn = fmaf(mu, ta.x, fmaf(dt, lpn, lv));   // lambda_v(k)
            const float gdp = mu * ta.y, gdv = mu * ta.z;
            Acc[0] = valid ? fmaf(mu, ta.w, Acc[0]) : Acc[0];
            Acc[1] = valid ? fmaf(mu, tb.x, Acc[1]) : Acc[1];
            Acc[2] = valid ? fmaf(mu, tb.x * pv.y, Acc[2]) : Acc[2];
            Acc[3] = valid ? fmaf(mu, tb.y, Acc[3]) : Acc[3];
            Acc[4] = valid ? fmaf(mu, tb.z, Acc[4]) : Acc[4];
            if (WD) Acc[5] = valid ? fmaf(mu, slot4(sm, c, 2, u, lane)->x, Acc[5]) : Acc[5];
            lp = valid ? lpn : lp;
            lv = valid ? lvn : lv;
            const size_t o = (size_t)k * ld + i;
            if (MODE == LOSS_GRAD) {
                if (valid && a.g_dp) a.g_dp[o] = gdp;
                if (valid && a.g_dv) a.g_dv[o] = gdv;
            } else if (MODE == FIT) {
                float4 m = *slot4(sm, c, 2, u, lane);
                const float dpn = adam1(pv.x, gdp, m.x, m.y, a1, isb2);
                const float dvn = adam1(pv.y, gdv, m.z, m.w, a1, isb2);
                if (valid) {
                    a.dp[o] = dpn;
                    a.dv[o] = dvn;
                    a.mom[o] = m;
                }
            }
        }
    }
    cp_wait<0>();
    lp_out = lp;
    lv_out = lv;
}

// Gradients of the six parameters from the sums of adj_phase.
__device__ __forceinline__ void param_grads(const Par &q, const float (&A)[6], float (&gr)[6])
{
    gr[0] = q.am * q.delta * A[4] * q.inv_v0;          // v0
    gr[1] = -A[1];                                     // T
    gr[2] = -A[0];                                     // s0
    gr[3] = A[3] + A[2] * q.c / (2.0f * q.am);         // a_max (through c)
    gr[4] = A[2] * q.c / (2.0f * q.b);                 // b (through c)
    gr[5] = -q.am * A[5];                              // delta
}

__device__ __forceinline__ Par load_par(const Args &a, int i)
{
    return make_par(a.th[0][i], a.th[1][i], a.th[2][i], a.th[3][i], a.th[4][i], a.th[5][i]);
}

// Horizon of trajectory i, 0 for an idle lane or an out-of-range value.
__device__ __forceinline__ int horizon(const Args &a, int i, bool act)
{
    if (!act) return 0;
    const int Ki = a.K[i];
    if (Ki < 0 || Ki > a.k_max) {
        atomicOr(a.status, IDM_STATUS_BAD_OBS);
        return 0;
    }
    return Ki;
}

template <int MODE, bool D4>
__device__ __forceinline__ void run_single(const Args &a, int i, bool act, int Ki, int Kw, float *sm, int lane)
{
    MetricAcc ma;
    float len_inv = 0.0f;
    if (MODE == METRICS && act) {
        const int j0 = min(max(a.obs_off[i], 0), a.n_obs), j1 = min(max(a.obs_off[i + 1], j0), a.n_obs);
        const float len = j1 > j0 ? fabsf(a.obs_p[j1 - 1] - a.obs_p[j0]) : 0.0f;
        len_inv = len > 0.0f ? 1.0f / len : 0.0f;
        if (len > 0.0f) {
            // observations at step 0 compare with the initial position
            const float p0 = a.p_init[i];
            for (int j = j0; j < j1 && a.obs_k[j] == 0; ++j) {
                ma.pos += fabs((double)(p0 - a.obs_p[j])) * len_inv;
                ++ma.n_pos;
            }
        }
    }
    const Par q = act ? load_par(a, i) : make_par(1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 4.0f);
    const bool wd = MODE == LOSS_GRAD && a.g6[5] != nullptr;
    const double L = wd ? fwd_phase<MODE, D4, true>(a, q, i, act, Ki, Kw, sm, lane, ma, len_inv)
                        : fwd_phase<MODE, D4, false>(a, q, i, act, Ki, Kw, sm, lane, ma, len_inv);
    if (MODE == METRICS) {
        if (len_inv == 0.0f) {
            ma.pos = 0.0;
            ma.n_pos = 0;
        }
        const double v[6] = {ma.pos, (double)ma.n_pos, ma.s1, ma.s2, (double)ma.n_a, (double)(act && ma.imp)};
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const double s = warp_sum(v[r]);
            if (lane == 0) atomicAdd(a.acc + r, s);
        }
        return;
    }
    if (MODE == LOSS_GRAD) {
        const double s = warp_sum(L);
        if (lane == 0 && a.loss) atomicAdd(a.loss, s);
        __threadfence_block();  // the tape written above is read back by this thread's copies
        float A[6], lp, lv, gr[6];
        if (wd)
            adj_phase<LOSS_GRAD, true>(a, i, Ki, Kw, sm, lane, 0.0f, 0.0f, A, lp, lv);
        else
            adj_phase<LOSS_GRAD, false>(a, i, Ki, Kw, sm, lane, 0.0f, 0.0f, A, lp, lv);
        if (!act) return;
        param_grads(q, A, gr);
        bool bad = !isfinite(lp) || !isfinite(lv);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            bad |= !isfinite(gr[r]);
            if (a.g6[r]) a.g6[r][i] = (r == 5 && !wd) ? 0.0f : gr[r];
        }
        if (a.g_p0) a.g_p0[i] = lp;   // observations at step 0 are not in the loss
        if (a.g_v0) a.g_v0[i] = lv;
        const size_t ld = (size_t)a.ld;
        for (int k = Ki; k < a.k_max; ++k) {
            if (a.g_dp) a.g_dp[(size_t)k * ld + i] = 0.0f;
            if (a.g_dv) a.g_dv[(size_t)k * ld + i] = 0.0f;
        }
        if (bad) atomicOr(a.status, IDM_STATUS_NONFINITE);
    }
}

template <int MODE>
__global__ void __launch_bounds__(32) recon_kernel(Args a)
{
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const bool act = i < a.N;
    const int Ki = horizon(a, i, act);
    const int Kw = __reduce_max_sync(FULL, (unsigned)Ki);
    const bool d4 = __all_sync(FULL, !act || a.th[5][i] == 4.0f);
    if (d4)
        run_single<MODE, true>(a, i, act, Ki, Kw, sm, lane);
    else
        run_single<MODE, false>(a, i, act, Ki, Kw, sm, lane);
}

// The whole fit of every trajectory of the warp: n_iter x {forward with the
// loss and seeds, adjoint with Adam on dp and dv, Adam on the parameters}.
template <bool D4>
__device__ __forceinline__ void fit_warp(const Args &a, int i, bool act, int Ki, int Kw, float *sm, int lane)
{
    Par q = act ? load_par(a, i) : make_par(1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 4.0f);
    float th[5] = {q.v0, q.T, q.s0, q.am, q.b};
    bool bad = false;
    MetricAcc ma;
    for (int it = 0; it < a.n_iter; ++it) {
        const double L = fwd_phase<FIT, D4, false>(a, q, i, act, Ki, Kw, sm, lane, ma, 0.0f);
        const double s = warp_sum(L);
        if (lane == 0 && a.loss) atomicAdd(a.loss + it, s);
        __threadfence_block();  // tape and updated dp, dv are read back by this thread's copies
        const int t = it + 1;
        const float lr = a.n_iter > 1 ? a.lr0 + (a.lr1 - a.lr0) * (float)it / (float)(a.n_iter - 1) : a.lr0;
        const float bc1 = 1.0f - __powf(0.9f, (float)t), bc2 = 1.0f - __powf(0.999f, (float)t);
        const float a1 = lr / bc1, isb2 = 1.0f / sqrtf(bc2);
        float A[6], lp, lv, gr[6];
        adj_phase<FIT, false>(a, i, Ki, Kw, sm, lane, a1, isb2, A, lp, lv);
        __threadfence_block();
        if (act) {
            param_grads(q, A, gr);
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                bad |= !isfinite(gr[r]);
                const size_t mi = (size_t)r * a.N + i;
                const float m = 0.9f * a.thm[mi] + 0.1f * gr[r];
                const float vv = 0.999f * a.thv[mi] + 0.001f * gr[r] * gr[r];
                a.thm[mi] = m;
                a.thv[mi] = vv;
                const float x = th[r] - lr * (m / bc1) / (sqrtf(vv / bc2) + 1e-8f);
                th[r] = fminf(fmaxf(x, a.lo[r]), a.hi[r]);
            }
            q = make_par(th[0], th[1], th[2], th[3], th[4], q.delta);
        }
    }
    if (act) {
#pragma unroll
        for (int r = 0; r < 5; ++r) a.th[r][i] = th[r];
        if (bad) atomicOr(a.status, IDM_STATUS_NONFINITE);
    }
}

__global__ void __launch_bounds__(32) recon_fit_kernel(Args a)
{
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const bool act = i < a.N;
    const int Ki = horizon(a, i, act);
    const int Kw = __reduce_max_sync(FULL, (unsigned)Ki);
    const bool d4 = __all_sync(FULL, !act || a.th[5][i] == 4.0f);
    if (d4)
        fit_warp<true>(a, i, act, Ki, Kw, sm, lane);
    else
        fit_warp<false>(a, i, act, Ki, Kw, sm, lane);
}

// ---- preparation --------------------------------------------------------------

// Largest i with off[i] <= j (off non-decreasing, off[0] = 0 <= j).
__device__ __forceinline__ int traj_of(const int32_t *off, int N, int j)
{
    int lo = 0, hi = N - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Nearest step of every observation, in double precision: floor(t / dt + 1/2).
__global__ void obs_steps_kernel(int N, int n_obs, const int32_t *off, const float *t, double dt, int32_t *obs_k,
                                 unsigned *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_obs) return;
    const int i = traj_of(off, N, j);
    const double tj = (double)t[j];
    const double kd = floor(tj / dt + 0.5);
    const bool bad_t = !(tj >= 0.0) || !(kd < 2147483647.0) || (j > max(off[i], 0) && t[j] < t[j - 1]);
    obs_k[j] = bad_t ? 0 : (int32_t)kd;
    if (bad_t) atomicOr(status, IDM_STATUS_BAD_OBS);
}

// Horizon and initial state of every trajectory (rules of Sec. V-B).
__global__ void traj_init_kernel(int N, int n_obs, const int32_t *off, const float *t, const float *p,
                                 const int32_t *obs_k, int32_t *K, float *p0, float *v0, int *k_max, unsigned *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j0 = off[i], j1 = off[i + 1];
    if ((i == 0 && j0 != 0) || j0 < 0 || j0 > j1 || j1 > n_obs || (i == N - 1 && j1 != n_obs)) {
        atomicOr(status, IDM_STATUS_BAD_OBS);
        K[i] = 0;
        p0[i] = 0.0f;
        v0[i] = 0.0f;
        return;
    }
    const int n = j1 - j0;
    const int Ki = n > 0 ? obs_k[j1 - 1] : 0;
    K[i] = Ki;
    p0[i] = n > 0 ? p[j0] : 0.0f;
    const float d01 = n > 1 ? t[j0 + 1] - t[j0] : 0.0f;
    v0[i] = d01 > 0.0f ? fmaxf((p[j0 + 1] - p[j0]) / d01, 0.0f) : 0.0f;
    atomicMax(k_max, Ki);
}

// Time-major observation index: row k of trajectory i names the first
// observation at step k+1 (its position and 8 j + min(count, 7)).
__global__ void obs_rows_kernel(int N, int n_obs, int k_max, int ld, const int32_t *off, const int32_t *obs_k,
                                const float *p, float *oyy, int32_t *oyc, int32_t *multi, unsigned *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_obs) return;
    const int i = traj_of(off, N, j);
    const int j0 = max(off[i], 0), j1 = min(off[i + 1], n_obs);
    if (j < j0 || j >= j1) return;  // malformed CSR (reported by idm_recon_prepare)
    const int s = obs_k[j];
    if (s < 0 || s > k_max || (j > j0 && obs_k[j - 1] > s)) {
        atomicOr(status, IDM_STATUS_BAD_OBS);
        return;
    }
    if (s == 0 || (j > j0 && obs_k[j - 1] == s)) return;
    int cnt = 1;
    while (cnt < 7 && j + cnt < j1 && obs_k[j + cnt] == s) ++cnt;
    const size_t o = (size_t)(s - 1) * ld + i;
    oyy[o] = p[j];
    oyc[o] = j * 8 + cnt;
    if (cnt > 1) multi[i] = 1;
}

__global__ void metrics_final_kernel(const double *acc, int n_traj, double *out)
{
    const double n_pos = acc[1], n_a = acc[4];
    const double mean = n_a > 0.0 ? acc[2] / n_a : 0.0;
    out[0] = n_pos > 0.0 ? acc[0] / n_pos : 0.0;
    out[1] = mean;
    out[2] = n_a > 0.0 ? sqrt(fmax(acc[3] / n_a - mean * mean, 0.0)) : 0.0;
    out[3] = n_traj > 0 ? acc[5] / n_traj : 0.0;
}

}  // namespace rec
}  // namespace idm

// ---- C ABI ---------------------------------------------------------------------

using namespace idm;
using namespace idm::abi;

namespace {

int check_rec(idm_ctx *c, const idm_recon_t *r, bool need_obs)
{
    if (!r) return fail(c, IDM_ERR_ARG, "rec is NULL");
    if (r->n_traj < 0) return fail(c, IDM_ERR_ARG, "n_traj must be >= 0");
    if (r->k_max < 1) return fail(c, IDM_ERR_ARG, "k_max must be >= 1 (got %d)", r->k_max);
    if (r->ld < r->n_traj || r->ld < 1) return fail(c, IDM_ERR_ARG, "ld must be >= max(n_traj, 1)");
    if ((size_t)r->k_max * (size_t)r->ld > ((size_t)1 << 40)) return fail(c, IDM_ERR_ARG, "k_max * ld too large");
    if (!(r->dt > 0.0f) || !std::isfinite(r->dt)) return fail(c, IDM_ERR_ARG, "dt must be finite and > 0");
    if (!(r->a_min < 0.0f) || !std::isfinite(r->a_min)) return fail(c, IDM_ERR_ARG, "a_min must be finite and < 0");
    if (r->n_traj > 0 && (!r->K || !r->p_init || !r->v_init))
        return fail(c, IDM_ERR_ARG, "K, p_init and v_init must be given");
    if (need_obs) {
        if (r->n_obs < 0 || r->n_obs >= ((int64_t)1 << 28))
            return fail(c, IDM_ERR_ARG, "n_obs must lie in [0, 2^28)");
        if (r->n_traj > 0 && !r->obs_off) return fail(c, IDM_ERR_ARG, "obs_off is NULL");
        if (r->n_obs > 0 && (!r->obs_k || !r->obs_p)) return fail(c, IDM_ERR_ARG, "obs_k and obs_p must be given");
    }
    return IDM_OK;
}

int check_par(idm_ctx *c, const idm_params_t *p)
{
    if (!p) return fail(c, IDM_ERR_ARG, "params is NULL");
    if (!p->v0 || !p->T || !p->s0 || !p->a_max || !p->b || !p->delta)
        return fail(c, IDM_ERR_ARG, "a parameter array is NULL");
    return IDM_OK;
}

rec::Args base_args(idm_ctx *c, const idm_recon_t *r, const idm_params_t *p, const float *dp, const float *dv)
{
    rec::Args a;
    memset(&a, 0, sizeof a);
    a.N = r->n_traj;
    a.n_obs = (int)r->n_obs;
    a.k_max = r->k_max;
    a.ld = r->ld;
    a.K = r->K;
    a.p_init = r->p_init;
    a.v_init = r->v_init;
    a.dt = r->dt;
    a.inv_dt = 1.0f / r->dt;
    a.a_min = r->a_min;
    float *th[6] = {p->v0, p->T, p->s0, p->a_max, p->b, p->delta};
    for (int q = 0; q < 6; ++q) a.th[q] = th[q];
    a.dp = const_cast<float *>(dp);
    a.dv = const_cast<float *>(dv);
    a.obs_off = r->obs_off;
    a.obs_k = r->obs_k;
    a.obs_p = r->obs_p;
    a.status = (unsigned *)c->status.p;
    // 16-byte row copies need 16-byte aligned rows of every staged array (the
    // observation rows share ld and are the context's own allocations)
    a.wide_ok = (r->ld % 4 == 0) && ((uintptr_t)dp % 16 == 0) && ((uintptr_t)dv % 16 == 0);
    return a;
}

// Build the time-major observation index of rec into the context.
int build_obs_rows(idm_ctx *c, const idm_recon_t *r, rec::Args &a, cudaStream_t st)
{
    const size_t rows = (size_t)r->k_max * r->ld;
    int rc;
    if ((rc = ensure(c, c->rec_oyy, sizeof(float) * rows, "observation rows"))) return rc;
    if ((rc = ensure(c, c->rec_oyc, sizeof(int32_t) * rows, "observation codes"))) return rc;
    if ((rc = ensure(c, c->rec_multi, sizeof(int32_t) * std::max<size_t>(r->ld, 1), "observation flags"))) return rc;
    IDM_CK(cudaMemsetAsync(c->rec_oyc.p, 0xff, sizeof(int32_t) * rows, st));
    IDM_CK(cudaMemsetAsync(c->rec_multi.p, 0, sizeof(int32_t) * std::max<size_t>(r->ld, 1), st));
    if (r->n_obs > 0 && r->n_traj > 0) {
        const int n = (int)r->n_obs;
        rec::obs_rows_kernel<<<(n + 255) / 256, 256, 0, st>>>(r->n_traj, n, r->k_max, r->ld, r->obs_off, r->obs_k,
                                                              r->obs_p, (float *)c->rec_oyy.p,
                                                              (int32_t *)c->rec_oyc.p, (int32_t *)c->rec_multi.p,
                                                              a.status);
        IDM_CK(cudaGetLastError());
    }
    a.oyy = (const float *)c->rec_oyy.p;
    a.oyc = (const int32_t *)c->rec_oyc.p;
    a.multi = (const int32_t *)c->rec_multi.p;
    return IDM_OK;
}

int ensure_tape(idm_ctx *c, const idm_recon_t *r, rec::Args &a)
{
    const size_t rows = (size_t)r->k_max * r->ld;
    int rc;
    if ((rc = ensure(c, c->rec_tape, sizeof(float) * 9 * rows, "adjoint tape"))) return rc;
    a.tape_a = (float4 *)c->rec_tape.p;
    a.tape_b = a.tape_a + rows;
    a.tape_d = (float *)(a.tape_b + rows);
    return IDM_OK;
}

template <typename K>
int launch_rec(idm_ctx *c, K kern, const rec::Args &a, cudaStream_t st)
{
    if (a.N == 0) return IDM_OK;
    IDM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, rec::SMEM));
    kern<<<(a.N + 31) / 32, 32, rec::SMEM, st>>>(a);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}

}  // namespace

extern "C" int idm_recon_prepare(idm_ctx_t *c, int32_t N, int64_t n_obs, const int32_t *obs_off, const float *obs_t,
                                 const float *obs_p, float dt, int32_t *obs_k, int32_t *K, float *p_init,
                                 float *v_init, int32_t *k_max_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (N < 0) return fail(c, IDM_ERR_ARG, "N must be >= 0");
    if (n_obs < 0 || n_obs >= ((int64_t)1 << 28)) return fail(c, IDM_ERR_ARG, "n_obs must lie in [0, 2^28)");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, IDM_ERR_ARG, "dt must be finite and > 0");
    if (N > 0 && (!obs_off || !K || !p_init || !v_init)) return fail(c, IDM_ERR_ARG, "a per-trajectory array is NULL");
    if (n_obs > 0 && (!obs_t || !obs_p || !obs_k)) return fail(c, IDM_ERR_ARG, "an observation array is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = ensure_status(c))) return rc;
    if ((rc = ensure(c, c->rec_kmax, sizeof(int) * 4, "k_max scalar"))) return rc;
    IDM_CK(cudaMemsetAsync(c->rec_kmax.p, 0, sizeof(int), st));
    unsigned *status = (unsigned *)c->status.p;
    if (n_obs > 0 && N > 0) {
        const int n = (int)n_obs;
        rec::obs_steps_kernel<<<(n + 255) / 256, 256, 0, st>>>(N, n, obs_off, obs_t, (double)dt, obs_k, status);
        IDM_CK(cudaGetLastError());
    }
    if (N > 0) {
        rec::traj_init_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, (int)n_obs, obs_off, obs_t, obs_p, obs_k, K, p_init,
                                                               v_init, (int *)c->rec_kmax.p, status);
        IDM_CK(cudaGetLastError());
    }
    if (k_max_out) {
        IDM_CK(cudaMemcpyAsync(k_max_out, c->rec_kmax.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        IDM_CK(cudaStreamSynchronize(st));
    }
    return IDM_OK;
}

extern "C" int idm_recon_forward(idm_ctx_t *c, const idm_recon_t *r, const idm_params_t *params, const float *dp,
                                 const float *dv, float *P, float *V, float *A, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_rec(c, r, false)) || (rc = check_par(c, params))) return rc;
    if (r->n_traj > 0 && (!dp || !dv)) return fail(c, IDM_ERR_ARG, "dp and dv must be given");
    if ((rc = ensure_status(c))) return rc;
    rec::Args a = base_args(c, r, params, dp, dv);
    a.P = P;
    a.V = V;
    a.A = A;
    cudaStream_t st = (cudaStream_t)stream;
    // row 0 of P and V: the initial state
    if (r->n_traj > 0 && P)
        IDM_CK(cudaMemcpyAsync(P, r->p_init, sizeof(float) * r->n_traj, cudaMemcpyDeviceToDevice, st));
    if (r->n_traj > 0 && V)
        IDM_CK(cudaMemcpyAsync(V, r->v_init, sizeof(float) * r->n_traj, cudaMemcpyDeviceToDevice, st));
    return launch_rec(c, rec::recon_kernel<rec::FWD_OUT>, a, st);
}

extern "C" int idm_recon_loss_grad(idm_ctx_t *c, const idm_recon_t *r, const idm_params_t *params, const float *dp,
                                   const float *dv, double *loss_out, idm_params_t *grad, float *g_dp, float *g_dv,
                                   float *g_p_init, float *g_v_init, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_rec(c, r, true)) || (rc = check_par(c, params))) return rc;
    if (r->n_traj > 0 && (!dp || !dv)) return fail(c, IDM_ERR_ARG, "dp and dv must be given");
    if ((rc = ensure_status(c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rec::Args a = base_args(c, r, params, dp, dv);
    if ((rc = build_obs_rows(c, r, a, st)) || (rc = ensure_tape(c, r, a))) return rc;
    a.loss = loss_out;
    if (grad) {
        float *g[6] = {grad->v0, grad->T, grad->s0, grad->a_max, grad->b, grad->delta};
        for (int q = 0; q < 6; ++q) a.g6[q] = g[q];
    }
    a.g_dp = g_dp;
    a.g_dv = g_dv;
    a.g_p0 = g_p_init;
    a.g_v0 = g_v_init;
    if (loss_out) IDM_CK(cudaMemsetAsync(loss_out, 0, sizeof(double), st));
    return launch_rec(c, rec::recon_kernel<rec::LOSS_GRAD>, a, st);
}

extern "C" int idm_recon_fit(idm_ctx_t *c, const idm_recon_t *r, idm_params_t *params, float *dp, float *dv,
                             int32_t n_iter, float lr0, float lr1, const float *box_lo, const float *box_hi,
                             double *loss_hist, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_rec(c, r, true)) || (rc = check_par(c, params))) return rc;
    if (r->n_traj > 0 && (!dp || !dv)) return fail(c, IDM_ERR_ARG, "dp and dv must be given");
    if (n_iter < 1 || n_iter > 100000) return fail(c, IDM_ERR_ARG, "n_iter must lie in [1, 100000]");
    if (!box_lo || !box_hi) return fail(c, IDM_ERR_ARG, "box_lo and box_hi must be given");
    if (!std::isfinite(lr0) || !std::isfinite(lr1)) return fail(c, IDM_ERR_ARG, "learning rates must be finite");
    for (int q = 0; q < 5; ++q)
        if (!(box_lo[q] <= box_hi[q])) return fail(c, IDM_ERR_ARG, "box_lo[%d] > box_hi[%d]", q, q);
    if ((rc = ensure_status(c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rec::Args a = base_args(c, r, params, dp, dv);
    if ((rc = build_obs_rows(c, r, a, st)) || (rc = ensure_tape(c, r, a))) return rc;
    const size_t rows = (size_t)r->k_max * r->ld, N = (size_t)r->n_traj;
    if ((rc = ensure(c, c->rec_mom, sizeof(float) * 4 * rows, "Adam moments of dp, dv"))) return rc;
    if ((rc = ensure(c, c->rec_thm, sizeof(float) * 10 * std::max<size_t>(N, 1), "Adam moments of the parameters")))
        return rc;
    IDM_CK(cudaMemsetAsync(c->rec_mom.p, 0, sizeof(float) * 4 * rows, st));
    IDM_CK(cudaMemsetAsync(c->rec_thm.p, 0, sizeof(float) * 10 * std::max<size_t>(N, 1), st));
    a.mom = (float4 *)c->rec_mom.p;
    a.thm = (float *)c->rec_thm.p;
    a.thv = a.thm + 5 * N;
    a.loss = loss_hist;
    a.n_iter = n_iter;
    a.lr0 = lr0;
    a.lr1 = lr1;
    for (int q = 0; q < 5; ++q) {
        a.lo[q] = box_lo[q];
        a.hi[q] = box_hi[q];
    }
    if (loss_hist) IDM_CK(cudaMemsetAsync(loss_hist, 0, sizeof(double) * n_iter, st));
    return launch_rec(c, rec::recon_fit_kernel, a, st);
}

extern "C" int idm_recon_metrics(idm_ctx_t *c, const idm_recon_t *r, const idm_params_t *params, const float *dp,
                                 const float *dv, double *out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_rec(c, r, true)) || (rc = check_par(c, params))) return rc;
    if (r->n_traj > 0 && (!dp || !dv)) return fail(c, IDM_ERR_ARG, "dp and dv must be given");
    if (!out) return fail(c, IDM_ERR_ARG, "out is NULL");
    if ((rc = ensure_status(c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rec::Args a = base_args(c, r, params, dp, dv);
    if ((rc = build_obs_rows(c, r, a, st))) return rc;
    if ((rc = ensure(c, c->rec_acc, sizeof(double) * 8, "metric sums"))) return rc;
    a.acc = (double *)c->rec_acc.p;
    IDM_CK(cudaMemsetAsync(a.acc, 0, sizeof(double) * 8, st));
    if ((rc = launch_rec(c, rec::recon_kernel<rec::METRICS>, a, st))) return rc;
    rec::metrics_final_kernel<<<1, 1, 0, st>>>(a.acc, r->n_traj, out);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}
