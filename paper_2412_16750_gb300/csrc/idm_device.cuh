// Device arithmetic of the modified IDM step (Eq. 1-3 and the softplus
// bounds of Sec. III-C, arXiv 2412.16750) and of its partial derivatives.
//
// Every rounding in the state update is written with explicit _rn
// intrinsics so that the forward kernel and the recompute inside the adjoint
// kernel produce bit-identical trajectories (no contraction freedom).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/idm.h"

namespace idm {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Softplus pieces: e = exp(-|x|) and sp(x) = max(x,0) + log(1 + e).
struct Soft {
    float e;   // exp(-|x|)
    float sp;  // softplus(x)
};

__device__ __forceinline__ Soft softplus(float x)
{
    Soft s;
    s.e = __expf(-fabsf(x));
    s.sp = __fadd_rn(fmaxf(x, 0.0f), __logf(__fadd_rn(1.0f, s.e)));
    return s;
}

// Logistic sigmoid from the e = exp(-|x|) already computed for softplus.
__device__ __forceinline__ float sigmoid_from(float x, float e)
{
    float d = rcp_approx(__fadd_rn(1.0f, e));
    return x >= 0.0f ? d : __fmul_rn(e, d);
}

// Per-vehicle constants of one call.
struct VehConst {
    float inv_v0;  // 1 / v0
    float T, s0, am, c;  // c = 1 / (2 sqrt(a_max b)), Eq. 1
    float delta;
};

__device__ __forceinline__ VehConst make_const(float v0, float T, float s0, float am, float b, float delta)
{
    VehConst k;
    k.inv_v0 = __frcp_rn(v0);
    k.T = T;
    k.s0 = s0;
    k.am = am;
    k.c = __fmul_rn(0.5f, rsqrtf(__fmul_rn(am, b)));
    k.delta = delta;
    return k;
}

// Ghost slots (padding at the end of a warp segment) and lane heads never
// feed a real vehicle; these constants keep their arithmetic finite.
__device__ __forceinline__ VehConst ghost_const()
{
    VehConst k;
    k.inv_v0 = 1.0f; k.T = 0.0f; k.s0 = 0.0f; k.am = 1.0f; k.c = 0.5f; k.delta = 4.0f;
    return k;
}

// (v / v0)^delta.  D4: every vehicle of the warp has delta == 4 (decided
// once per segment), so the power is two squarings and the step body has no
// per-vehicle branch.
template <bool D4>
__device__ __forceinline__ float pow_delta(float r, float delta)
{
    if (D4) {
        float r2 = __fmul_rn(r, r);
        return __fmul_rn(r2, r2);
    }
    return r > 0.0f ? __powf(r, delta) : 0.0f;
}

// Bounded acceleration a* of one vehicle from its speed v, its raw gap
// (p_h - p - length_h; +inf for a lane head) and its leader's speed vh.
template <bool D4>
__device__ __forceinline__ float accel_star(float v, float gap_raw, float vh, const VehConst &k,
                                            float inv_dt, float a_min)
{
    float gap = gap_raw < IDM_GAP_FLOOR ? IDM_GAP_FLOOR : gap_raw;
    float dv = __fsub_rn(v, vh);                                   // Sec. III-A
    float s_opt = __fmaf_rn(v, __fmaf_rn(dv, k.c, k.T), k.s0);    // Eq. 1
    Soft s1 = softplus(s_opt);                                     // Sec. III-C
    float z = __fmul_rn(s1.sp, rcp_approx(gap));                   // 0 for a head
    float r = __fmul_rn(v, k.inv_v0);
    float rd = pow_delta<D4>(r, k.delta);
    float a = __fmul_rn(k.am, __fsub_rn(__fsub_rn(1.0f, rd), __fmul_rn(z, z)));  // Eq. 2
    float lbv = -__fmul_rn(v, inv_dt);
    float a_lb = lbv > a_min ? lbv : a_min;                        // Sec. III-C
    Soft s2 = softplus(__fsub_rn(a, a_lb));
    return __fadd_rn(a_lb, s2.sp);
}

// Vehicle state: absolute position as an unevaluated float pair (ph + pl,
// ph the float32 position, pl the accumulated rounding error), speed, and
// raw gap to the leader.
struct State {
    float ph, pl, v, gap;
};

// Explicit Euler step (Eq. 3): positions use the old speeds, so the gap
// moves by dt (vh - v); the position is accumulated with TwoSum plus the
// exact rounding error of dt*v, so ph + pl stays within ~1e-10 relative of
// the exact sum.
__device__ __forceinline__ void euler(State &s, float a_star, float vh, float dt)
{
    float d = __fmul_rn(dt, s.v);
    float d_err = __fmaf_rn(dt, s.v, -d);
    float t = __fadd_rn(s.ph, d);
    float bb = __fsub_rn(t, s.ph);
    float err = __fadd_rn(__fsub_rn(s.ph, __fsub_rn(t, bb)), __fsub_rn(d, bb));
    s.ph = t;
    s.pl = __fadd_rn(s.pl, __fadd_rn(err, d_err));
    s.gap = __fmaf_rn(dt, __fsub_rn(vh, s.v), s.gap);
    s.v = __fmaf_rn(dt, a_star, s.v);
}

// ph + pl - y.  ph - y is exact when the target is within a factor two of the
// position (Sterbenz) and otherwise rounds at the scale of the residual, so the
// residual keeps the pair's precision even kilometres from the origin.
__device__ __forceinline__ float residual(const State &s, float y)
{
    return __fadd_rn(__fsub_rn(s.ph, y), s.pl);
}

__device__ __forceinline__ float position(const State &s) { return __fadd_rn(s.ph, s.pl); }

// Leader values in the strided slot mapping: slot q = lane + 32 j of the
// warp; the leader of slot q is q-1 (thread lane-1, same j; for lane 0,
// thread 31 of j-1).  The warp's first slot receives lead_in (the previous
// warp's last slot, or 0 at the start of a segment, which is a lane head).
template <int VPT>
__device__ __forceinline__ void leader_vals(const float (&x)[VPT], float (&out)[VPT], int lane, float lead_in)
{
    float rot[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) rot[j] = __shfl_sync(FULL, x[j], (lane + 31) & 31);
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        float prev = j > 0 ? rot[j - 1] : lead_in;
        out[j] = lane == 0 ? prev : rot[j];
    }
}

// Follower values: slot q receives from slot q+1 (thread lane+1, same j;
// for lane 31, thread 0 of j+1).  The warp's last slot receives fin (the
// next warp's first slot, or 0 at the end of a segment).
template <int VPT>
__device__ __forceinline__ void follower_vals(const float (&x)[VPT], float (&out)[VPT], int lane, float fin)
{
    float rot[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) rot[j] = __shfl_sync(FULL, x[j], (lane + 1) & 31);
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        float nxt = j + 1 < VPT ? rot[j + 1] : fin;
        out[j] = lane == 31 ? nxt : rot[j];
    }
}

}  // namespace idm

namespace idm {

// Coefficients of one reverse step for one vehicle (the adjoint of
// accel_star and euler), independent of the incoming adjoint.  With
// sigma2 = d a*/d a, sigma1 = d s*/d s_opt, S = d a/d s*, G = d a/d gap:
//   Ap  = d a*/d p         = -sigma2 G     (the leader's d a*/d p_h is -Ap)
//   Av  = d a*/d v         (own speed, incl. the a_lb branch)
//   Avh = d a*/d v_leader  = w0 (-c v),  w0 = sigma2 S sigma1
// and the parameter-gradient factors (per-vehicle constants multiply the
// sums once at the end): w0, w0 v, w0 v dv, sigma2 (1 - r^delta - z^2),
// sigma2 r^delta, sigma2 r^delta ln r.  The reverse step multiplies all of
// them by mu = dt * (adjoint of the step-(k+1) speed), so this part can be
// evaluated ahead of the dependent adjoint chain.
struct AdjJac {
    float Ap, Av, Avh;
    float w0, w0v, w0vdv, fa, frd, frdl;
};

template <bool WANT_DELTA, bool D4>
__device__ __forceinline__ AdjJac adjoint_jac(float v, float gap_raw, float vh, const VehConst &k, float inv_dt,
                                              float a_min)
{
    AdjJac J;
    const bool floored = gap_raw < IDM_GAP_FLOOR;
    const float gap = floored ? IDM_GAP_FLOOR : gap_raw;
    const float dv = __fsub_rn(v, vh);
    const float s_opt = __fmaf_rn(v, __fmaf_rn(dv, k.c, k.T), k.s0);
    const Soft s1 = softplus(s_opt);
    const float sig1 = sigmoid_from(s_opt, s1.e);
    const float inv_gap = rcp_approx(gap);
    const float z = __fmul_rn(s1.sp, inv_gap);
    const float r = __fmul_rn(v, k.inv_v0);
    float rd, rdm1;
    if (D4) {
        const float r2 = __fmul_rn(r, r);
        rd = __fmul_rn(r2, r2);
        rdm1 = __fmul_rn(r2, r);
    } else {
        rd = r > 0.0f ? __powf(r, k.delta) : 0.0f;
        rdm1 = r > 0.0f ? __powf(r, k.delta - 1.0f) : (k.delta > 1.0f ? 0.0f : (k.delta == 1.0f ? 1.0f : INFINITY));
    }
    const float free_and_int = __fsub_rn(__fsub_rn(1.0f, rd), __fmul_rn(z, z));
    const float a = __fmul_rn(k.am, free_and_int);
    const float lbv = -__fmul_rn(v, inv_dt);
    const bool beta = lbv > a_min;
    const float a_lb = beta ? lbv : a_min;
    const float x2 = __fsub_rn(a, a_lb);
    const float e2 = __expf(-fabsf(x2));
    const float d2 = rcp_approx(__fadd_rn(1.0f, e2));
    const float ed2 = __fmul_rn(e2, d2);
    const float sig2 = x2 >= 0.0f ? d2 : ed2;        // sigma(x2)
    const float one_m_sig2 = x2 >= 0.0f ? ed2 : d2;  // sigma(-x2)

    const float S = -2.0f * k.am * z * inv_gap;  // d a / d s*
    const float G = floored ? 0.0f : -S * z;     // d a / d gap = 2 a_max z^2 / gap
    const float w0 = sig2 * S * sig1;
    const float dfree_dv = -k.am * (D4 ? 4.0f : k.delta) * rdm1 * k.inv_v0;
    J.Ap = -sig2 * G;
    J.Av = sig2 * dfree_dv + w0 * (k.T + k.c * (v + dv)) - (beta ? one_m_sig2 * inv_dt : 0.0f);
    J.Avh = -w0 * k.c * v;
    J.w0 = w0;
    J.w0v = w0 * v;
    J.w0vdv = J.w0v * dv;
    J.fa = sig2 * free_and_int;
    J.frd = sig2 * rd;
    J.frdl = (WANT_DELTA && rd > 0.0f) ? J.frd * __logf(r) : 0.0f;
    return J;
}

}  // namespace idm
