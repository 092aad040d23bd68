// Device arithmetic of the modified IDM step (Eq. 1-3 and the softplus
// bounds of Sec. III-C, arXiv 2412.16750) and of its partial derivatives.
//
// Two vehicles are processed per instruction: every value is a float2 pair
// and the FP32 arithmetic uses the packed sm_100+ forms (FADD2 / FMUL2 /
// FFMA2) with round-to-nearest, so each component is rounded exactly as a
// scalar op would round it.  Special functions (exp2, log2, reciprocal) are
// per component on the SFU.  Every rounding in the state update is explicit,
// so the forward kernel and the recompute inside the adjoint kernel produce
// bit-identical trajectories.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/idm.h"

namespace idm {

constexpr unsigned FULL = 0xffffffffu;
constexpr float LOG2E = 1.44269504088896340736f;
constexpr float LN2 = 0.69314718055994530942f;

// ---- special-function unit (PTX approximate ops) ---------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- packed pairs ------------------------------------------------------------
using f2 = float2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b per component, rounded to nearest (the packed subtract instruction,
// no separate negation).
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ f2 ex2(f2 x) { return make_float2(ex2_approx(x.x), ex2_approx(x.y)); }
__device__ __forceinline__ f2 lg2(f2 x) { return make_float2(lg2_approx(x.x), lg2_approx(x.y)); }
__device__ __forceinline__ f2 rcp2(f2 x) { return make_float2(rcp_approx(x.x), rcp_approx(x.y)); }
__device__ __forceinline__ f2 vmax(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 vabs(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

// Softplus pieces: e = exp(-|x|) = 2^(-|x| log2 e) and
// sp(x) = max(x, 0) + ln(1 + e) = log2(1 + e) * ln 2 + max(x, 0).
struct Soft2 {
    f2 e;
    f2 sp;
};

__device__ __forceinline__ Soft2 softplus2(f2 x)
{
    Soft2 s;
    s.e = make_float2(ex2_approx(fabsf(x.x) * -LOG2E), ex2_approx(fabsf(x.y) * -LOG2E));
    s.sp = fma2(lg2(add2(F2(1.0f), s.e)), F2(LN2), vmax(x, F2(0.0f)));
    return s;
}

// Logistic sigmoid from the e = exp(-|x|) of softplus2: sigma(x) and
// sigma(-x) = 1 - sigma(x) without cancellation.
__device__ __forceinline__ void sigmoid2(f2 x, f2 e, f2 &sig, f2 &sig_neg)
{
    const f2 d = rcp2(add2(F2(1.0f), e));
    const f2 ed = mul2(e, d);
    sig = make_float2(x.x >= 0.0f ? d.x : ed.x, x.y >= 0.0f ? d.y : ed.y);
    sig_neg = make_float2(x.x >= 0.0f ? ed.x : d.x, x.y >= 0.0f ? ed.y : d.y);
}

// Per-vehicle constants of one call, for a pair of vehicles.
struct VehConst2 {
    f2 inv_v0;          // 1 / v0
    f2 T, s0, am, c;    // c = 1 / (2 sqrt(a_max b)), Eq. 1
    f2 delta;
};

// c = 1 / (2 sqrt(a_max b)), correctly rounded steps (a per-vehicle constant:
// an approximate square root would perturb every step of the vehicle the
// same way).
__device__ __forceinline__ float c_of(float am, float b) { return __fdiv_rn(0.5f, __fsqrt_rn(__fmul_rn(am, b))); }


// (v / v0)^delta.  D4: every vehicle of the warp has delta == 4 (decided once
// per segment), so the power is two squarings.
template <bool D4>
__device__ __forceinline__ f2 pow_delta2(f2 r, f2 delta)
{
    if (D4) {
        const f2 r2 = mul2(r, r);
        return mul2(r2, r2);
    }
    return make_float2(r.x > 0.0f ? __powf(r.x, delta.x) : 0.0f, r.y > 0.0f ? __powf(r.y, delta.y) : 0.0f);
}

// max(gap, floor): one min/max op per element (a non-finite gap only arises
// from a non-finite state, which the status word reports).
__device__ __forceinline__ f2 floor_gap(f2 g) { return vmax(g, F2(IDM_GAP_FLOOR)); }

// a_lb = max(-v/dt, a_min) with the strict-inequality tie rule (Sec. III-C).
__device__ __forceinline__ f2 lower_bound(f2 lbv, float a_min, bool &bx, bool &by)
{
    bx = lbv.x > a_min;
    by = lbv.y > a_min;
    return vmax(lbv, F2(a_min));  // equal values give a_min either way
}

// Bounded acceleration a* of two vehicles from their speeds v, raw gaps
// (p_h - p - length_h; +inf for a lane head) and leaders' speeds vh.
template <bool D4>
__device__ __forceinline__ f2 accel_star2(f2 v, f2 gap_raw, f2 vh, const VehConst2 &k, float inv_dt, float a_min)
{
    const f2 gap = floor_gap(gap_raw);
    const f2 dv = sub2(v, vh);                                  // Sec. III-A
    const f2 s_opt = fma2(v, fma2(dv, k.c, k.T), k.s0);         // Eq. 1
    const Soft2 s1 = softplus2(s_opt);                          // Sec. III-C
    const f2 z = mul2(s1.sp, rcp2(gap));                        // 0 for a head
    const f2 r = mul2(v, k.inv_v0);
    const f2 rd = pow_delta2<D4>(r, k.delta);
    const f2 a = mul2(k.am, sub2(sub2(F2(1.0f), rd), mul2(z, z)));  // Eq. 2
    bool bx, by;
    const f2 a_lb = lower_bound(mul2(v, F2(-inv_dt)), a_min, bx, by);  // Sec. III-C
    const Soft2 s2 = softplus2(sub2(a, a_lb));
    return add2(a_lb, s2.sp);
}

// Vehicle-pair state: absolute position as an unevaluated float pair
// (ph + pl, ph the float32 position, pl the accumulated rounding error),
// speed as a Kahan-compensated sum (v the float32 running sum of the
// increments dt a*, vc minus its lost low part: the speed is v - vc), and
// raw gap to the leader.  The step's model is evaluated at v, which stays
// within an ulp or so of the speed.  Without the compensation the rounding
// of v at every step (half an ulp, ~1e-6 m/s at 20 m/s) accumulates into a
// position drift of ~1 cm over 2,000 steps; the gap moves with the
// compensated speeds of both vehicles (vh - v + vc - vch), so that it stays
// the difference of the positions.
struct State2 {
    f2 ph, pl, v, gap, vc;
};

// Explicit Euler step (Eq. 3): positions use the old speeds, so the gap moves
// by dt (vh - v).  The position is accumulated with Dekker's Fast2Sum plus
// the exact rounding error of dt*v (en = d - dt*v, so the error is -en) and
// the speed's compensation (-dt vc), keeping ph + pl within ~1e-10 relative
// of the sum of dt times the speeds.  Fast2Sum's error term is exact while
// |ph| >= |d| (a step is at most a few metres); in the one or two steps in
// which a vehicle passes within |d| of position 0 it is off by at most half
// an ulp of the sum (~5e-7 m), three operations fewer per step than TwoSum.
// The speed takes dt a* by Kahan's compensated summation.
__device__ __forceinline__ void euler2(State2 &s, f2 a_star, f2 vh, f2 vch, float dt)
{
    const f2 d = mul2(F2(dt), s.v);
    const f2 en = fma2(F2(-dt), s.v, d);
    const f2 t = add2(s.ph, d);
    const f2 err = sub2(d, sub2(t, s.ph));
    s.ph = t;
    s.pl = fma2(F2(-dt), s.vc, add2(s.pl, sub2(err, en)));
    s.gap = fma2(F2(dt), add2(sub2(vh, s.v), sub2(s.vc, vch)), s.gap);
    const f2 y = sub2(mul2(F2(dt), a_star), s.vc);
    const f2 tv = add2(s.v, y);
    s.vc = sub2(sub2(tv, s.v), y);
    s.v = tv;
}

// The speed of the state: the running sum minus its compensation.
__device__ __forceinline__ f2 speed2(const State2 &s) { return sub2(s.v, s.vc); }

// ph + pl - y.  ph - y is exact when the target is within a factor two of the
// position (Sterbenz) and otherwise rounds at the scale of the residual.
__device__ __forceinline__ f2 residual2(const State2 &s, f2 y) { return add2(sub2(s.ph, y), s.pl); }

__device__ __forceinline__ f2 position2(const State2 &s) { return add2(s.ph, s.pl); }

// ---- neighbours in the warp's slot mapping -----------------------------------
// Pair p of lane l holds the consecutive slots 64p + 2l (.x) and 64p + 2l + 1
// (.y).  The leader of .y is the same thread's .x; the leader of .x is lane
// l-1's .y (for lane 0: lane 31's .y of pair p-1, or lead_in for p = 0, the
// previous warp's last slot or 0 at a segment start).
template <int NP>
__device__ __forceinline__ void leader_vals2(const f2 (&x)[NP], f2 (&out)[NP], int lane, float lead_in)
{
    float ry[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) ry[p] = __shfl_sync(FULL, x[p].y, (lane + 31) & 31);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float prev = p > 0 ? ry[p - 1] : lead_in;
        out[p].x = lane == 0 ? prev : ry[p];
        out[p].y = x[p].x;
    }
}

// Follower values: the follower of .x is the same thread's .y; the follower
// of .y is lane l+1's .x (for lane 31: lane 0's .x of pair p+1, or fin for the
// warp's last slot).
template <int NP>
__device__ __forceinline__ void follower_vals2(const f2 (&x)[NP], f2 (&out)[NP], int lane, float fin)
{
    float rx[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) rx[p] = __shfl_sync(FULL, x[p].x, (lane + 1) & 31);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float nxt = p + 1 < NP ? rx[p + 1] : fin;
        out[p].x = x[p].y;
        out[p].y = lane == 31 ? nxt : rx[p];
    }
}

// ---- adjoint coefficients ------------------------------------------------------
// Coefficients of one reverse step for a vehicle pair (the adjoint of
// accel_star2 and euler2), independent of the incoming adjoint.  With
// sigma2 = d a*/d a, sigma1 = d s*/d s_opt, Sn = -d a/d s* = 2 a_max z / gap
// and G = d a/d gap = Sn z (0 below the gap floor):
//   Aph = d a*/d p_leader  =  sigma2 G  (own d a*/d p is -Aph)
//   Av  = d a*/d v         (own speed, incl. the a_lb branch)
//   Avh = d a*/d v_leader  =  w0n c v,  w0n = sigma2 Sn sigma1
// and the parameter-gradient factors, all sign-positive forms (per-vehicle
// constants and signs are applied once at the end): w0n, w0n v, w0n v dv,
// sigma2 (1 - r^delta - z^2), sigma2 r^delta, sigma2 r^delta ln r.  The
// reverse step multiplies all of them by mu = dt * (adjoint of the
// step-(k+1) speed).
struct AdjJac2 {
    f2 Aph, Av, Avh;
    f2 w0n, w0nv, w0nvdv, fa, frd, frdl;
};

// qc: with D4, the per-vehicle constant 4 a_max / v0 of the free-road term's
// speed derivative (ignored otherwise).
template <bool WANT_DELTA, bool D4>
__device__ __forceinline__ AdjJac2 adjoint_jac2(f2 v, f2 gap_raw, f2 vh, const VehConst2 &k, float inv_dt,
                                                float a_min, f2 qc = F2(0.0f))
{
    AdjJac2 J;
    const bool fx = gap_raw.x < IDM_GAP_FLOOR, fy = gap_raw.y < IDM_GAP_FLOOR;
    const f2 gap = floor_gap(gap_raw);
    const f2 dv = sub2(v, vh);
    const f2 s_opt = fma2(v, fma2(dv, k.c, k.T), k.s0);
    const Soft2 s1 = softplus2(s_opt);
    // sigma(s_opt) = exp(s_opt - sp(s_opt)): the exponent is <= 0 and carries
    // no cancellation of note (sp(x) - x = sp(-x)); no selects on the sign
    const f2 sig1 = ex2(mul2(sub2(s_opt, s1.sp), F2(LOG2E)));
    const f2 inv_gap = rcp2(gap);
    const f2 z = mul2(s1.sp, inv_gap);
    const f2 r = mul2(v, k.inv_v0);
    f2 rd, rdm1;
    if (D4) {
        const f2 r2 = mul2(r, r);
        rd = mul2(r2, r2);
        rdm1 = mul2(r2, r);
    } else {
        rd = pow_delta2<false>(r, k.delta);
        rdm1 = make_float2(
            r.x > 0.0f ? __powf(r.x, k.delta.x - 1.0f) : (k.delta.x > 1.0f ? 0.0f : (k.delta.x == 1.0f ? 1.0f : INFINITY)),
            r.y > 0.0f ? __powf(r.y, k.delta.y - 1.0f) : (k.delta.y > 1.0f ? 0.0f : (k.delta.y == 1.0f ? 1.0f : INFINITY)));
    }
    const f2 free_and_int = sub2(sub2(F2(1.0f), rd), mul2(z, z));
    const f2 a = mul2(k.am, free_and_int);
    bool bx, by;
    const f2 a_lb = lower_bound(mul2(v, F2(-inv_dt)), a_min, bx, by);
    const f2 x2 = sub2(a, a_lb);
    const f2 e2 = make_float2(ex2_approx(fabsf(x2.x) * -LOG2E), ex2_approx(fabsf(x2.y) * -LOG2E));
    f2 sig2, one_m_sig2;
    sigmoid2(x2, e2, sig2, one_m_sig2);

    const f2 Sn = mul2(mul2(add2(k.am, k.am), z), inv_gap);   // -d a / d s* = 2 a_max z / gap
    f2 G = mul2(Sn, z);                                          // d a / d gap = 2 a_max z^2 / gap
    G.x = fx ? 0.0f : G.x;
    G.y = fy ? 0.0f : G.y;
    const f2 w0n = mul2(mul2(sig2, Sn), sig1);
    const f2 q = D4 ? mul2(qc, rdm1) : mul2(mul2(k.am, k.delta), mul2(rdm1, k.inv_v0));  // -d(free term)/dv
    f2 beta_term = mul2(one_m_sig2, F2(inv_dt));
    beta_term.x = bx ? beta_term.x : 0.0f;
    beta_term.y = by ? beta_term.y : 0.0f;
    J.Aph = mul2(sig2, G);
    const f2 u = fma2(k.c, add2(v, dv), k.T);                    // d s_opt / d v
    J.Av = mul2(fma2(sig2, q, fma2(w0n, u, beta_term)), F2(-1.0f));
    J.Avh = mul2(mul2(w0n, k.c), v);
    J.w0n = w0n;
    J.w0nv = mul2(w0n, v);
    J.w0nvdv = mul2(J.w0nv, dv);
    J.fa = mul2(sig2, free_and_int);
    J.frd = mul2(sig2, rd);
    if (WANT_DELTA) {
        const f2 lnr = mul2(lg2(r), F2(LN2));
        const f2 t = mul2(J.frd, lnr);
        // r^delta ln r -> 0 as r -> 0+.  Near rest the a_lb = -v/dt branch
        // leaves v + dt a* within rounding of 0: a speed a few ulps below 0,
        // or a denormal that the flush-to-zero logarithm reads as 0, also
        // take the limit (r^delta has underflowed to 0 there)
        J.frdl = make_float2(r.x > 0.0f && rd.x > 0.0f ? t.x : 0.0f, r.y > 0.0f && rd.y > 0.0f ? t.y : 0.0f);
    } else {
        J.frdl = F2(0.0f);
    }
    return J;
}

}  // namespace idm
