// Multi-threaded CPU backend (include/idm_cpu.h): the modified IDM of arXiv
// 2412.16750 (Eq. 1-3, bounds of Sec. III-C), the squared-error loss, its
// reverse-time adjoint and Adam, with OpenMP threads over lanes.
//
// Per lane the forward keeps the tape of every step (speed and raw gap of
// every vehicle), so the adjoint needs no recompute; the fit runs all
// iterations of one lane before the next, keeping the lane's tape, state and
// Adam moments in the core's cache.  The state is (position as an FP32 pair,
// speed, raw gap integrated as gap' = gap + dt (v_leader - v)), the same
// state the CUDA kernels integrate.
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <new>
#include <vector>

#include "../../include/idm.h"
#include "../../include/idm_cpu.h"

namespace {

struct Veh {
    float v0, T, s0, am, b, delta, inv_v0, c;
};

inline float sp(float x, float &e)
{
    e = expf(-fabsf(x));
    return fmaxf(x, 0.0f) + log1pf(e);
}

inline float sigm(float x, float e) { return x >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e); }

inline float powd(float r, float delta)
{
    if (delta == 4.0f) {
        const float r2 = r * r;
        return r2 * r2;
    }
    return r > 0.0f ? powf(r, delta) : 0.0f;
}

// a* of Eq. 1-2 with the Sec. III-C bounds; gap is the raw gap (+inf for a
// lane head), vh the leader's speed.
inline float accel(float v, float gap, float vh, const Veh &q, float inv_dt, float a_min)
{
    const float g = fmaxf(gap, IDM_GAP_FLOOR);
    const float s_opt = q.s0 + v * q.T + v * (v - vh) * q.c;
    float e1;
    const float z = sp(s_opt, e1) / g;
    const float a = q.am * (1.0f - powd(v * q.inv_v0, q.delta) - z * z);
    const float lbv = -v * inv_dt;
    const float a_lb = lbv > a_min ? lbv : a_min;
    float e2;
    return a_lb + sp(a - a_lb, e2);
}

// Partials of a* at (v, gap, vh): own speed, leader speed, gap, and the
// parameter factors (v0, T, s0, a_max, b, delta).
struct Part {
    float dv, dvh, dgap, dth[6];
};

inline Part partials(float v, float gap, float vh, const Veh &q, float inv_dt, float a_min)
{
    Part o;
    const bool floored = gap < IDM_GAP_FLOOR;
    const float g = fmaxf(gap, IDM_GAP_FLOOR);
    const float ig = std::isinf(g) ? 0.0f : 1.0f / g;
    const float dvel = v - vh;
    const float s_opt = q.s0 + v * q.T + v * dvel * q.c;
    float e1;
    const float ss = sp(s_opt, e1);
    const float sig1 = sigm(s_opt, e1);
    const float z = ss * ig;
    const float r = v * q.inv_v0;
    const float rd = powd(r, q.delta);
    float rdm1;
    if (q.delta == 4.0f)
        rdm1 = r * r * r;
    else
        rdm1 = r > 0.0f ? powf(r, q.delta - 1.0f) : (q.delta > 1.0f ? 0.0f : (q.delta == 1.0f ? 1.0f : INFINITY));
    const float fa = 1.0f - rd - z * z;
    const float a = q.am * fa;
    const float lbv = -v * inv_dt;
    const bool beta = lbv > a_min;
    const float a_lb = beta ? lbv : a_min;
    float e2;
    sp(a - a_lb, e2);
    const float sig2 = sigm(a - a_lb, e2);
    const float Sn = 2.0f * q.am * z * ig;                 // -d a / d s*
    const float w = sig2 * Sn * sig1;                      // -d a* / d s_opt
    o.dv = -sig2 * q.am * q.delta * rdm1 * q.inv_v0 - w * (q.T + q.c * (dvel + v)) +
           (beta ? -(1.0f - sig2) * inv_dt : 0.0f);
    o.dvh = w * q.c * v;
    o.dgap = floored ? 0.0f : sig2 * Sn * z;
    o.dth[0] = sig2 * q.am * q.delta * rd * q.inv_v0;
    o.dth[1] = -w * v;
    o.dth[2] = -w;
    o.dth[3] = sig2 * fa + w * v * dvel * q.c / (2.0f * q.am);
    o.dth[4] = w * v * dvel * q.c / (2.0f * q.b);
    o.dth[5] = (r > 0.0f && rd > 0.0f) ? -sig2 * q.am * rd * logf(r) : 0.0f;   // r -> 0+ limit near rest
    return o;
}

struct Problem {
    const idm_cpu_scene_t *sc;
    float *th[6];
    const float *p_init, *v_init;
    int K;
    float dt, inv_dt, a_min;
    const float *targets;
    int stride, n_obs;
};

// Per-thread scratch for one lane.
struct Lane {
    int n = 0;
    std::vector<Veh> q;
    std::vector<float> ph, pl, v, gap, tv, tg, seed, lp, lv, lg, mu;
    std::vector<double> lossv, gsum;
    void resize(int n_, int K, int n_obs)
    {
        n = n_;
        q.resize(n);
        for (auto *a : {&ph, &pl, &v, &gap, &lp, &lv, &lg, &mu}) a->resize(n + 1);
        tv.resize((size_t)K * n);
        tg.resize((size_t)K * n);
        seed.resize((size_t)std::max(n_obs, 1) * n);
        lossv.resize(n);
        gsum.resize((size_t)6 * n);
    }
};

void load_params(const Problem &P, int i0, Lane &L)
{
    for (int i = 0; i < L.n; ++i) {
        Veh &q = L.q[i];
        const int g = i0 + i;
        q.v0 = P.th[0][g];
        q.T = P.th[1][g];
        q.s0 = P.th[2][g];
        q.am = P.th[3][g];
        q.b = P.th[4][g];
        q.delta = P.th[5][g];
        q.inv_v0 = 1.0f / q.v0;
        q.c = 0.5f / sqrtf(q.am * q.b);   // 1 / (2 sqrt(a_max b)), Eq. 1
    }
}

// Forward over K steps of the lane starting at global index i0.  With seeds,
// records the tape and the loss seeds 2 r / n_obs; returns the lane's loss.
double lane_forward(const Problem &P, int i0, Lane &L, bool tape, float *traj, float *vtraj, bool &bad)
{
    const int n = L.n;
    const size_t N = (size_t)P.sc->n_vehicles;
    const float *len = P.sc->length;
    for (int i = 0; i < n; ++i) {
        L.ph[i] = P.p_init[i0 + i];
        L.pl[i] = 0.0f;
        L.v[i] = P.v_init[i0 + i];
        L.gap[i] = i == 0 ? std::numeric_limits<float>::infinity()
                          : P.p_init[i0 + i - 1] - P.p_init[i0 + i] - len[i0 + i - 1];
        L.lossv[i] = 0.0;
    }
    if (traj)
        for (int i = 0; i < n; ++i) traj[i0 + i] = L.ph[i];
    if (vtraj)
        for (int i = 0; i < n; ++i) vtraj[i0 + i] = L.v[i];
    const float dt = P.dt;
    for (int k = 0; k < P.K; ++k) {
        if (tape) {
            memcpy(&L.tv[(size_t)k * n], L.v.data(), sizeof(float) * n);
            memcpy(&L.tg[(size_t)k * n], L.gap.data(), sizeof(float) * n);
        }
        // back to front, so v[i-1] is still the step-k speed of i's leader
        for (int i = n - 1; i >= 0; --i) {
            const float vi = L.v[i];
            const float vh = i > 0 ? L.v[i - 1] : vi;
            const float as = accel(vi, L.gap[i], vh, L.q[i], P.inv_dt, P.a_min);
            // position pair: TwoSum of ph + dt v plus the rounding error of dt v
            const float d = dt * vi;
            const float en = fmaf(-dt, vi, d);
            const float t = L.ph[i] + d;
            const float bb = t - L.ph[i];
            const float err = (L.ph[i] - (t - bb)) + (d - bb);
            L.ph[i] = t;
            L.pl[i] += err - en;
            if (i > 0) L.gap[i] = fmaf(dt, vh - vi, L.gap[i]);
            L.v[i] = fmaf(dt, as, vi);
        }
        const int k1 = k + 1;
        if (traj)
            for (int i = 0; i < n; ++i) traj[(size_t)k1 * N + i0 + i] = L.ph[i] + L.pl[i];
        if (vtraj)
            for (int i = 0; i < n; ++i) vtraj[(size_t)k1 * N + i0 + i] = L.v[i];
        if (P.targets && P.n_obs > 0 && k1 % P.stride == 0 && k1 / P.stride <= P.n_obs) {
            const int j = k1 / P.stride - 1;
            const float *y = P.targets + (size_t)j * N + i0;
            for (int i = 0; i < n; ++i) {
                const float r = (L.ph[i] - y[i]) + L.pl[i];
                L.lossv[i] += (double)r * (double)r;
                if (tape) L.seed[(size_t)j * n + i] = 2.0f * r / (float)P.n_obs;
            }
        }
    }
    double lane_loss = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(L.v[i]) || !std::isfinite(L.ph[i])) bad = true;
        if (P.n_obs > 0) lane_loss += L.lossv[i] / P.n_obs;
    }
    return lane_loss;
}

// Reverse sweep over the tape: parameter-gradient sums gsum[6][n] (double),
// lp, lv (adjoints of the initial position and speed; lg of the initial gap).
void lane_adjoint(const Problem &P, Lane &L, bool want_delta, bool &bad)
{
    const int n = L.n;
    const float dt = P.dt;
    std::fill(L.lp.begin(), L.lp.end(), 0.0f);
    std::fill(L.lv.begin(), L.lv.end(), 0.0f);
    std::fill(L.lg.begin(), L.lg.end(), 0.0f);
    std::fill(L.gsum.begin(), L.gsum.end(), 0.0);
    for (int k = P.K - 1; k >= 0; --k) {
        const int k1 = k + 1;
        // seeds of the state at step k+1
        if (P.n_obs > 0 && k1 % P.stride == 0 && k1 / P.stride <= P.n_obs) {
            const float *s = &L.seed[(size_t)(k1 / P.stride - 1) * n];
            for (int i = 0; i < n; ++i) L.lp[i] += s[i];
        }
        const float *v = &L.tv[(size_t)k * n];
        const float *g = &L.tg[(size_t)k * n];
        for (int i = 0; i < n; ++i) L.mu[i] = dt * L.lv[i];
        // lambda(k) from lambda(k+1); the follower terms read mu[i+1] and
        // the step-(k+1) gap adjoint of the follower, both still unchanged
        float mu_f = 0.0f, dvh_f = 0.0f, lg_f = 0.0f;   // follower (i+1) terms
        for (int i = n - 1; i >= 0; --i) {
            const float vh = i > 0 ? v[i - 1] : v[i];
            const Part d = partials(v[i], g[i], vh, L.q[i], P.inv_dt, P.a_min);
            const float mu = L.mu[i];
            for (int r = 0; r < 6; ++r)
                if (r < 5 || want_delta) L.gsum[(size_t)r * n + i] += (double)mu * (double)d.dth[r];
            const float lg_i = L.lg[i];                 // step-(k+1) gap adjoint of i
            const float lv_new = L.lv[i] + dt * L.lp[i] + mu * d.dv + mu_f * dvh_f + dt * (lg_f - (i > 0 ? lg_i : 0.0f));
            L.lg[i] = i > 0 ? lg_i + mu * d.dgap : 0.0f;
            mu_f = mu;
            dvh_f = d.dvh;
            lg_f = lg_i;
            L.lv[i] = lv_new;
        }
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(L.lv[i]) || !std::isfinite(L.lp[i])) bad = true;
}

int check_common(const idm_cpu_scene_t *sc, const idm_cpu_params_t *p, const float *p_init, const float *v_init,
                 const idm_sim_t *sim)
{
    if (!sc || !p || !sim) return IDM_ERR_ARG;
    if (sc->n_lanes < 0 || sc->n_vehicles < 0) return IDM_ERR_ARG;
    if (sc->n_vehicles > 0 && (!sc->length || !p_init || !v_init)) return IDM_ERR_ARG;
    if (sc->n_lanes > 0 && !sc->lane_off) return IDM_ERR_ARG;
    if (!p->v0 || !p->T || !p->s0 || !p->a_max || !p->b || !p->delta) return IDM_ERR_ARG;
    if (sim->K < 1 || !(sim->dt > 0.0f) || !std::isfinite(sim->dt) || !(sim->a_min < 0.0f)) return IDM_ERR_ARG;
    if (sc->n_lanes > 0) {
        if (sc->lane_off[0] != 0 || sc->lane_off[sc->n_lanes] != sc->n_vehicles) return IDM_ERR_ARG;
        for (int l = 0; l < sc->n_lanes; ++l)
            if (sc->lane_off[l + 1] < sc->lane_off[l]) return IDM_ERR_ARG;
    } else if (sc->n_vehicles != 0) {
        return IDM_ERR_ARG;
    }
    return IDM_OK;
}

int threads_of(int n_threads) { return n_threads > 0 ? n_threads : omp_get_max_threads(); }

Problem make_problem(const idm_cpu_scene_t *sc, const idm_cpu_params_t *p, const float *p_init, const float *v_init,
                     const idm_sim_t *sim, const float *targets, int stride)
{
    Problem P;
    P.sc = sc;
    float *th[6] = {p->v0, p->T, p->s0, p->a_max, p->b, p->delta};
    for (int q = 0; q < 6; ++q) P.th[q] = th[q];
    P.p_init = p_init;
    P.v_init = v_init;
    P.K = sim->K;
    P.dt = sim->dt;
    P.inv_dt = 1.0f / sim->dt;
    P.a_min = sim->a_min;
    P.targets = targets;
    P.stride = stride > 0 ? stride : 1;
    P.n_obs = targets ? sim->K / P.stride : 0;
    return P;
}

}  // namespace

extern "C" int idm_cpu_max_threads(void) { return omp_get_max_threads(); }

extern "C" int idm_cpu_forward(int n_threads, const idm_cpu_scene_t *sc, const idm_cpu_params_t *p,
                               const float *p_init, const float *v_init, const idm_sim_t *sim, float *traj,
                               float *vtraj)
{
    int rc = check_common(sc, p, p_init, v_init, sim);
    if (rc) return rc;
    const Problem P = make_problem(sc, p, p_init, v_init, sim, nullptr, 1);
    bool bad = false, oom = false;
#pragma omp parallel num_threads(threads_of(n_threads)) reduction(|| : bad, oom)
    {
        Lane L;
#pragma omp for schedule(dynamic, 1)
        for (int l = 0; l < sc->n_lanes; ++l) {
            const int i0 = sc->lane_off[l], n = sc->lane_off[l + 1] - i0;
            if (n == 0) continue;
            try {
                L.resize(n, 0, 0);
            } catch (const std::bad_alloc &) {
                oom = true;
                continue;
            }
            load_params(P, i0, L);
            lane_forward(P, i0, L, false, traj, vtraj, bad);
        }
    }
    if (oom) return IDM_ERR_WORKSPACE;
    return bad ? IDM_ERR_NONFINITE : IDM_OK;
}

extern "C" int idm_cpu_loss_grad(int n_threads, const idm_cpu_scene_t *sc, const idm_cpu_params_t *p,
                                 const float *p_init, const float *v_init, const idm_sim_t *sim, const float *targets,
                                 int32_t obs_stride, double *loss_out, idm_cpu_params_t *grad, float *g_p_init,
                                 float *g_v_init)
{
    int rc = check_common(sc, p, p_init, v_init, sim);
    if (rc) return rc;
    if (obs_stride < 1) return IDM_ERR_ARG;
    const Problem P = make_problem(sc, p, p_init, v_init, sim, targets, obs_stride);
    if (P.n_obs > 0 && !targets) return IDM_ERR_ARG;
    float *gout[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (grad) {
        float *g[6] = {grad->v0, grad->T, grad->s0, grad->a_max, grad->b, grad->delta};
        for (int q = 0; q < 6; ++q) gout[q] = g[q];
    }
    const bool want_delta = gout[5] != nullptr;
    std::vector<double> lane_loss((size_t)std::max(sc->n_lanes, 1), 0.0);
    bool bad = false, oom = false;
#pragma omp parallel num_threads(threads_of(n_threads)) reduction(|| : bad, oom)
    {
        Lane L;
#pragma omp for schedule(dynamic, 1)
        for (int l = 0; l < sc->n_lanes; ++l) {
            const int i0 = sc->lane_off[l], n = sc->lane_off[l + 1] - i0;
            if (n == 0) continue;
            try {
                L.resize(n, P.K, P.n_obs);
            } catch (const std::bad_alloc &) {
                oom = true;
                continue;
            }
            load_params(P, i0, L);
            lane_loss[l] = lane_forward(P, i0, L, true, nullptr, nullptr, bad);
            lane_adjoint(P, L, want_delta, bad);
            for (int i = 0; i < n; ++i) {
                for (int r = 0; r < 6; ++r)
                    if (gout[r]) gout[r][i0 + i] = (r == 5 && !want_delta) ? 0.0f : (float)L.gsum[(size_t)r * n + i];
                // initial state: the initial gap of i is p_{i-1} - p_i - len, so
                // the position adjoint also collects -lg_i + lg_{i+1}
                if (g_p_init) g_p_init[i0 + i] = L.lp[i] - (i > 0 ? L.lg[i] : 0.0f) + (i + 1 < n ? L.lg[i + 1] : 0.0f);
                if (g_v_init) g_v_init[i0 + i] = L.lv[i];
            }
        }
    }
    if (oom) return IDM_ERR_WORKSPACE;
    if (loss_out) {
        double s = 0.0;
        for (int l = 0; l < sc->n_lanes; ++l) s += lane_loss[l];
        *loss_out = s;
    }
    return bad ? IDM_ERR_NONFINITE : IDM_OK;
}

extern "C" int idm_cpu_fit(int n_threads, const idm_cpu_scene_t *sc, idm_cpu_params_t *p, const float *p_init,
                           const float *v_init, const idm_sim_t *sim, const float *targets, int32_t obs_stride,
                           int32_t n_iter, float lr0, float lr1, const float *box_lo, const float *box_hi,
                           double *loss_hist)
{
    int rc = check_common(sc, p, p_init, v_init, sim);
    if (rc) return rc;
    if (obs_stride < 1 || n_iter < 1 || n_iter > 100000 || !box_lo || !box_hi) return IDM_ERR_ARG;
    const Problem P = make_problem(sc, p, p_init, v_init, sim, targets, obs_stride);
    if (P.n_obs > 0 && !targets) return IDM_ERR_ARG;
    std::vector<double> lane_loss;
    try {
        lane_loss.assign((size_t)std::max(sc->n_lanes, 1) * n_iter, 0.0);
    } catch (const std::bad_alloc &) {
        return IDM_ERR_WORKSPACE;
    }
    bool bad = false, oom = false;
#pragma omp parallel num_threads(threads_of(n_threads)) reduction(|| : bad, oom)
    {
        Lane L;
        std::vector<float> m, w;
#pragma omp for schedule(dynamic, 1)
        for (int l = 0; l < sc->n_lanes; ++l) {
            const int i0 = sc->lane_off[l], n = sc->lane_off[l + 1] - i0;
            if (n == 0) continue;
            try {
                L.resize(n, P.K, P.n_obs);
                m.assign((size_t)5 * n, 0.0f);
                w.assign((size_t)5 * n, 0.0f);
            } catch (const std::bad_alloc &) {
                oom = true;
                continue;
            }
            for (int it = 0; it < n_iter; ++it) {
                load_params(P, i0, L);
                lane_loss[(size_t)l * n_iter + it] = lane_forward(P, i0, L, true, nullptr, nullptr, bad);
                lane_adjoint(P, L, false, bad);
                const int t = it + 1;
                const float lr = n_iter > 1 ? lr0 + (lr1 - lr0) * (float)it / (float)(n_iter - 1) : lr0;
                const float bc1 = 1.0f - powf(0.9f, (float)t), bc2 = 1.0f - powf(0.999f, (float)t);
                for (int i = 0; i < n; ++i)
                    for (int r = 0; r < 5; ++r) {
                        const float g = (float)L.gsum[(size_t)r * n + i];
                        float &mm = m[(size_t)r * n + i], &ww = w[(size_t)r * n + i];
                        mm = 0.9f * mm + 0.1f * g;
                        ww = 0.999f * ww + 0.001f * g * g;
                        float x = P.th[r][i0 + i] - lr * (mm / bc1) / (sqrtf(ww / bc2) + 1e-8f);
                        P.th[r][i0 + i] = fminf(fmaxf(x, box_lo[r]), box_hi[r]);
                    }
            }
        }
    }
    if (oom) return IDM_ERR_WORKSPACE;
    if (loss_hist)
        for (int it = 0; it < n_iter; ++it) {
            double s = 0.0;
            for (int l = 0; l < sc->n_lanes; ++l) s += lane_loss[(size_t)l * n_iter + it];
            loss_hist[it] = s;
        }
    return bad ? IDM_ERR_NONFINITE : IDM_OK;
}
