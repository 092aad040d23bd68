/*
 * FP64 CPU oracle of the single-trajectory reconstruction mode of the paper
 * (Sec. IV-A): every trajectory is one ego vehicle simulated with the
 * modified IDM (Eq. 1-3 and the bounds of Sec. III-C) behind a virtual
 * leader whose gap dp_k and speed difference dv_k at every step k are free
 * variables (initialised to 10 and 0 in the paper), fitted together with the
 * five IDM parameters by minimising the summed absolute error between the
 * observed positions and the simulated position at the nearest step.
 *
 * TEST INFRASTRUCTURE ONLY (as idm_oracle.c): loaded by the tests, the smoke
 * check and the CPU legs of the benchmark; shares nothing with the CUDA
 * library.
 *
 * Readings (also listed in the design notes):
 *   - dv_k is v - v_leader (Sec. III-A), a free variable: ds_opt/dv = T +
 *     c dv_k (no dependence of dv_k on v).
 *   - The gap floor of the coupled model applies to dp_k (max(dp_k, 0.1 m),
 *     derivative 0 below).
 *   - The nearest step of a timestamp t is k = floor(t / dt + 1/2) (half up);
 *     observations that map to step 0 (the given initial state) are not
 *     part of the loss.
 *   - |x| has subgradient sign(x) with sign(0) = 0.
 *   - Initial state (Sec. V-B): p(0) = the first observed position and v(0)
 *     = (second - first observed position) / (their time difference),
 *     clamped at 0 (the simulator keeps speeds non-negative, Sec. III-C);
 *     0 with fewer than two observations or equal first timestamps.
 *   - Trajectory i is simulated for K_i = the nearest step of its last
 *     observation; arrays are time-major [K_max (+1)][N]; entries beyond K_i
 *     hold the final state (positions, speeds) or zero (accelerations,
 *     gradients).
 *   - Adam as in the coupled fit; the parameters are projected onto the box,
 *     dp_k and dv_k are unconstrained.
 *   - Metrics (Sec. V-B): Pos. = mean over all observations of |error| /
 *     (trajectory length = |last - first observed position|); Acc. = mean and
 *     standard deviation of |a*| over every simulated step of every
 *     trajectory; Imp. = fraction of trajectories with some |a*| > 10.
 * Parity unpinned: none (the CPU tests pin every function).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define R_FLOOR 0.1

static double r_sp(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }
static double r_sigm(double x)
{
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x));
    double e = exp(x);
    return e / (1.0 + e);
}

typedef struct {
    double a_star;
    double d_v, d_dp, d_dv;  /* partials of a* w.r.t. own speed, dp_k, dv_k */
    double d_th[6];          /* w.r.t. v0, T, s0, a_max, b, delta */
} vl_eval;

/* The modified IDM of one ego vehicle with speed v behind a virtual leader
 * at gap dp_raw with speed difference dv (Eq. 1-2, Sec. III-C). */
static vl_eval eval_vl(double v, double dp_raw, double dv, const double th[6], double dt, double a_min)
{
    const double v0 = th[0], T = th[1], s0 = th[2], am = th[3], b = th[4], dl = th[5];
    vl_eval o;
    memset(&o, 0, sizeof o);
    double r = v / v0, rd = pow(r, dl);
    double dp = dp_raw;
    int floored = 0;
    if (dp < R_FLOOR) { dp = R_FLOOR; floored = 1; }
    double c = 1.0 / (2.0 * sqrt(am * b));              /* Eq. 1 */
    double s_opt = s0 + v * T + v * dv * c;              /* Eq. 1 */
    double sstar = r_sp(s_opt), sig1 = r_sigm(s_opt);   /* Sec. III-C */
    double z = sstar / dp;
    double a = am * (1.0 - rd - z * z);                  /* Eq. 2 */
    double lb_v = -v / dt;
    int beta = lb_v > a_min;
    double a_lb = beta ? lb_v : a_min;
    o.a_star = a_lb + r_sp(a - a_lb);
    double sig2 = r_sigm(a - a_lb);

    double S = -2.0 * am * z / dp;                       /* da/ds* */
    double G = floored ? 0.0 : 2.0 * am * z * z / dp;    /* da/d dp */
    double da_dv_direct = (v > 0.0 || dl > 1.0) ? -am * dl * pow(r, dl - 1.0) / v0
                                                 : (dl == 1.0 ? -am / v0 : -INFINITY);
    double da_dv = da_dv_direct + S * sig1 * (T + c * dv);  /* ds_opt/dv = T + c dv_k */
    double da_ddv = S * sig1 * (v * c);                     /* ds_opt/d dv_k = c v */
    o.d_v = sig2 * da_dv + (1.0 - sig2) * (beta ? -1.0 / dt : 0.0);
    o.d_dp = sig2 * G;
    o.d_dv = sig2 * da_ddv;
    double lnr = (r > 0.0) ? log(r) : 0.0;
    o.d_th[0] = sig2 * (am * dl * rd / v0);
    o.d_th[1] = sig2 * (S * sig1 * v);
    o.d_th[2] = sig2 * (S * sig1);
    o.d_th[3] = sig2 * ((1.0 - rd - z * z) + S * sig1 * (-v * dv * c / (2.0 * am)));
    o.d_th[4] = sig2 * (S * sig1 * (-v * dv * c / (2.0 * b)));
    o.d_th[5] = sig2 * (-am * rd * lnr);
    return o;
}

/* Nearest step of a timestamp (seconds from the trajectory's start). */
int orc_recon_nearest_step(double t, double dt) { return (int)floor(t / dt + 0.5); }

void orc_recon_nearest_steps(int64_t n, const double *t, double dt, int32_t *k)
{
    for (int64_t j = 0; j < n; ++j) k[j] = orc_recon_nearest_step(t[j], dt);
}

/* Initial state of Sec. V-B from the first two observations of each
 * trajectory (observations obs_off[i] .. obs_off[i+1]-1, in time order). */
void orc_recon_init_state(int N, const int32_t *obs_off, const double *obs_t, const double *obs_p, double *p0,
                          double *v0)
{
    for (int i = 0; i < N; ++i) {
        int j0 = obs_off[i], n = obs_off[i + 1] - j0;
        p0[i] = n > 0 ? obs_p[j0] : 0.0;
        double dt01 = n > 1 ? obs_t[j0 + 1] - obs_t[j0] : 0.0;
        v0[i] = dt01 > 0.0 ? fmax((obs_p[j0 + 1] - obs_p[j0]) / dt01, 0.0) : 0.0;
    }
}

/* Forward simulation (Eq. 3) of every trajectory for its K[i] steps. */
void orc_recon_forward(int N, int K_max, const int32_t *K, const double *dp, const double *dv,
                       const double *const th6[6], const double *p0, const double *v0, double dt, double a_min,
                       double *P, double *V, double *A)
{
    for (int i = 0; i < N; ++i) {
        double th[6];
        for (int q = 0; q < 6; ++q) th[q] = th6[q][i];
        double p = p0[i], v = v0[i];
        P[i] = p;
        if (V) V[i] = v;
        for (int k = 0; k < K_max; ++k) {
            size_t at = (size_t)k * N + i, next = (size_t)(k + 1) * N + i;
            if (k < K[i]) {
                vl_eval e = eval_vl(v, dp[at], dv[at], th, dt, a_min);
                if (A) A[at] = e.a_star;
                double pn = p + dt * v;           /* Eq. 3: position uses the old speed */
                v = v + dt * e.a_star;
                p = pn;
            } else if (A) {
                A[at] = 0.0;
            }
            P[next] = p;
            if (V) V[next] = v;
        }
    }
}

/* Summed absolute error at the observed steps (observations at step 0 or
 * beyond K[i] excluded) and the seeds dL/dP[k][i] (sign of the error, added
 * for every observation at that step). */
double orc_recon_mae_seed(int N, int K_max, const int32_t *K, const int32_t *obs_off, const int32_t *obs_k,
                          const double *obs_p, const double *P, double *gP)
{
    memset(gP, 0, sizeof(double) * (size_t)(K_max + 1) * N);
    double L = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = obs_off[i]; j < obs_off[i + 1]; ++j) {
            int k = obs_k[j];
            if (k < 1 || k > K[i]) continue;
            double r = P[(size_t)k * N + i] - obs_p[j];
            L += fabs(r);
            gP[(size_t)k * N + i] += (r > 0.0) - (r < 0.0);
        }
    return L;
}

/* Reverse-time adjoint of orc_recon_forward for seeds gP: gradients of the
 * parameters (g6, 6 x N), of dp and dv ([K_max][N]) and of the initial
 * state.  With mu = dt lambda_v(k+1) and a_star the bounded acceleration:
 *   lambda_p(k) = gP[k] + lambda_p(k+1),
 *   lambda_v(k) = dt lambda_p(k+1) + lambda_v(k+1) + mu (d a_star / d v),
 *   dL/d dp_k = mu (d a_star / d dp_k),  dL/d dv_k = mu (d a_star / d dv_k),
 *   dL/d theta += mu (d a_star / d theta). */
void orc_recon_adjoint(int N, int K_max, const int32_t *K, const double *dp, const double *dv,
                       const double *const th6[6], double dt, double a_min, const double *V, const double *gP,
                       double *const g6[6], double *gdp, double *gdv, double *gp0, double *gv0)
{
    for (int i = 0; i < N; ++i) {
        double th[6];
        for (int q = 0; q < 6; ++q) th[q] = th6[q][i];
        double lp = gP[(size_t)K[i] * N + i], lv = 0.0, gt[6] = {0, 0, 0, 0, 0, 0};
        for (int k = K_max - 1; k >= K[i]; --k) {
            gdp[(size_t)k * N + i] = 0.0;
            gdv[(size_t)k * N + i] = 0.0;
        }
        for (int k = K[i] - 1; k >= 0; --k) {
            size_t at = (size_t)k * N + i;
            vl_eval e = eval_vl(V[at], dp[at], dv[at], th, dt, a_min);
            double mu = dt * lv;
            gdp[at] = mu * e.d_dp;
            gdv[at] = mu * e.d_dv;
            for (int q = 0; q < 6; ++q) gt[q] += mu * e.d_th[q];
            double nlp = (k >= 1 ? gP[at] : 0.0) + lp;
            double nlv = dt * lp + lv + mu * e.d_v;
            lp = nlp;
            lv = nlv;
        }
        for (int q = 0; q < 6; ++q) g6[q][i] = gt[q];
        if (gp0) gp0[i] = lp;
        if (gv0) gv0[i] = lv;
    }
}

static void adam(double *x, const double *g, double *m, double *v, int t, double lr, double lo, double hi, int box)
{
    double bc1 = 1.0 - pow(0.9, t), bc2 = 1.0 - pow(0.999, t);
    *m = 0.9 * *m + 0.1 * *g;
    *v = 0.999 * *v + 0.001 * *g * *g;
    double nx = *x - lr * (*m / bc1) / (sqrt(*v / bc2) + 1e-8);
    if (box) nx = fmin(fmax(nx, lo), hi);
    *x = nx;
}

double orc_lr(int it, int n_iter, double lr0, double lr1);

/* n_iter Adam iterations on (v0, T, s0, a_max, b) (box) and every dp_k, dv_k
 * (k < K[i], unconstrained); loss_hist[it] = the loss before update it. */
void orc_recon_fit(int N, int K_max, const int32_t *K, double *dp, double *dv, double *const th6[6],
                   const double *p0, const double *v0, double dt, double a_min, const int32_t *obs_off,
                   const int32_t *obs_k, const double *obs_p, int n_iter, double lr0, double lr1,
                   const double lo[5], const double hi[5], double *loss_hist)
{
    size_t SN = (size_t)(K_max + 1) * N, KN = (size_t)K_max * N;
    double *P = malloc(sizeof(double) * SN), *V = malloc(sizeof(double) * SN), *gP = malloc(sizeof(double) * SN);
    double *gdp = calloc(KN ? KN : 1, sizeof(double)), *gdv = calloc(KN ? KN : 1, sizeof(double));
    double *mdp = calloc(KN ? KN : 1, sizeof(double)), *vdp = calloc(KN ? KN : 1, sizeof(double));
    double *mdv = calloc(KN ? KN : 1, sizeof(double)), *vdv = calloc(KN ? KN : 1, sizeof(double));
    double *g[6], *m[5], *vv[5];
    for (int q = 0; q < 6; ++q) g[q] = calloc((size_t)N, sizeof(double));
    for (int q = 0; q < 5; ++q) { m[q] = calloc((size_t)N, sizeof(double)); vv[q] = calloc((size_t)N, sizeof(double)); }
    for (int it = 0; it < n_iter; ++it) {
        const double *cth[6];
        for (int q = 0; q < 6; ++q) cth[q] = th6[q];
        orc_recon_forward(N, K_max, K, dp, dv, cth, p0, v0, dt, a_min, P, V, NULL);
        loss_hist[it] = orc_recon_mae_seed(N, K_max, K, obs_off, obs_k, obs_p, P, gP);
        orc_recon_adjoint(N, K_max, K, dp, dv, cth, dt, a_min, V, gP, g, gdp, gdv, NULL, NULL);
        double lr = orc_lr(it, n_iter, lr0, lr1);
        for (int i = 0; i < N; ++i) {
            for (int q = 0; q < 5; ++q) adam(&th6[q][i], &g[q][i], &m[q][i], &vv[q][i], it + 1, lr, lo[q], hi[q], 1);
            for (int k = 0; k < K[i]; ++k) {
                size_t at = (size_t)k * N + i;
                adam(&dp[at], &gdp[at], &mdp[at], &vdp[at], it + 1, lr, 0, 0, 0);
                adam(&dv[at], &gdv[at], &mdv[at], &vdv[at], it + 1, lr, 0, 0, 0);
            }
        }
    }
    free(P); free(V); free(gP); free(gdp); free(gdv); free(mdp); free(vdp); free(mdv); free(vdv);
    for (int q = 0; q < 6; ++q) free(g[q]);
    for (int q = 0; q < 5; ++q) { free(m[q]); free(vv[q]); }
}

/* Metrics of Sec. V-B: out[0] Pos. (mean relative positional error), out[1]
 * mean |a*|, out[2] standard deviation of |a*|, out[3] Imp. (fraction of
 * trajectories with some |a*| > 10). */
void orc_recon_metrics(int N, int K_max, const int32_t *K, const int32_t *obs_off, const int32_t *obs_k,
                       const double *obs_p, const double *P, const double *A, double *out)
{
    double pos = 0.0, s1 = 0.0, s2 = 0.0;
    long n_pos = 0, n_a = 0, n_imp = 0;
    for (int i = 0; i < N; ++i) {
        int j0 = obs_off[i], j1 = obs_off[i + 1];
        double len = j1 > j0 ? fabs(obs_p[j1 - 1] - obs_p[j0]) : 0.0;
        for (int j = j0; j < j1; ++j) {
            int k = obs_k[j];
            if (k < 0 || k > K[i] || len <= 0.0) continue;
            pos += fabs(P[(size_t)k * N + i] - obs_p[j]) / len;
            ++n_pos;
        }
        int imp = 0;
        for (int k = 0; k < K[i]; ++k) {
            double a = fabs(A[(size_t)k * N + i]);
            s1 += a;
            s2 += a * a;
            ++n_a;
            if (a > 10.0) imp = 1;
        }
        n_imp += imp;
    }
    double mean = n_a ? s1 / n_a : 0.0;
    out[0] = n_pos ? pos / n_pos : 0.0;
    out[1] = mean;
    out[2] = n_a ? sqrt(fmax(s2 / n_a - mean * mean, 0.0)) : 0.0;
    out[3] = N ? (double)n_imp / N : 0.0;
}
