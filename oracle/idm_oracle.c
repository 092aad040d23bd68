/*
 * FP64 CPU oracle for the modified Intelligent Driver Model (IDM) simulator
 * and its reverse-time adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library; it is a plain, single-threaded,
 * deliberately unoptimised restatement of the method, so that a reader can
 * check each line against the paper.
 *
 * Paper: "Gradient-based Trajectory Optimization with Parallelized
 * Differentiable Traffic Simulation" (arXiv 2412.16750).
 *   Sec. III-A : leader relation (gap, speed difference), Eq. 1 (desired gap),
 *                Eq. 2 (IDM acceleration), Eq. 3 (explicit Euler step).
 *   Sec. III-C : realism fixes -- softplus lower bound on the desired gap and
 *                softplus lower bound a_lb = max(-v/dt, a_min) on the
 *                acceleration.
 *   Sec. IV-A  : reconstruction loss over observed steps, the five optimised
 *                parameters, their boxes and a_min = -10.
 *   Sec. V-B   : Adam with the learning rate decayed linearly 0.1 -> 0.01.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - Jacobi update: every vehicle at step k reads its leader's step-k state.
 *   - Lane head (no leader): free-road term only, z = 0.
 *   - Gap floor: dp = max(dp, S_FLOOR) with S_FLOOR = 0.1 m, derivative 0 when
 *     the raw gap is strictly below the floor.
 *   - a_lb = -v/dt when -v/dt > a_min strictly; a tie takes a_min (derivative 0).
 *   - Loss: sum over vehicles of that vehicle's mean squared error over the
 *     observed steps k = s, 2s, ..., <= K (step 0 never observed).  The paper
 *     sums per-trajectory losses; the multi-vehicle fits here use the squared
 *     error (the single-trajectory absolute error is recon_oracle.c).
 *   - Parameter order used everywhere in this file:
 *       0 v0 (= v_targ), 1 T (= T_pref), 2 s0 (= s_min), 3 a_max,
 *       4 b (= a_pref), 5 delta.
 *
 * Parity unpinned: none of the functions below -- every one is pinned by the
 * CPU tests (closed forms, invariants, finite differences, brute force, an
 * independent library routine).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define S_FLOOR 0.1

/* Softplus as written in Sec. III-C, sp(x) = log(1 + exp(x)), evaluated in a
 * form that does not overflow: max(x, 0) + log1p(exp(-|x|)). */
static double sp(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

/* Logistic sigmoid, the derivative of sp. */
static double sigm(double x)
{
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x));
    double e = exp(x);
    return e / (1.0 + e);
}

/* Everything the forward step and the adjoint need about one vehicle at one
 * step, evaluated from the step-k state. */
typedef struct {
    double a_star;   /* bounded acceleration a* (Sec. III-C) */
    /* partial derivatives of a* */
    double d_p;      /* w.r.t. own position */
    double d_v;      /* w.r.t. own speed */
    double d_ph;     /* w.r.t. leader position */
    double d_vh;     /* w.r.t. leader speed */
    double d_th[6];  /* w.r.t. v0, T, s0, a_max, b, delta */
} step_eval;

/*
 * One evaluation of the modified IDM for a vehicle with speed v, leader data
 * (has_leader, dp_raw = p_h - p - length_h, v_h) and parameters th[6].
 */
static step_eval eval_vehicle(int has_leader, double v, double dp_raw, double vh,
                              const double th[6], double dt, double a_min)
{
    const double v0 = th[0], T = th[1], s0 = th[2], am = th[3], b = th[4], dl = th[5];
    step_eval o;
    memset(&o, 0, sizeof o);

    /* free-road term (v / v_targ)^delta of Eq. 2 */
    double r = v / v0;
    double rd = pow(r, dl);

    /* interaction term (s*_opt / dp)^2 of Eq. 2, with s*_opt = sp(s_opt)
     * (Sec. III-C) and s_opt from Eq. 1 */
    double z = 0.0, sstar = 0.0, sig1 = 0.0, c = 0.0, dv = 0.0, dp = 0.0;
    int floored = 0;
    if (has_leader) {
        dp = dp_raw;
        if (dp < S_FLOOR) { dp = S_FLOOR; floored = 1; }
        dv = v - vh;                                   /* Sec. III-A */
        c = 1.0 / (2.0 * sqrt(am * b));                /* Eq. 1 */
        double s_opt = s0 + v * T + v * dv * c;        /* Eq. 1 */
        sstar = sp(s_opt);
        sig1 = sigm(s_opt);
        z = sstar / dp;
    }
    double a = am * (1.0 - rd - z * z);                /* Eq. 2 */

    /* lower bound of Sec. III-C */
    double lb_v = -v / dt;
    int beta = lb_v > a_min;
    double a_lb = beta ? lb_v : a_min;
    o.a_star = a_lb + sp(a - a_lb);
    double sig2 = sigm(a - a_lb);

    /* derivatives of a (before the bound) */
    double da_dv_direct = (v > 0.0 || dl > 1.0) ? -am * dl * pow(r, dl - 1.0) / v0
                                                 : (dl == 1.0 ? -am / v0 : -INFINITY);
    double S = 0.0, G = 0.0;       /* da/ds*, da/ddp */
    if (has_leader) {
        S = -2.0 * am * z / dp;
        G = floored ? 0.0 : 2.0 * am * z * z / dp;
    }
    double da_dv = da_dv_direct + S * sig1 * (T + c * (dv + v)); /* ds_opt/dv = T + c dv + c v */
    double da_dvh = S * sig1 * (-c * v);                          /* ds_opt/dvh = -c v */
    /* chain through a* = a_lb + sp(a - a_lb) */
    o.d_p = sig2 * (-G);
    o.d_ph = sig2 * G;
    o.d_vh = sig2 * da_dvh;
    o.d_v = sig2 * da_dv + (1.0 - sig2) * (beta ? -1.0 / dt : 0.0);

    double lnr = (r > 0.0) ? log(r) : 0.0;
    o.d_th[0] = sig2 * (am * dl * rd / v0);                              /* v0 */
    o.d_th[1] = sig2 * (S * sig1 * v);                                   /* T */
    o.d_th[2] = sig2 * (S * sig1);                                       /* s0 */
    o.d_th[3] = sig2 * ((1.0 - rd - z * z) + S * sig1 * (-v * dv * c / (2.0 * am))); /* a_max */
    o.d_th[4] = sig2 * (S * sig1 * (-v * dv * c / (2.0 * b)));           /* b */
    o.d_th[5] = sig2 * (-am * rd * lnr);                                 /* delta */
    return o;
}

/* Parameters as six separate arrays, each of length N. */
typedef struct { const double *v0, *T, *s0, *a_max, *b, *delta; } orc_params;

static void load_theta(const double *const th6[6], int i, double th[6])
{
    for (int q = 0; q < 6; ++q) th[q] = th6[q][i];
}

/*
 * Forward simulation over K steps (Eq. 2, Eq. 3 and the bounds of
 * Sec. III-C).  Vehicles are stored lane by lane, lane head first, so that
 * the leader of vehicle i (when it is not the head of its lane) is i-1.
 *   lane_off[n_lanes+1] : CSR offsets of the lanes
 *   length[N]           : vehicle lengths
 *   th6[6][N]           : parameters (v0, T, s0, a_max, b, delta)
 *   P, V [(K+1) * N]    : output positions and speeds, time-major
 *   A    [K * N]        : output bounded accelerations a* (may be NULL)
 */
void orc_forward(int n_lanes, const int32_t *lane_off, const double *length,
                 const double *const th6[6], const double *p_init, const double *v_init,
                 int K, double dt, double a_min, double *P, double *V, double *A)
{
    const int N = lane_off[n_lanes];
    for (int i = 0; i < N; ++i) { P[i] = p_init[i]; V[i] = v_init[i]; }
    for (int k = 0; k < K; ++k) {
        const double *p = P + (size_t)k * N, *v = V + (size_t)k * N;
        double *pn = P + (size_t)(k + 1) * N, *vn = V + (size_t)(k + 1) * N;
        for (int l = 0; l < n_lanes; ++l) {
            for (int i = lane_off[l]; i < lane_off[l + 1]; ++i) {
                int has_leader = i > lane_off[l];
                double dp_raw = 0.0, vh = 0.0;
                if (has_leader) {
                    dp_raw = p[i - 1] - p[i] - length[i - 1];   /* Sec. III-A */
                    vh = v[i - 1];
                }
                double th[6];
                load_theta(th6, i, th);
                step_eval e = eval_vehicle(has_leader, v[i], dp_raw, vh, th, dt, a_min);
                if (A) A[(size_t)k * N + i] = e.a_star;
                pn[i] = p[i] + dt * v[i];                       /* Eq. 3, old speed */
                vn[i] = v[i] + dt * e.a_star;                   /* Eq. 3 */
            }
        }
    }
}

/*
 * Squared-error reconstruction loss (the squared-error form of the loss of
 * Sec. IV-A, summed over vehicles) and its seed dL/dP.
 *   targets[n_obs][N] with n_obs = floor(K / s): row j-1 is observed step j*s.
 *   Returns L = sum_i (1/n_obs) sum_j (P[j s][i] - targets[j-1][i])^2
 *   and writes gP[(K+1) * N] (zero where unobserved), when gP != NULL.
 */
double orc_mse_seed(int N, int K, const double *P, const double *targets, int s, double *gP)
{
    int n_obs = K / s;
    if (gP) memset(gP, 0, sizeof(double) * (size_t)(K + 1) * N);
    if (n_obs == 0) return 0.0;
    double L = 0.0;
    for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int j = 1; j <= n_obs; ++j) {
            int k = j * s;
            double r = P[(size_t)k * N + i] - targets[(size_t)(j - 1) * N + i];
            acc += r * r;
            if (gP) gP[(size_t)k * N + i] = 2.0 * r / n_obs;
        }
        L += acc / n_obs;
    }
    return L;
}

/*
 * Reverse-time adjoint of orc_forward.  With lp, lv the adjoints of the
 * step-(k+1) positions and speeds, mu_i = dt * lv_i and f the follower of i
 * (i+1 in the same lane), step k gives
 *   lp_k,i = gP_k,i + lp_i + mu_i dA_i/dp_i + mu_f dA_f/dp_h
 *   lv_k,i = gV_k,i + dt lp_i + lv_i + mu_i dA_i/dv_i + mu_f dA_f/dv_h
 *   g_theta_i += mu_i dA_i/dtheta_i
 * evaluated at the stored step-k state (P, V from orc_forward).
 *   gP, gV [(K+1) * N] : direct loss gradients (gV may be NULL)
 *   gth6[6][N]         : output parameter gradients (overwritten)
 *   g_p_init, g_v_init : output gradients w.r.t. the initial state
 */
void orc_adjoint(int n_lanes, const int32_t *lane_off, const double *length,
                 const double *const th6[6], int K, double dt, double a_min,
                 const double *P, const double *V, const double *gP, const double *gV,
                 double *const gth6[6], double *g_p_init, double *g_v_init)
{
    const int N = lane_off[n_lanes];
    double *lp = calloc((size_t)N, sizeof(double));
    double *lv = calloc((size_t)N, sizeof(double));
    double *nlp = calloc((size_t)N, sizeof(double));
    double *nlv = calloc((size_t)N, sizeof(double));
    step_eval *ev = calloc((size_t)N, sizeof(step_eval));
    int *has_leader = calloc((size_t)N, sizeof(int));
    for (int q = 0; q < 6; ++q) memset(gth6[q], 0, sizeof(double) * N);
    for (int l = 0; l < n_lanes; ++l)
        for (int i = lane_off[l]; i < lane_off[l + 1]; ++i) has_leader[i] = i > lane_off[l];

    for (int i = 0; i < N; ++i) {
        lp[i] = gP ? gP[(size_t)K * N + i] : 0.0;
        lv[i] = gV ? gV[(size_t)K * N + i] : 0.0;
    }
    for (int k = K - 1; k >= 0; --k) {
        const double *p = P + (size_t)k * N, *v = V + (size_t)k * N;
        for (int i = 0; i < N; ++i) {
            double dp_raw = 0.0, vh = 0.0;
            if (has_leader[i]) { dp_raw = p[i - 1] - p[i] - length[i - 1]; vh = v[i - 1]; }
            double th[6];
            load_theta(th6, i, th);
            ev[i] = eval_vehicle(has_leader[i], v[i], dp_raw, vh, th, dt, a_min);
        }
        for (int i = 0; i < N; ++i) {
            double mu = dt * lv[i];
            nlp[i] = lp[i] + mu * ev[i].d_p;
            nlv[i] = dt * lp[i] + lv[i] + mu * ev[i].d_v;
            for (int q = 0; q < 6; ++q) gth6[q][i] += mu * ev[i].d_th[q];
        }
        for (int i = 0; i < N; ++i) {
            if (!has_leader[i]) continue;
            double mu_f = dt * lv[i];          /* i is the follower of i-1 */
            nlp[i - 1] += mu_f * ev[i].d_ph;
            nlv[i - 1] += mu_f * ev[i].d_vh;
        }
        for (int i = 0; i < N; ++i) {
            lp[i] = nlp[i] + (gP ? gP[(size_t)k * N + i] : 0.0);
            lv[i] = nlv[i] + (gV ? gV[(size_t)k * N + i] : 0.0);
        }
    }
    for (int i = 0; i < N; ++i) {
        if (g_p_init) g_p_init[i] = lp[i];
        if (g_v_init) g_v_init[i] = lv[i];
    }
    free(lp); free(lv); free(nlp); free(nlv); free(ev); free(has_leader);
}

/*
 * One Adam step (Kingma & Ba, bias-corrected, no weight decay) on the five
 * optimised parameters of Sec. IV-A (v0, T, s0, a_max, b), followed by
 * projection onto the box [lo[q], hi[q]] (the constraint mechanism is not
 * stated in the paper; projection is this oracle's reading).  t >= 1.
 */
void orc_adam_step(int N, double *const th5[5], const double *const g5[5],
                   double *const m5[5], double *const v5[5], int t, double lr,
                   double beta1, double beta2, double eps, const double lo[5], const double hi[5])
{
    double bc1 = 1.0 - pow(beta1, t), bc2 = 1.0 - pow(beta2, t);
    for (int q = 0; q < 5; ++q) {
        for (int i = 0; i < N; ++i) {
            double g = g5[q][i];
            m5[q][i] = beta1 * m5[q][i] + (1.0 - beta1) * g;
            v5[q][i] = beta2 * v5[q][i] + (1.0 - beta2) * g * g;
            double mh = m5[q][i] / bc1, vh = v5[q][i] / bc2;
            double x = th5[q][i] - lr * mh / (sqrt(vh) + eps);
            if (x < lo[q]) x = lo[q];
            if (x > hi[q]) x = hi[q];
            th5[q][i] = x;
        }
    }
}

/* Learning rate of iteration it (0-based) out of n_iter: linear from lr0 to
 * lr1 (Sec. V-B). */
double orc_lr(int it, int n_iter, double lr0, double lr1)
{
    if (n_iter <= 1) return lr0;
    return lr0 + (lr1 - lr0) * (double)it / (double)(n_iter - 1);
}

/*
 * Gradient-based fit of Sec. IV-A: n_iter iterations of
 * {forward, squared-error loss, adjoint, Adam, projection}.  th6 is updated
 * in place (delta is never changed).  loss_hist[it] is the loss evaluated at
 * the parameters before update it.  Adam moments start at zero.
 */
void orc_fit(int n_lanes, const int32_t *lane_off, const double *length,
             double *const th6[6], const double *p_init, const double *v_init,
             int K, double dt, double a_min, const double *targets, int s,
             int n_iter, double lr0, double lr1, const double lo[5], const double hi[5],
             double *loss_hist)
{
    const int N = lane_off[n_lanes];
    size_t SN = (size_t)(K + 1) * N;
    double *P = malloc(sizeof(double) * SN), *V = malloc(sizeof(double) * SN);
    double *gP = malloc(sizeof(double) * SN);
    double *g[6], *m[5], *v2[5];
    for (int q = 0; q < 6; ++q) g[q] = calloc((size_t)N, sizeof(double));
    for (int q = 0; q < 5; ++q) { m[q] = calloc((size_t)N, sizeof(double)); v2[q] = calloc((size_t)N, sizeof(double)); }
    for (int it = 0; it < n_iter; ++it) {
        const double *cth[6];
        for (int q = 0; q < 6; ++q) cth[q] = th6[q];
        orc_forward(n_lanes, lane_off, length, cth, p_init, v_init, K, dt, a_min, P, V, NULL);
        loss_hist[it] = orc_mse_seed(N, K, P, targets, s, gP);
        orc_adjoint(n_lanes, lane_off, length, cth, K, dt, a_min, P, V, gP, NULL, g, NULL, NULL);
        const double *cg[5] = {g[0], g[1], g[2], g[3], g[4]};
        orc_adam_step(N, th6, cg, m, v2, it + 1, orc_lr(it, n_iter, lr0, lr1),
                      0.9, 0.999, 1e-8, lo, hi);
    }
    free(P); free(V); free(gP);
    for (int q = 0; q < 6; ++q) free(g[q]);
    for (int q = 0; q < 5; ++q) { free(m[q]); free(v2[q]); }
}

/*
 * Scene layout: order vehicles by (lane ascending, position descending,
 * original index ascending), so that each lane starts with its head and the
 * leader of a non-head vehicle is the vehicle before it (Sec. III-A, the
 * leader h(i) is the vehicle directly ahead in the same lane).
 *   perm[N]           : perm[j] = original index of the j-th sorted vehicle
 *   lane_off[n_lanes+1]: CSR offsets.  Returns 0, or -1 if a lane id is out
 *                       of [0, n_lanes).
 */
static const int32_t *g_lane;
static const double *g_pos;
static int cmp_vehicle(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (g_lane[i] != g_lane[j]) return g_lane[i] < g_lane[j] ? -1 : 1;
    if (g_pos[i] != g_pos[j]) return g_pos[i] > g_pos[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

int orc_layout(int N, int n_lanes, const int32_t *lane_id, const double *pos,
               int32_t *perm, int32_t *lane_off)
{
    for (int i = 0; i < N; ++i)
        if (lane_id[i] < 0 || lane_id[i] >= n_lanes) return -1;
    for (int i = 0; i < N; ++i) perm[i] = i;
    g_lane = lane_id;
    g_pos = pos;
    qsort(perm, (size_t)N, sizeof(int32_t), cmp_vehicle);
    for (int l = 0; l <= n_lanes; ++l) lane_off[l] = 0;
    for (int i = 0; i < N; ++i) lane_off[lane_id[i] + 1] += 1;
    for (int l = 0; l < n_lanes; ++l) lane_off[l + 1] += lane_off[l];
    return 0;
}
