// Lane geometry of the training-free prediction (arXiv 2412.16750, Sec. IV-B,
// Sec. V-C): polyline projection and lane assignment, back-projection of
// 1-D rollouts onto the centre line, rollout initial state, displacement
// metrics.  Definitions in include/idm_lanes.h.
//
// Projection runs one warp per query point: the warp's lanes stride over the
// segments of the candidate lanes (a scenario's polylines are shared by all
// its agents and stay in L1/L2), each keeps its nearest segment, and a
// lexicographic warp reduction (distance, lane, segment) picks the winner, so
// the tie rule of the definition holds whatever the stride.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include "../../include/idm.h"
#include "../../include/idm_lanes.h"
#include "idm_ctx.h"

namespace idm {
namespace lanes {

constexpr unsigned FULL = 0xffffffffu;

__global__ void prepare_kernel(int n_lanes, int n_points, const int32_t *off, const float *px, const float *py,
                               float *cum, unsigned *status)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lanes) return;
    const int p0 = off[l], p1 = off[l + 1];
    if (p0 < 0 || p1 > n_points || p1 - p0 < 2) {
        atomicOr(status, IDM_STATUS_BAD_LANES);
        return;
    }
    double c = 0.0;
    cum[p0] = 0.0f;
    for (int m = p0; m + 1 < p1; ++m) {
        const double dx = (double)px[m + 1] - (double)px[m], dy = (double)py[m + 1] - (double)py[m];
        c += sqrt(dx * dx + dy * dy);
        cum[m + 1] = (float)c;
    }
    if (!(c > 0.0)) atomicOr(status, IDM_STATUS_BAD_LANES);
}

struct Best {
    float d2;
    int lane, seg;
    float t;
};

// a better than b: smaller distance, then lower lane, then lower segment
__device__ __forceinline__ bool better(const Best &a, const Best &b)
{
    if (a.d2 != b.d2) return a.d2 < b.d2;
    if (a.lane != b.lane) return a.lane < b.lane;
    return a.seg < b.seg;
}

__global__ void project_kernel(idm_lanes_t L, long long n_q, int n_cols, const float *qx, const float *qy,
                               const int32_t *lo, const int32_t *hi, int32_t *lane_out, float *s_out, float *d_out,
                               unsigned *status)
{
    const long long j = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (j >= n_q) return;   // warp-uniform
    const float x = qx[j], y = qy[j];
    const int col = (int)(j % n_cols);
    int l0 = lo[col];
    int l1 = hi ? hi[col] : l0 + 1;
    Best b{INFINITY, 0x7fffffff, 0x7fffffff, 0.0f};
    const bool bad = l0 < 0 || l1 > L.n_lanes || l0 >= l1;
    if (!bad) {
        for (int l = l0; l < l1; ++l) {
            const int p0 = L.pt_off[l], p1 = L.pt_off[l + 1];
            for (int m = p0 + lane; m + 1 < p1; m += 32) {
                const float ax = L.px[m], ay = L.py[m];
                const float ex = L.px[m + 1] - ax, ey = L.py[m + 1] - ay;
                const float e2 = ex * ex + ey * ey;
                if (e2 == 0.0f) continue;
                const float qxa = x - ax, qya = y - ay;
                const float t = fminf(fmaxf((qxa * ex + qya * ey) / e2, 0.0f), 1.0f);
                const float fx = qxa - t * ex, fy = qya - t * ey;
                const Best c{fx * fx + fy * fy, l, m, t};
                if (better(c, b)) b = c;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best c;
        c.d2 = __shfl_xor_sync(FULL, b.d2, o);
        c.lane = __shfl_xor_sync(FULL, b.lane, o);
        c.seg = __shfl_xor_sync(FULL, b.seg, o);
        c.t = __shfl_xor_sync(FULL, b.t, o);
        if (better(c, b)) b = c;
    }
    if (lane != 0) return;
    if (bad || b.lane == 0x7fffffff) {
        atomicOr(status, IDM_STATUS_BAD_LANES);
        if (lane_out) lane_out[j] = -1;
        if (s_out) s_out[j] = NAN;
        if (d_out) d_out[j] = NAN;
        return;
    }
    const int m = b.seg;
    const float ax = L.px[m], ay = L.py[m];
    const float ex = L.px[m + 1] - ax, ey = L.py[m + 1] - ay;
    const float dist = sqrtf(b.d2);
    const float cross = ex * (y - ay) - ey * (x - ax);
    if (lane_out) lane_out[j] = b.lane;
    if (s_out) s_out[j] = L.lane_len[m] + b.t * sqrtf(ex * ex + ey * ey);
    if (d_out) d_out[j] = cross >= 0.0f ? dist : -dist;
}

__global__ void unproject_kernel(idm_lanes_t L, int n_rows, int n_cols, const float *s, const int32_t *lane_of_col,
                                 float *x_out, float *y_out, unsigned *status)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)n_rows * n_cols) return;
    const int l = lane_of_col[j % n_cols];
    if (l < 0 || l >= L.n_lanes) {
        atomicOr(status, IDM_STATUS_BAD_LANES);
        x_out[j] = NAN;
        y_out[j] = NAN;
        return;
    }
    const int p0 = L.pt_off[l], p1 = L.pt_off[l + 1];
    const float *c = L.lane_len;
    const float sj = s[j];
    int m;
    if (sj <= 0.0f) {
        m = p0;
        while (m + 2 < p1 && !(c[m + 1] > c[m])) ++m;      // first segment of positive length
    } else if (sj >= c[p1 - 1]) {
        m = p1 - 2;
        while (m > p0 && !(c[m + 1] > c[m])) --m;          // last segment of positive length
    } else {
        int a = p0, b = p1 - 1;                            // largest m with c[m] <= s
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (c[mid] <= sj)
                a = mid;
            else
                b = mid - 1;
        }
        m = a;
    }
    const float len = c[m + 1] - c[m];
    const float f = len > 0.0f ? (sj - c[m]) / len : 0.0f;
    x_out[j] = L.px[m] + f * (L.px[m + 1] - L.px[m]);
    y_out[j] = L.py[m] + f * (L.py[m + 1] - L.py[m]);
}

__global__ void rollout_state_kernel(int N, const float *s, int ra, int rb, float inv_span, float *p, float *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float sb = s[(size_t)rb * N + i], sa = s[(size_t)ra * N + i];
    p[i] = sb;
    v[i] = fmaxf((sb - sa) * inv_span, 0.0f);
}

__global__ void displacement_kernel(int F, int N, const float *px, const float *py, const float *tx, const float *ty,
                                    float miss, float *ade, float *fde, double *sums)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, fd = 0.0, ms = 0.0;
    if (i < N) {
        float e = 0.0f;
        for (int f = 0; f < F; ++f) {
            const size_t o = (size_t)f * N + i;
            const float dx = px[o] - tx[o], dy = py[o] - ty[o];
            e = sqrtf(dx * dx + dy * dy);
            a += e;
        }
        a /= F;
        fd = e;
        ms = e > miss ? 1.0 : 0.0;
        if (ade) ade[i] = (float)a;
        if (fde) fde[i] = e;
    }
    if (sums) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(FULL, a, o);
            fd += __shfl_xor_sync(FULL, fd, o);
            ms += __shfl_xor_sync(FULL, ms, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(sums, a);
            atomicAdd(sums + 1, fd);
            atomicAdd(sums + 2, ms);
        }
    }
}

}  // namespace lanes
}  // namespace idm

using namespace idm::abi;

namespace {

int check_lanes(idm_ctx *c, const idm_lanes_t *L)
{
    if (!L) return fail(c, IDM_ERR_ARG, "lanes is NULL");
    if (L->n_lanes < 1 || L->n_points < 2) return fail(c, IDM_ERR_ARG, "need >= 1 lane and >= 2 points");
    if (!L->pt_off || !L->px || !L->py || !L->lane_len) return fail(c, IDM_ERR_ARG, "a lane array is NULL");
    return IDM_OK;
}

}  // namespace

extern "C" int idm_lane_prepare(idm_ctx_t *c, int32_t n_lanes, int32_t n_points, const int32_t *pt_off,
                                const float *px, const float *py, float *lane_len_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (n_lanes < 1 || n_points < 2) return fail(c, IDM_ERR_ARG, "need >= 1 lane and >= 2 points");
    if (!pt_off || !px || !py || !lane_len_out) return fail(c, IDM_ERR_ARG, "a lane array is NULL");
    int rc;
    if ((rc = ensure_status(c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    idm::lanes::prepare_kernel<<<(n_lanes + 127) / 128, 128, 0, st>>>(n_lanes, n_points, pt_off, px, py,
                                                                       lane_len_out, (unsigned *)c->status.p);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}

extern "C" int idm_lane_project(idm_ctx_t *c, const idm_lanes_t *L, int32_t n_rows, int32_t n_cols, const float *qx,
                                const float *qy, const int32_t *lane_lo, const int32_t *lane_hi, int32_t *lane_out,
                                float *s_out, float *d_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_lanes(c, L))) return rc;
    if (n_rows < 0 || n_cols < 0) return fail(c, IDM_ERR_ARG, "n_rows and n_cols must be >= 0");
    const long long n_q = (long long)n_rows * n_cols;
    if (n_q > 0 && (!qx || !qy || !lane_lo)) return fail(c, IDM_ERR_ARG, "qx, qy and lane_lo must be given");
    if ((rc = ensure_status(c))) return rc;
    if (n_q == 0) return IDM_OK;
    const int wpb = 8;
    const long long blocks = (n_q + wpb - 1) / wpb;
    if (blocks > 2147483647LL) return fail(c, IDM_ERR_ARG, "n_q too large");
    idm::lanes::project_kernel<<<(unsigned)blocks, 32 * wpb, 0, (cudaStream_t)stream>>>(
        *L, n_q, n_cols, qx, qy, lane_lo, lane_hi, lane_out, s_out, d_out, (unsigned *)c->status.p);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}

extern "C" int idm_lane_unproject(idm_ctx_t *c, const idm_lanes_t *L, int32_t n_rows, int32_t n_cols, const float *s,
                                  const int32_t *lane_of_col, float *x_out, float *y_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_lanes(c, L))) return rc;
    if (n_rows < 0 || n_cols < 0) return fail(c, IDM_ERR_ARG, "n_rows and n_cols must be >= 0");
    const long long n = (long long)n_rows * n_cols;
    if (n > 0 && (!s || !lane_of_col || !x_out || !y_out)) return fail(c, IDM_ERR_ARG, "an array is NULL");
    if ((rc = ensure_status(c))) return rc;
    if (n == 0) return IDM_OK;
    idm::lanes::unproject_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        *L, n_rows, n_cols, s, lane_of_col, x_out, y_out, (unsigned *)c->status.p);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}

extern "C" int idm_rollout_state(idm_ctx_t *c, int32_t N, const float *s_rows, int32_t row_a, int32_t row_b, float dt,
                                 float *p_out, float *v_out, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (N < 0 || row_a < 0 || row_b <= row_a) return fail(c, IDM_ERR_ARG, "need N >= 0 and 0 <= row_a < row_b");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(c, IDM_ERR_ARG, "dt must be finite and > 0");
    if (N > 0 && (!s_rows || !p_out || !v_out)) return fail(c, IDM_ERR_ARG, "an array is NULL");
    if (N == 0) return IDM_OK;
    idm::lanes::rollout_state_kernel<<<(N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        N, s_rows, row_a, row_b, 1.0f / ((float)(row_b - row_a) * dt), p_out, v_out);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}

extern "C" int idm_displacement(idm_ctx_t *c, int32_t F, int32_t N, const float *px, const float *py, const float *tx,
                                const float *ty, float miss_m, float *ade, float *fde, double *sums, void *stream)
{
    if (!c) return IDM_ERR_ARG;
    if (F < 1 || N < 0) return fail(c, IDM_ERR_ARG, "need F >= 1 and N >= 0");
    if (N > 0 && (!px || !py || !tx || !ty)) return fail(c, IDM_ERR_ARG, "an array is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (sums) IDM_CK(cudaMemsetAsync(sums, 0, sizeof(double) * 3, st));
    if (N == 0) return IDM_OK;
    idm::lanes::displacement_kernel<<<(N + 255) / 256, 256, 0, st>>>(F, N, px, py, tx, ty, miss_m, ade, fde, sums);
    IDM_CK(cudaGetLastError());
    return IDM_OK;
}
