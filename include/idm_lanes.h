/*
 * libidm -- lane geometry for training-free trajectory prediction
 * (arXiv 2412.16750, Sec. IV-B "Trajectory Prediction", Sec. V-C): agents'
 * 2-D positions are projected onto lane centre lines (polylines) to give the
 * 1-D positions the simulator works in, agents are assigned to the nearest
 * lane, fitted IDM rollouts are projected back onto the centre lines, and
 * the rollouts are scored by their displacement from the true positions.
 *
 * Lanes.  n_lanes polylines in one CSR: lane l has the points
 *   pt_off[l] .. pt_off[l+1]-1 (at least two, not all equal), coordinates
 *   px[], py[] (m).  lane_len[] (from idm_lane_prepare) holds the cumulative
 *   arc length at every point (0 at each lane's first point).
 *
 * Projection (definitions, also those of the test oracle): the projection
 *   of q onto a lane is its closest point: for every segment m with
 *   direction e = a_{m+1} - a_m (|e| > 0) the parameter t = clamp((q - a_m) .
 *   e / |e|^2, 0, 1) and the distance |q - a_m - t e|; the smallest distance
 *   wins (ties: the lower segment).  s = lane_len[m] + t |e|; d = the
 *   distance, positive to the left of the lane direction.  Assignment over a
 *   range of candidate lanes takes the smallest distance (ties: the lower
 *   lane index).  Back-projection of s: the point at arc length s on the
 *   centre line, continued along the first / last segment of positive
 *   length before 0 / beyond the end (no lateral offset: rollouts follow the
 *   centre line, Sec. V-C).
 *
 * Arrays are DEVICE memory owned by the caller; calls are asynchronous on
 * `stream`; a lane index outside [0, n_lanes) or a malformed pt_off sets
 * IDM_STATUS_BAD_LANES in the context's status word (idm_status then returns
 * IDM_ERR_LANES) and the affected outputs are NaN.  Arithmetic in FP32
 * (cumulative lengths summed in FP64).
 */
#ifndef IDM_LANES_H_
#define IDM_LANES_H_

#include <stdint.h>

#include "idm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define IDM_ERR_LANES 8
#define IDM_STATUS_BAD_LANES 32u

typedef struct {
    int32_t n_lanes;
    int32_t n_points;
    const int32_t *pt_off;    /* [n_lanes+1] */
    const float *px, *py;     /* [n_points] */
    const float *lane_len;    /* [n_points] cumulative arc length (idm_lane_prepare) */
} idm_lanes_t;

/* Cumulative arc length of every lane point into lane_len_out [n_points]. */
int idm_lane_prepare(idm_ctx_t *ctx, int32_t n_lanes, int32_t n_points, const int32_t *pt_off, const float *px,
                     const float *py, float *lane_len_out, void *stream);

/* Project the points (qx, qy) of an [n_rows][n_cols] row-major array (rows
 * = frames, columns = agents) onto lanes.  Point (r, c) is projected onto
 * every lane in [lane_lo[c], lane_hi[c]) and assigned to the nearest; with
 * lane_hi == NULL, onto the single lane lane_lo[c].  Outputs (same layout,
 * device, each may be NULL): lane_out (the chosen lane), s_out, d_out. */
int idm_lane_project(idm_ctx_t *ctx, const idm_lanes_t *lanes, int32_t n_rows, int32_t n_cols, const float *qx,
                     const float *qy, const int32_t *lane_lo, const int32_t *lane_hi, int32_t *lane_out,
                     float *s_out, float *d_out, void *stream);

/* Back-project: point j of rows x cols (row-major, [n_rows][n_cols]) lies at
 * arc length s[j] of lane lane_of_col[j % n_cols]; writes x_out, y_out
 * (same layout). */
int idm_lane_unproject(idm_ctx_t *ctx, const idm_lanes_t *lanes, int32_t n_rows, int32_t n_cols, const float *s,
                       const int32_t *lane_of_col, float *x_out, float *y_out, void *stream);

/* Rollout initial state from two rows a < b of a time-major [rows][N]
 * array of arc lengths: p = s[b], v = max((s[b] - s[a]) / ((b - a) dt), 0). */
int idm_rollout_state(idm_ctx_t *ctx, int32_t N, const float *s_rows, int32_t row_a, int32_t row_b, float dt,
                      float *p_out, float *v_out, void *stream);

/* Displacement of F predicted frames from the truth, time-major [F][N]
 * (x and y arrays): per agent ade[i] = mean_f |pred_f - true_f|, fde[i] =
 * |pred_F - true_F| (device out [N], may be NULL); sums (device, double [3],
 * may be NULL) = (sum ade, sum fde, number of agents with fde > miss_m). */
int idm_displacement(idm_ctx_t *ctx, int32_t F, int32_t N, const float *px, const float *py, const float *tx,
                     const float *ty, float miss_m, float *ade, float *fde, double *sums, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IDM_LANES_H_ */
