// Scene layout for libidm: order vehicles lane by lane, head first
// (Sec. III-A of arXiv 2412.16750: the leader h(i) is the vehicle directly
// ahead in the same lane), so that the leader of a non-head vehicle is the
// vehicle before it.
//
// Steps: count vehicles per lane (atomics), exclusive scan into lane_off,
// bucket each vehicle into its lane (atomic cursor; order within a lane is
// arbitrary here), then sort every lane by the unique key
// (position descending, original index ascending) with a bitonic sort in
// shared memory, one block per lane.  The result is deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "idm_device.cuh"
#include "idm_internal.h"

namespace idm {

constexpr int LAYOUT_MAX_LANE = 4096;

__global__ void count_kernel(int N, int n_lanes, const int32_t *lane_id, int *counts, unsigned *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int l = lane_id[i];
    if (l < 0 || l >= n_lanes) { atomicOr(status, IDM_STATUS_BAD_LANE_OFF); return; }
    atomicAdd(&counts[l], 1);
}

// Single-block exclusive scan of counts into lane_off, plus the longest lane.
__global__ void __launch_bounds__(1024)
scan_kernel(int n_lanes, const int *counts, int32_t *lane_off, int32_t *max_lane, int *cursor, unsigned *status)
{
    __shared__ int sc[1024];
    __shared__ int mx[1024];
    const int t = threadIdx.x;
    const int per = (n_lanes + 1023) / 1024;
    const int l0 = min(n_lanes, t * per), l1 = min(n_lanes, l0 + per);
    int s = 0, m = 0;
    for (int l = l0; l < l1; ++l) { s += counts[l]; m = max(m, counts[l]); }
    sc[t] = s;
    mx[t] = m;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? sc[t - off] : 0;
        int w = t >= off ? mx[t - off] : 0;
        __syncthreads();
        sc[t] += v;
        mx[t] = max(mx[t], w);
        __syncthreads();
    }
    int run = sc[t] - s;
    for (int l = l0; l < l1; ++l) {
        lane_off[l] = run;
        cursor[l] = run;
        run += counts[l];
    }
    if (t == 1023) {
        lane_off[n_lanes] = sc[t];
        if (max_lane) *max_lane = mx[t];
        if (mx[t] > LAYOUT_MAX_LANE) atomicOr(status, IDM_STATUS_LANE_TOO_LONG);
    }
}

__global__ void bucket_kernel(int N, int n_lanes, const int32_t *lane_id, int *cursor, int32_t *perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int l = lane_id[i];
    if (l < 0 || l >= n_lanes) return;
    int pos = atomicAdd(&cursor[l], 1);
    perm[pos] = i;
}

// Order-preserving map of a float to uint32 (ascending); -0 and +0 map alike.
__device__ __forceinline__ uint32_t float_key(float x)
{
    if (x == 0.0f) x = 0.0f;
    uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(256)
lane_sort_kernel(int n_lanes, const int32_t *lane_off, const float *pos, int32_t *perm)
{
    __shared__ unsigned long long key[LAYOUT_MAX_LANE];
    const int l = blockIdx.x;
    if (l >= n_lanes) return;
    const int a = lane_off[l], n = lane_off[l + 1] - a;
    if (n <= 1 || n > LAYOUT_MAX_LANE) return;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < n) {
            int idx = perm[a + i];
            // descending position = ascending of the complemented key
            uint32_t kp = ~float_key(pos[idx]);
            key[i] = ((unsigned long long)kp << 32) | (uint32_t)idx;
        } else {
            key[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    unsigned long long x = key[i], y = key[j];
                    if ((x > y) == up) { key[i] = y; key[j] = x; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[a + i] = (int32_t)(key[i] & 0xffffffffu);
}

cudaError_t launch_layout(int N, int n_lanes, const int32_t *lane_id, const float *pos, int32_t *perm,
                          int32_t *lane_off, int32_t *max_lane, int *counts, int *cursor, unsigned *status,
                          cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)n_lanes, st);
    if (e != cudaSuccess) return e;
    if (N > 0) count_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, n_lanes, lane_id, counts, status);
    scan_kernel<<<1, 1024, 0, st>>>(n_lanes, counts, lane_off, max_lane, cursor, status);
    if (N > 0) bucket_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, n_lanes, lane_id, cursor, perm);
    if (n_lanes > 0) lane_sort_kernel<<<n_lanes, 256, 0, st>>>(n_lanes, lane_off, pos, perm);
    return cudaGetLastError();
}

constexpr int GATHER_MAX = 16;
struct GatherPtrs {
    const float *src[GATHER_MAX];
    float *dst[GATHER_MAX];
};

__global__ void gather_kernel(int N, const int32_t *perm, int count, GatherPtrs p)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int s = perm[i];
    for (int c = 0; c < count; ++c) p.dst[c][i] = p.src[c][s];
}

cudaError_t launch_gather(int N, const int32_t *perm, int count, const float *const *srcs, float *const *dsts,
                          cudaStream_t st)
{
    for (int base = 0; base < count; base += GATHER_MAX) {
        GatherPtrs p;
        int c = count - base < GATHER_MAX ? count - base : GATHER_MAX;
        for (int q = 0; q < c; ++q) { p.src[q] = srcs[base + q]; p.dst[q] = dsts[base + q]; }
        if (N > 0) gather_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, perm, c, p);
    }
    return cudaGetLastError();
}

// dst[r][j] = src[r][perm[j]] for a row-major [n_rows][N] matrix (columns
// are vehicles): coalesced writes, gathered reads.
// dst[r][j] = src[r][perm[j]] over the flattened [n_rows][N] index space:
// block b covers elements [b * ROWS_CHUNK, (b + 1) * ROWS_CHUNK), so the blocks
// resident at any time (dispatched in index order) work on one or two rows.
// The random reads of a row then hit its copy in L2 (each 32-byte sector is
// fetched from DRAM once and serves all eight of its elements) instead of
// fetching a sector per element, and perm stays in L2 across rows.  Each
// thread takes GR_PER elements and issues all their loads before its stores,
// so the random reads overlap instead of waiting one by one.
constexpr int GR_PER = 8;
constexpr int ROWS_CHUNK = 256 * GR_PER;

__global__ void __launch_bounds__(256) gather_rows_kernel(int N, long long total, const int32_t *__restrict__ perm,
                                                          const float *__restrict__ src, float *__restrict__ dst)
{
    const long long base = (long long)blockIdx.x * ROWS_CHUNK;
    long long r = base / N;
    int j = (int)(base - r * N) + (int)threadIdx.x;
    size_t at[GR_PER];
    int col[GR_PER];
    bool ok[GR_PER];
#pragma unroll
    for (int e = 0; e < GR_PER; ++e, j += 256) {
        while (j >= N) {
            j -= N;
            ++r;
        }
        ok[e] = base + (long long)(e * 256 + (int)threadIdx.x) < total;
        at[e] = (size_t)r * (size_t)N;
        col[e] = j;
    }
    int sj[GR_PER];
#pragma unroll
    for (int e = 0; e < GR_PER; ++e) sj[e] = ok[e] ? __ldg(perm + col[e]) : 0;
    float v[GR_PER];
#pragma unroll
    for (int e = 0; e < GR_PER; ++e) v[e] = ok[e] ? __ldg(src + at[e] + sj[e]) : 0.0f;
#pragma unroll
    for (int e = 0; e < GR_PER; ++e)
        if (ok[e]) dst[at[e] + col[e]] = v[e];
}

cudaError_t launch_gather_rows(int N, int n_rows, const int32_t *perm, const float *src, float *dst, cudaStream_t st)
{
    if (N > 0 && n_rows > 0) {
        const long long total = (long long)N * n_rows;
        const long long blocks = (total + ROWS_CHUNK - 1) / ROWS_CHUNK;
        gather_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(N, total, perm, src, dst);
    }
    return cudaGetLastError();
}

}  // namespace idm
