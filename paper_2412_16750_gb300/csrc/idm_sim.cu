// Simulation kernels of libidm for sm_103a: initial gaps, lane packing into
// segments, the fused forward (Eq. 1-3 with the Sec. III-C bounds,
// checkpoints, optional trajectory output) and the launch / dispatch code of
// the reverse-time adjoint, whose kernels live in idm_adjoint.cuh
// (arXiv 2412.16750, Sec. III and IV-A).
//
// Mapping.  Vehicles are ordered lane by lane, head first.  Whole lanes are
// packed into segments of at most 32*VPT*G vehicles, each run by G warps of
// one block.  Thread l of a warp holds pairs of adjacent slots (pair p:
// slots 64p + 2l and 64p + 2l + 1), so the leader of a pair's second slot is
// in the same register pair and the leader of its first slot is one warp
// shuffle away; across warps the value goes through shared cells and one
// named barrier per step.  Groups take segments from a global atomic counter
// (persistent grid).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idm_forward.cuh"

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
constexpr int BUILD_THREADS = SEG_BUILD_CHUNKS;

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

// The losses of all iterations of a single-launch fit: block it sums the
// partials of iteration it in the order of loss_finalize_kernel, so each
// value equals that of the per-iteration reduction.
__global__ void __launch_bounds__(1024)
loss_finalize_iters_kernel(const double *part, long long stride, const int *n_seg, int per_seg, double *out)
{
    __shared__ double sh[1024];
    const long long n = (long long)*n_seg * per_seg;
    if (n > stride) {  // flagged by the fit kernel
        if (threadIdx.x == 0) out[blockIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const double *pi = part + (size_t)blockIdx.x * (size_t)stride;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += pi[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

cudaError_t launch_loss_finalize_iters(const double *loss_part, long long stride, const int *n_seg, int per_seg,
                                       int n_iter, double *out, cudaStream_t st)
{
    if (n_iter < 1) return cudaSuccess;
    loss_finalize_iters_kernel<<<n_iter, 1024, 0, st>>>(loss_part, stride, n_seg, per_seg, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
// Forward kernels of every shape live in idm_shape_v<V>_g<G>.cu (COUNT: the
// variant that also counts gap-floor and kink-band events).
static void *forward_fn_v(int vpt, int G, bool count)
{
#define IDM_PICK(V, GW) \
    if (vpt == V && G == GW) return forward_fn_v##V##_g##GW(count);
    IDM_SHAPES(IDM_PICK)
#undef IDM_PICK
    return nullptr;
}

cudaError_t launch_forward(int vpt, int G, bool traj, bool vtraj, bool ckpt, const SimArgs &a, int grid, int wpb,
                           cudaStream_t st)
{
    FwdFlags f{traj, vtraj, ckpt, a.eval_targets != nullptr && a.eval_part != nullptr};
    void *fn = forward_fn_v(vpt, G, a.events != nullptr);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = forward_smem_bytes(vpt, G, wpb);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SimArgs args = a;
    args.G = G;
    void *params[] = {&args, &f};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * wpb), params, smem, st);
}

size_t backward_smem_bytes(int vpt, bool dense_seed, int T, int G, int wpb, bool prefetch)
{
    return (size_t)bwd_group_floats(vpt, dense_seed, T, G, prefetch) * (wpb / G) * sizeof(float);
}

size_t forward_smem_bytes(int vpt, int G, int wpb)
{
    (void)vpt;
    return (size_t)grp_ctrl_floats(G) * (wpb / G) * sizeof(float);
}

// Adjoint variants of every shape live in idm_shape_v<V>_g<G>.cu (with
// 4 vehicles per thread, segments of up to 4 warps run in 4-warp blocks and
// 8-warp segments in 8-warp blocks); SUB: tape shallower than the checkpoint
// interval.
static void *backward_fn_v(int vpt, int G, bool dense, bool adam, bool wd, bool sub)
{
#define IDM_PICK(V, GW) \
    if (vpt == V && G == GW) return backward_fn_v##V##_g##GW(dense, adam, wd, sub);
    IDM_SHAPES(IDM_PICK)
#undef IDM_PICK
    return nullptr;
}

int backward_max_warps(int vpt, int G) { return (vpt == 4 && G <= 4) ? 4 : 8; }

int backward_resident_warps(int vpt, int G)
{
    if (vpt == 2) return 16;
    if (vpt == 4 && G <= 4) return 12;
    return 8;
}

cudaError_t launch_backward(int vpt, int G, bool dense_seed, bool adam, bool want_delta, const SimArgs &a, int grid,
                            int wpb, cudaStream_t st)
{
    if (dense_seed && adam) return cudaErrorInvalidValue;
    if (wpb > backward_max_warps(vpt, G) || wpb % G) return cudaErrorInvalidValue;
    void *fn = backward_fn_v(vpt, G, dense_seed, adam, want_delta && !adam, a.tape_T < a.C);
    if (!fn) return cudaErrorInvalidValue;
    size_t smem = backward_smem_bytes(vpt, dense_seed, a.tape_T, G, wpb, a.bwd_pf != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SimArgs args = a;
    args.G = G;
    void *params[] = {&args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * wpb), params, smem, st);
}

// Single-launch fit kernels of every shape live in idm_shape_v<V>_g<G>.cu.
static void *fused_fn_v(int vpt, int G, bool sub)
{
#define IDM_PICK(V, GW) \
    if (vpt == V && G == GW) return fused_fn_v##V##_g##GW(sub);
    IDM_SHAPES(IDM_PICK)
#undef IDM_PICK
    return nullptr;
}

cudaError_t launch_fit_fused(int vpt, int G, const SimArgs &a, long long part_stride, int grid, int wpb,
                             cudaStream_t st)
{
    if (wpb > backward_max_warps(vpt, G) || wpb % G) return cudaErrorInvalidValue;
    void *fn = fused_fn_v(vpt, G, a.tape_T < a.C);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = backward_smem_bytes(vpt, false, a.tape_T, G, wpb, a.bwd_pf != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * wpb, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int cap = n_sm * (occ > 0 ? occ : 1);
    SimArgs args = a;
    args.G = G;
    long long stride = part_stride;
    void *params[] = {&args, &stride};
    return cudaLaunchKernel(fn, dim3(grid < cap ? grid : cap), dim3(32 * wpb), params, smem, st);
}

int occupancy_blocks(int vpt, int G, bool backward, bool dense, bool adam, bool want_delta, int wpb, size_t smem,
                     bool sub)
{
    void *fn = nullptr;
    if (!backward) {
        fn = forward_fn_v(vpt, G, false);
        smem = forward_smem_bytes(vpt, G, wpb);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
        fn = backward_fn_v(vpt, G, dense, adam, want_delta && !adam, sub);
        if (fn) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (!fn) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * wpb, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace idm
