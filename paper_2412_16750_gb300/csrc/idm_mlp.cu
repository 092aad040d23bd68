// Learned initializer: feature extraction, the BF16 tensor-core GEMM with
// fused epilogues, and the training / inference drivers of the 80-256-256-
// 256-5 GELU network declared in idm_mlp.h.
//
// Training step for a batch of B rows (B padded to Bp, a multiple of 128;
// padded rows are zeros and carry no gradient):
//   forward   Z_l = H_{l-1} W_l^T + b_l, H_l = gelu(Z_l) (l = 1..3), stored
//             as Z_l (FP32), H_l and H_l^T (bf16); O = H_3 W_4^T + b_4;
//   loss      S = sigmoid(O), L = sum (S - label)^2 / (5 B), and
//             dO = 2 (S - label) S (1 - S) / (5 B) as dO and dO^T (bf16),
//             all in the epilogue of the last GEMM;
//   backward  dZ_l = (dZ_{l+1} W_{l+1}) * gelu'(Z_l) in the epilogue of the
//             GEMM against W^T (bf16 copies kept transposed), as dZ_l and
//             dZ_l^T;  dW_l = dZ_l^T H_{l-1} as split-K FP32 partials
//             (operands transposed so that K = batch is contiguous);
//             db_l = column sums of dZ_l;
//   update    one kernel sums the partials and applies Adam to the FP32
//             master weights, then refreshes the bf16 copies W and W^T.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "../../include/idm.h"
#include "../../include/idm_mlp.h"
#include "idm_device.cuh"
#include "idm_gemm_tc.cuh"

namespace idm {
namespace mlp {

using bf16 = __nv_bfloat16;

constexpr int IN = IDM_MLP_IN, HID = IDM_MLP_HIDDEN, OUT = IDM_MLP_OUT, OUTP = 16, PREFIX = IDM_MLP_PREFIX;
// flat parameter offsets
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID,
              OFF_B4 = OFF_W4 + OUT * HID, NPARAM = OFF_B4 + OUT;
static_assert(NPARAM == IDM_MLP_N_PARAMS, "parameter count");

enum Mode { GELU_FWD = 0, OUT_TRAIN = 1, OUT_INFER = 2, DGELU = 3, F32_PART = 4 };

struct GemmArgs {
    const bf16 *A, *B;
    int M_valid;     // rows of A holding data (later rows read as zeros)
    int M_rows;      // rows of the outputs (stores skip rows >= M_rows)
    int N, K, BN, k_chunk;
    const float *bias;   // [N] (GELU_FWD, OUT_*)
    float *Z;            // [M_rows][N] FP32: written (GELU_FWD) or read (DGELU)
    bf16 *H, *HT;        // [M_rows][N] and [N][ldt] bf16 outputs (may be NULL)
    int ldt;
    float *Cf;           // [splits][M_rows][N] FP32 partials (F32_PART)
    const float *label;  // [M_valid][5] (OUT_TRAIN)
    double *loss_part;   // [gridDim.x * 4] (OUT_TRAIN)
    float scale;         // 1 / (5 B) (OUT_TRAIN)
    float *out[OUT];     // OUT_INFER: parameter arrays; else out[0] = [M_valid][5] sigmoid outputs or NULL
    float lo[OUT], hi[OUT];
    unsigned *status;
    int stages;          // A stages of the persistent kernel
    unsigned wait_iters; // polls per tensor-core wait before giving up (tc::WAIT_ITERS normally)
};

// Normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2 and density phi(z) with erf
// from Abramowitz & Stegun, Handbook of Mathematical Functions, formula
// 7.1.26: for x >= 0, erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// exp(-x^2) with t = 1 / (1 + p x), |error| <= 1.5e-7; odd in x.  The
// exponential exp(-x^2) = exp(-z^2 / 2) is shared with phi.
struct NormalCdf {
    float cdf, pdf;
};
__device__ __forceinline__ NormalCdf normal_cdf(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = idm::rcp_approx(fmaf(0.3275911f, x, 1.0f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    const float e = idm::ex2_approx(-x * x * 1.44269504088896341f);  // exp(-x^2)
    const float half_tail = 0.5f * t * poly * e;            // (1 - erf(x)) / 2
    NormalCdf r;
    r.cdf = z >= 0.0f ? 1.0f - half_tail : half_tail;
    r.pdf = 0.39894228040143268f * e;
    return r;
}

// The same arithmetic for two values at once with the packed FP32
// instructions (every product and fused multiply-add rounds as its scalar
// counterpart, so the results equal normal_cdf's bit for bit).
struct NormalCdf2 {
    float2 cdf, pdf;
};
__device__ __forceinline__ NormalCdf2 normal_cdf2(float2 z)
{
    using idm::F2;
    using idm::fma2;
    using idm::mul2;
    const float2 x = make_float2(fabsf(z.x) * 0.70710678118654752f, fabsf(z.y) * 0.70710678118654752f);
    const float2 den = fma2(F2(0.3275911f), x, F2(1.0f));
    const float2 t = make_float2(idm::rcp_approx(den.x), idm::rcp_approx(den.y));
    float2 poly = fma2(t, F2(1.061405429f), F2(-1.453152027f));
    poly = fma2(t, poly, F2(1.421413741f));
    poly = fma2(t, poly, F2(-0.284496736f));
    poly = fma2(t, poly, F2(0.254829592f));
    const float2 arg = mul2(mul2(make_float2(-x.x, -x.y), x), F2(1.44269504088896341f));
    const float2 e = make_float2(idm::ex2_approx(arg.x), idm::ex2_approx(arg.y));  // exp(-x^2)
    const float2 half_tail = mul2(mul2(mul2(F2(0.5f), t), poly), e);            // (1 - erf(x)) / 2
    const float2 upper = idm::sub2(F2(1.0f), half_tail);
    NormalCdf2 r;
    r.cdf = make_float2(z.x >= 0.0f ? upper.x : half_tail.x, z.y >= 0.0f ? upper.y : half_tail.y);
    r.pdf = mul2(F2(0.39894228040143268f), e);
    return r;
}

__device__ __forceinline__ float gelu(float z) { return z * normal_cdf(z).cdf; }
__device__ __forceinline__ float gelu_grad(float z)
{
    const NormalCdf n = normal_cdf(z);
    return fmaf(z, n.pdf, n.cdf);
}

__global__ void gelu_eval_kernel(const float *z, float *g, float *dg, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (g) g[i] = gelu(z[i]);
    if (dg) dg[i] = gelu_grad(z[i]);
}
__device__ __forceinline__ float sigmoid(float o) { return 1.0f / (1.0f + expf(-o)); }

__device__ __forceinline__ void store16_bf16(bf16 *dst, const float (&h)[16])
{
    __align__(16) bf16 tmp[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) tmp[i] = __float2bfloat16_rn(h[i]);
    reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(tmp)[0];
    reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(tmp)[1];
}

__device__ __forceinline__ void store16_f32(float *dst, const float (&v)[16])
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
        reinterpret_cast<float4 *>(dst)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// 16 accumulator columns [n, n + 16) of row r after the tensor-memory load.
template <int MODE>
__device__ __forceinline__ void epilogue_chunk(const GemmArgs &g, int r, int n, int split, const float *bias,
                                               float (&v)[16])
{
    const bool row_ok = r < g.M_rows;
    if (MODE == F32_PART) {
        if (row_ok) store16_f32(g.Cf + ((size_t)split * g.M_rows + r) * g.N + n, v);
        return;
    }
    float h[16];
    if (MODE == GELU_FWD) {
        const float4 *b4 = reinterpret_cast<const float4 *>(bias + n);  // 16-byte aligned (n % 16 == 0)
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            const float4 bq = b4[i / 4];
            const float2 z0 = idm::add2(make_float2(v[i], v[i + 1]), make_float2(bq.x, bq.y));
            const float2 z1 = idm::add2(make_float2(v[i + 2], v[i + 3]), make_float2(bq.z, bq.w));
            v[i] = z0.x;
            v[i + 1] = z0.y;
            v[i + 2] = z1.x;
            v[i + 3] = z1.y;
        }
        if (g.Z && row_ok) store16_f32(g.Z + (size_t)r * g.N + n, v);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const float2 zz = make_float2(v[i], v[i + 1]);
            const float2 gg = idm::mul2(zz, normal_cdf2(zz).cdf);
            h[i] = gg.x;
            h[i + 1] = gg.y;
        }
    } else {  // DGELU
        float z[16];
        if (row_ok) {
            const float4 *zp = reinterpret_cast<const float4 *>(g.Z + (size_t)r * g.N + n);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 q = zp[i];
                z[4 * i] = q.x; z[4 * i + 1] = q.y; z[4 * i + 2] = q.z; z[4 * i + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const float2 zz = make_float2(z[i], z[i + 1]);
            const NormalCdf2 nc = normal_cdf2(zz);
            const float2 gg = idm::mul2(make_float2(v[i], v[i + 1]), idm::fma2(zz, nc.pdf, nc.cdf));
            h[i] = gg.x;
            h[i + 1] = gg.y;
        }
    }
    if (row_ok) {
        if (g.H) store16_bf16(g.H + (size_t)r * g.N + n, h);
        if (g.HT) {
#pragma unroll
            for (int i = 0; i < 16; ++i) g.HT[(size_t)(n + i) * g.ldt + r] = __float2bfloat16_rn(h[i]);
        }
    }
}

// Epilogue of one accumulator row: row r of the output, tw = the tensor-
// memory address of this row's column 0 of the tile, columns [c0, c1) of the
// tile (global column n0 + c), split = K-split index (F32_PART), loss_slot =
// this warp's loss partial (OUT_TRAIN, written by lane 0).
template <int MODE>
__device__ __forceinline__ void epilogue_row(const GemmArgs &g, int r, uint32_t tw, int n0, int c0, int c1, bool empty,
                                             int split, int loss_slot, const float *bias)
{
    const bool row_ok = r < g.M_rows;
    if constexpr (MODE == OUT_TRAIN || MODE == OUT_INFER) {
        float v[16];
        if (empty) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.0f;
        } else {
            tc::tmem_ld16(tw, v);
        }
        float s[OUT];
#pragma unroll
        for (int q = 0; q < OUT; ++q) s[q] = sigmoid(v[q] + bias[q]);
        if constexpr (MODE == OUT_INFER) {
            if (r < g.M_valid) {
                if (g.out[1]) {
#pragma unroll
                    for (int q = 0; q < OUT; ++q) g.out[q][r] = g.lo[q] + (g.hi[q] - g.lo[q]) * s[q];
                } else if (g.out[0]) {
#pragma unroll
                    for (int q = 0; q < OUT; ++q) g.out[0][(size_t)r * OUT + q] = s[q];
                }
            }
            return;
        }
        float d[16];
        double l = 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i) d[i] = 0.0f;
        if (r < g.M_valid) {
#pragma unroll
            for (int q = 0; q < OUT; ++q) {
                const float res = s[q] - g.label[(size_t)r * OUT + q];
                l += (double)res * (double)res;
                d[q] = 2.0f * res * s[q] * (1.0f - s[q]) * g.scale;
            }
        }
        if (row_ok) {
            store16_bf16(g.H + (size_t)r * OUTP, d);
#pragma unroll
            for (int i = 0; i < OUTP; ++i) g.HT[(size_t)i * g.ldt + r] = __float2bfloat16_rn(d[i]);
        }
        l = warp_sum(l);
        if ((threadIdx.x & 31) == 0) g.loss_part[loss_slot] = l * (double)g.scale;
    } else {
        // 64 columns per tensor-memory load where the range allows, else 16
        for (int c = c0; c < c1;) {
            if (c + 64 <= c1) {
                float w[64];
                if (empty) {
#pragma unroll
                    for (int i = 0; i < 64; ++i) w[i] = 0.0f;
                } else {
                    tc::tmem_ld64(tw + (uint32_t)c, w);
                }
#pragma unroll
                for (int part = 0; part < 4; ++part) {
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = w[16 * part + i];
                    epilogue_chunk<MODE>(g, r, n0 + c + 16 * part, split, bias, v);
                }
                c += 64;
                continue;
            }
            float v[16];
            if (empty) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.0f;
            } else {
                tc::tmem_ld16(tw + (uint32_t)c, v);
            }
            epilogue_chunk<MODE>(g, r, n0 + c, split, bias, v);
            c += 16;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(tc::NTHREADS) mlp_gemm_kernel(const GemmArgs g)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int BN = g.BN;
    const uint32_t ncols = tc::tmem_cols_for(BN);
    uint8_t *ctl = smem + 2 * tc::A_STAGE_BYTES + 2 * tc::b_stage_bytes(BN);
    const uint32_t bars = tc::smem_u32(ctl);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ctl + 16);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), ncols);
    if (threadIdx.x == 32) {
        tc::mbar_init(bars, 1);
        tc::mbar_init(bars + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    tc::TileArgs t;
    t.A = g.A;
    t.B = g.B;
    t.K = g.K;
    t.M_valid = g.M_valid;
    t.m0 = blockIdx.x * tc::BM;
    t.n0 = blockIdx.y * BN;
    t.BN = BN;
    t.kb = blockIdx.z * g.k_chunk;
    t.ke = min(g.K, t.kb + g.k_chunk);
    bool empty = false;
    const bool ok = tc::mainloop(t, smem, tmem, g.status, &empty, g.wait_iters);
    if (ok)
        epilogue_row<MODE>(g, t.m0 + threadIdx.x, tmem + ((uint32_t)(warp * 32) << 16), t.n0, 0, t.BN, empty, blockIdx.z,
                           blockIdx.x * 4 + warp, g.bias);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// Host launch of one GEMM; grid = (ceil(M/128), N/BN, splits).
template <int MODE>
cudaError_t gemm(const GemmArgs &g, int M_tiles_rows, int splits, cudaStream_t st)
{
    const int smem = tc::smem_bytes(g.BN);
    cudaError_t e = cudaFuncSetAttribute(mlp_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((M_tiles_rows + tc::BM - 1) / tc::BM, g.N / g.BN, splits);
    mlp_gemm_kernel<MODE><<<grid, tc::NTHREADS, smem, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent weight-stationary GEMM for the batch-sized products
// (C[M x N] = A[M x K] . W[N x K]^T with N <= 256, K <= 256): each CTA keeps W
// in shared memory and walks 128-row tiles of A.  Warp 0 streams the A tiles
// (64 columns per stage, 4-stage ring) with cp.async, warp 1 (one thread)
// issues the tcgen05.mma of a tile into one of two tensor-memory
// accumulators, warps 2-9 run the epilogue of the previous tile from the
// other accumulator.  Hand-offs are mbarriers: full / empty per stage, full /
// empty per accumulator.  Every wait is bounded and shares an abort flag, so
// a role that gives up releases the others.
// ---------------------------------------------------------------------------
namespace ws {
constexpr int MAX_STAGES = 8;
constexpr int EPI_WARPS = 8;    // two per tensor-memory lane quarter (column halves)
constexpr int NTHREADS = 32 * (2 + EPI_WARPS);
constexpr int CTL_BYTES = 8 * (2 * MAX_STAGES + 6) + 16;
constexpr int SMEM_LIMIT = 227 * 1024;
__host__ __device__ constexpr int w_bytes(int N, int K) { return N * K * 2; }
// A stages that fit beside the resident weights (at least 2); nbias = the
// staged bias floats
__host__ __device__ inline int max_stages(int N, int K, int nbias)
{
    const int s = (SMEM_LIMIT - w_bytes(N, K) - 1024 - CTL_BYTES - 4 * nbias) / tc::A_STAGE_BYTES;
    return s < 2 ? 2 : (s > MAX_STAGES ? MAX_STAGES : s);
}
__host__ __device__ inline int ctl_off(int N, int K, int S) { return w_bytes(N, K) + 1024 + S * tc::A_STAGE_BYTES; }
__host__ __device__ inline int smem_bytes(int N, int K, int S) { return ctl_off(N, K, S) + CTL_BYTES; }
}  // namespace ws

template <int MODE>
__global__ void __launch_bounds__(ws::NTHREADS, 1)
    mlp_gemm_ws_kernel(const GemmArgs g, const __grid_constant__ CUtensorMap tmA)
{
    extern __shared__ __align__(128) uint8_t smem[];
    // this CTA's columns: [n0, n0 + N) of the product (N = g.BN, the width
    // of the weight slice it keeps resident)
    const int N = g.BN, K = g.K, KC = K >> 3, n0 = blockIdx.y * g.BN;
    const int nkt = (K + tc::BK - 1) / tc::BK;
    const int ntiles = (g.M_rows + tc::BM - 1) / tc::BM;
    const uint32_t acc_cols = tc::tmem_cols_for(N), ncols = 2 * acc_cols;
    // A stages 1024-byte aligned (their 128-byte swizzle); the layout keeps
    // 1 KB of slack for the rounding
    const uint32_t sW = tc::smem_u32(smem), sA = (sW + (uint32_t)ws::w_bytes(N, K) + 1023u) & ~1023u;
    const int S = g.stages;
    uint8_t *ctl = smem + ws::ctl_off(N, K, S);
    const uint32_t bars = tc::smem_u32(ctl);
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (ws::MAX_STAGES + s); };
    auto tfull_bar = [&](int a) { return bars + 8u * (2 * ws::MAX_STAGES + a); };
    auto tempty_bar = [&](int a) { return bars + 8u * (2 * ws::MAX_STAGES + 2 + a); };
    const uint32_t wbar = bars + 8u * (2 * ws::MAX_STAGES + 4), drain = wbar + 8u;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ctl + 8 * (2 * ws::MAX_STAGES + 6));
    volatile int *abort = reinterpret_cast<volatile int *>(ctl + 8 * (2 * ws::MAX_STAGES + 6) + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), ncols);
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full_bar(s), 1);  // the producer's arrival with the stage's TMA byte count
            tc::mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tfull_bar(a), 1);
            tc::mbar_init(tempty_bar(a), ws::EPI_WARPS);
        }
        tc::mbar_init(wbar, 1);
        tc::mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: W once, then the A tiles -------------------------------
        for (int c = lane; c < N * KC; c += 32) {
            const int row = c / KC, kc = c - row * KC;
            tc::cp_async16(sW + (uint32_t)(((row >> 3) * KC + kc) * 128 + (row & 7) * 16),
                           g.B + (size_t)(n0 + row) * K + kc * 8, 16u);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(wbar);
        int q = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = tile * tc::BM;
            for (int kt = 0; kt < nkt; ++kt, ++q) {
                const int s = q % S;
                int got = lane == 0 ? (int)tc::mbar_wait_abort(empty_bar(s), (uint32_t)(((q / S) & 1) ^ 1), abort,
                                                               g.wait_iters)
                                    : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                const int k0 = kt * tc::BK, nch = min(tc::BK, K - k0) >> 3;
                const uint32_t dst = sA + (uint32_t)s * tc::A_STAGE_BYTES;
                // one TMA box: 128 rows x 64 K-columns, 128-byte swizzle
                // (rows past M_valid and columns past K arrive as zeros)
                (void)nch;
                if (lane == 0) {
                    tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)tc::A_STAGE_BYTES);
                    tc::tma_load_2d(dst, &tmA, k0, m0, full_bar(s));
                }
                __syncwarp();
            }
        }
        // every stage issued has landed before the CTA can leave (after a
        // give-up the tensor core may not have consumed them)
        if (lane == 0 && q > 0)
            for (int s = 0; s < S && s < q; ++s) {
                const int q_last = q - 1 - ((q - 1 - s) % S);  // last issue on stage s
                tc::mbar_wait(full_bar(s), (uint32_t)((q_last / S) & 1));
            }
        __syncwarp();
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 1) {
        // ---- MMA issue (one thread) --------------------------------------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(tc::BM, N);
            bool ok = tc::mbar_wait_abort(wbar, 0, abort, g.wait_iters);
            int q = 0, i = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
                const int acc = i & 1, u = i >> 1;
                if (!(ok = tc::mbar_wait_abort(tempty_bar(acc), (uint32_t)((u & 1) ^ 1), abort, g.wait_iters))) break;
                tc::fence_after_sync();
                for (int kt = 0; kt < nkt && ok; ++kt, ++q) {
                    const int s = q % S;
                    if (!(ok = tc::mbar_wait_abort(full_bar(s), (uint32_t)((q / S) & 1), abort, g.wait_iters))) break;
                    // the stage was written by cp.async (generic proxy); the
                    // tensor core reads it through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc::fence_after_sync();
                    const int kw = min(tc::BK, K - kt * tc::BK);
                    const uint32_t a_buf = sA + (uint32_t)s * tc::A_STAGE_BYTES;
                    for (int ks = 0; ks < (kw >> 4); ++ks) {
                        const uint64_t ad = tc::smem_desc_sw128(a_buf + (uint32_t)(ks * 32));
                        const uint64_t bd = tc::smem_desc(sW + (uint32_t)(kt * 8 + ks * 2) * 128, 128, (uint32_t)KC * 128);
                        tc::mma_bf16(tmem + (uint32_t)acc * acc_cols, ad, bd, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(empty_bar(s));
                }
                if (ok) tc::mma_commit(tfull_bar(acc));
            }
            // everything issued has completed before the tensor memory is freed
            tc::mma_commit(drain);
            tc::mbar_wait(drain, 0);
        }
    } else {
        // ---- epilogue warps ------------------------------------------------------
        // warp w serves tensor-memory lanes 32 (w % 4) .. + 31 (its rows of the
        // tile) and column part (w - 2) / 4 of the tile's 16-column chunks
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        const int nparts = ws::EPI_WARPS / 4, nch = N >> 4;
        const int c0 = 16 * ((nch * part) / nparts), c1 = 16 * ((nch * (part + 1)) / nparts);
        const bool out_mode = MODE == OUT_TRAIN || MODE == OUT_INFER;
        // the bias, once per CTA, in shared memory (read as broadcasts)
        float *bias_s = reinterpret_cast<float *>(smem + ws::smem_bytes(N, K, S));  // all g.N columns
        if (g.bias)
            for (int c = threadIdx.x - 64; c < g.N; c += 32 * ws::EPI_WARPS) bias_s[c] = g.bias[c];
        asm volatile("bar.sync 1, %0;" ::"n"(32 * ws::EPI_WARPS) : "memory");
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int acc = i & 1, u = i >> 1;
            int got = lane == 0 ? (int)tc::mbar_wait_abort(tfull_bar(acc), (uint32_t)(u & 1), abort, g.wait_iters) : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            tc::fence_after_sync();
            const uint32_t tw = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * acc_cols;
            const int r = tile * tc::BM + quarter * 32 + lane;
            if (out_mode ? part == 0 : c1 > c0)
                epilogue_row<MODE>(g, r, tw, n0, c0, c1, false, 0, tile * 4 + quarter, bias_s);
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tempty_bar(acc));
        }
    }
    if (threadIdx.x == 0 && *abort) atomicOr(g.status, IDM_STATUS_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// Tensor map of the A operand [M_valid x K] bf16 row-major for the TMA
// boxes of the persistent GEMM: 64 columns (128 bytes) x 128 rows, 128-byte
// swizzle, zero fill outside.  The encoder is the driver's
// cuTensorMapEncodeTiled, looked up once.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder()
{
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess && f)
            encode = reinterpret_cast<EncodeTiled>(f);
    }
    return encode;
}

cudaError_t a_tensor_map(const GemmArgs &g, CUtensorMap *tm)
{
    const EncodeTiled encode = encoder();
    if (!encode) return cudaErrorNotSupported;
    // the row pitch must be a multiple of 16 bytes (K % 8 == 0) and the base
    // 16-byte aligned; an empty A has no rows to describe
    if (g.K % 8 != 0 || g.M_valid < 1 || (reinterpret_cast<uintptr_t>(g.A) & 15u) != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)g.K, (cuuint64_t)g.M_valid};
    const cuuint64_t strides[1] = {(cuuint64_t)g.K * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(g.A), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Launch of the persistent GEMM: CTAs keep column slices of nsplit equal
// parts of the weights; each walks row tiles (grid x) of its slice (grid y).
template <int MODE>
cudaError_t gemm_ws(const GemmArgs &g0, int n_sm, int nsplit, cudaStream_t st)
{
    GemmArgs g = g0;
    g.BN = g.N / nsplit;
    // with split columns every CTA has few row tiles: 4 stages (a whole
    // K = 256 tile) leave room for a second resident CTA
    g.stages = ws::max_stages(g.BN, g.K, g.N);
    if (nsplit > 1 && g.stages > 4) g.stages = 4;
    const int smem = ws::smem_bytes(g.BN, g.K, g.stages) + 4 * g.N;  // + the bias
    cudaError_t e = cudaFuncSetAttribute(mlp_gemm_ws_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int ntiles = (g.M_rows + tc::BM - 1) / tc::BM;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mlp_gemm_ws_kernel<MODE>, ws::NTHREADS, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    // resident CTAs must also fit the 512 tensor-memory columns of an SM
    // (a CTA that cannot allocate would wait for another to finish)
    occ = std::max(1, std::min(occ, (int)(512 / (2 * tc::tmem_cols_for(g.BN)))));
    const int grid = std::max(1, std::min(ntiles, (n_sm * occ + nsplit - 1) / nsplit));
    CUtensorMap tmA;
    if ((e = a_tensor_map(g, &tmA)) != cudaSuccess) return e;
    mlp_gemm_ws_kernel<MODE><<<dim3(grid, nsplit), ws::NTHREADS, smem, st>>>(g, tmA);
    return cudaGetLastError();
}

// Batch-sized product: the persistent kernel when there are enough row tiles
// to keep every SM busy for several tiles (it loads the whole weight matrix
// once per CTA and overlaps each tile's epilogue with the next tile's
// products), else one CTA per 128 x BN tile.
template <int MODE>
cudaError_t gemm_batch(const GemmArgs &g, int n_sm, cudaStream_t st)
{
    const int ntiles = (g.M_rows + tc::BM - 1) / tc::BM;
    // few row tiles: split the columns so that more SMs work (each CTA then
    // keeps a narrower weight slice)
    int nsplit = 1;
    while (ntiles * nsplit < n_sm && g.N / (2 * nsplit) >= 64 && (g.N / (2 * nsplit)) % 16 == 0) nsplit *= 2;
    return gemm_ws<MODE>(g, n_sm, nsplit, st);
}

// ---------------------------------------------------------------------------
// Features (layout in idm_mlp.h).
// ---------------------------------------------------------------------------
struct FeatArgs {
    const int *lane_off;
    int n_lanes, N;
    const float *p_init, *v_init, *targets;
    int obs_stride;
    float dt;
    const int *perm;
    int n_rows;
    bf16 *X;
    const float *th[OUT];
    float *labels;
    float lo[OUT], hi[OUT];
};

__device__ __forceinline__ bool is_lane_head(const int *lane_off, int n_lanes, int i)
{
    int lo = 0, hi = n_lanes;  // find the lane l with lane_off[l] <= i < lane_off[l+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lane_off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lane_off[lo] == i;
}

__device__ __forceinline__ float obs_at(const FeatArgs &f, int i, int j)
{
    return j == 0 ? f.p_init[i] : f.targets[(size_t)(j - 1) * f.N + i];
}

__global__ void __launch_bounds__(128) features_kernel(const FeatArgs f)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= f.n_rows) return;
    const int i = f.perm ? f.perm[r] : r;
    if (i < 0 || i >= f.N) return;
    const bool head = is_lane_head(f.lane_off, f.n_lanes, i);
    const float inv_2sdt = 1.0f / (2.0f * (float)f.obs_stride * f.dt);
    const float y0 = f.p_init[i];
    float feat[4 * PREFIX];
    for (int who = 0; who < 2; ++who) {
        const int k = who == 0 ? i : i - 1;
        float *x = feat + 2 * PREFIX * who, *v = x + PREFIX;
        if (who == 1 && head) {
            for (int j = 0; j < PREFIX; ++j) {
                x[j] = feat[j] + 2.0f;
                v[j] = feat[PREFIX + j];
            }
            break;
        }
        float prev = obs_at(f, k, 0), cur = obs_at(f, k, 1);
        x[0] = (prev - y0) / 100.0f;
        v[0] = f.v_init[k] / 30.0f;
        for (int j = 1; j < PREFIX; ++j) {
            const float next = obs_at(f, k, j + 1);
            x[j] = (cur - y0) / 100.0f;
            v[j] = (next - prev) * inv_2sdt / 30.0f;
            prev = cur;
            cur = next;
        }
    }
    __align__(16) bf16 row[4 * PREFIX];
    for (int q = 0; q < 4 * PREFIX; ++q) row[q] = __float2bfloat16_rn(feat[q]);
    uint4 *dst = reinterpret_cast<uint4 *>(f.X + (size_t)r * IN);
    for (int q = 0; q < IN / 8; ++q) dst[q] = reinterpret_cast<const uint4 *>(row)[q];
    if (f.labels) {
        for (int q = 0; q < OUT; ++q) f.labels[(size_t)r * OUT + q] = (f.th[q][i] - f.lo[q]) / (f.hi[q] - f.lo[q]);
    }
}

// ---------------------------------------------------------------------------
// Small kernels: transpose of the input batch, column sums (bias
// gradients), the parameter update, the loss reduction.
// ---------------------------------------------------------------------------
// out[c][r] = in[r][c] for r < rows_valid, 0 for rows_valid <= r < rows_pad.
__global__ void transpose_kernel(const bf16 *in, int rows_valid, int rows_pad, int cols, bf16 *out)
{
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < rows_valid && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (c < cols && r < rows_pad) out[(size_t)c * rows_pad + r] = tile[threadIdx.x][y];
    }
}

// out[row] = sum_{c < n} in[row][c] (FP32, fixed order).
__global__ void __launch_bounds__(256) colsum_kernel(const bf16 *in, int ld, int n, float *out)
{
    __shared__ float sh[256];
    const bf16 *p = in + (size_t)blockIdx.x * ld;
    float s = 0.0f;
    for (int c = threadIdx.x; c < n; c += 256) s += __bfloat162float(p[c]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

struct UpdArgs {
    float *w, *m, *v;        // master weights and Adam moments [NPARAM]
    float *grad_out;         // GRAD mode output [NPARAM]
    const float *P[4];       // split-K partials of dW1 [S][256][80], dW2, dW3 [S][256][256], dW4^T [S][256][16]
    int S[4];
    const float *db;         // [256 * 3 + 16]: db1, db2, db3, db4
    bf16 *Wb[4], *Wt[4];     // bf16 copies (Wt[0] unused)
    float lr;
    int t;                   // Adam step number (1-based)
    int mode;                // 0 pack only, 1 gradient out, 2 Adam + pack
};

__device__ __forceinline__ float sum_parts(const float *P, int S, size_t stride, size_t idx)
{
    float s = 0.0f;
    for (int q = 0; q < S; ++q) s += P[q * stride + idx];
    return s;
}

__global__ void __launch_bounds__(256) update_kernel(const UpdArgs u)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    int layer, o, j, in_dim, outp;
    bool bias;
    if (i < OFF_B1) { layer = 0; bias = false; o = (i - OFF_W1) / IN; j = (i - OFF_W1) % IN; in_dim = IN; outp = HID; }
    else if (i < OFF_W2) { layer = 0; bias = true; o = i - OFF_B1; j = 0; in_dim = IN; outp = HID; }
    else if (i < OFF_B2) { layer = 1; bias = false; o = (i - OFF_W2) / HID; j = (i - OFF_W2) % HID; in_dim = HID; outp = HID; }
    else if (i < OFF_W3) { layer = 1; bias = true; o = i - OFF_B2; j = 0; in_dim = HID; outp = HID; }
    else if (i < OFF_B3) { layer = 2; bias = false; o = (i - OFF_W3) / HID; j = (i - OFF_W3) % HID; in_dim = HID; outp = HID; }
    else if (i < OFF_W4) { layer = 2; bias = true; o = i - OFF_B3; j = 0; in_dim = HID; outp = HID; }
    else if (i < OFF_B4) { layer = 3; bias = false; o = (i - OFF_W4) / HID; j = (i - OFF_W4) % HID; in_dim = HID; outp = OUTP; }
    else { layer = 3; bias = true; o = i - OFF_B4; j = 0; in_dim = HID; outp = OUTP; }

    float w = u.w[i];
    if (u.mode != 0) {
        float gr;
        if (bias) {
            gr = u.db[layer * HID + o];
        } else if (layer < 3) {
            gr = sum_parts(u.P[layer], u.S[layer], (size_t)HID * in_dim, (size_t)o * in_dim + j);
        } else {
            gr = sum_parts(u.P[3], u.S[3], (size_t)HID * OUTP, (size_t)j * OUTP + o);
        }
        if (u.mode == 1) {
            u.grad_out[i] = gr;
            return;
        }
        const float m = 0.9f * u.m[i] + 0.1f * gr;
        const float vv = 0.999f * u.v[i] + 0.001f * gr * gr;
        u.m[i] = m;
        u.v[i] = vv;
        const float bc1 = 1.0f - powf(0.9f, (float)u.t), bc2 = 1.0f - powf(0.999f, (float)u.t);
        w -= u.lr * (m / bc1) / (sqrtf(vv / bc2) + 1e-8f);
        u.w[i] = w;
    }
    if (!bias) {
        const bf16 wb = __float2bfloat16_rn(w);
        u.Wb[layer][(size_t)o * in_dim + j] = wb;
        if (layer > 0) u.Wt[layer][(size_t)j * outp + o] = wb;
    }
}

__global__ void loss_sum_kernel(const double *part, int n, double *out, unsigned *status)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (!isfinite(sh[0])) atomicOr(status, IDM_STATUS_NONFINITE);
        if (out) *out = sh[0];
    }
}

}  // namespace mlp
}  // namespace idm

using namespace idm::mlp;
namespace tc = idm::tc;

struct idm_mlp {
    int device = 0, n_sm = 1;
    int max_batch = 0, bp_cap = 0;  // rows; bp_cap = max_batch rounded up to 128
    int S_cap = 1;                  // split-K capacity of the weight-gradient partials
    void *arena = nullptr;
    float *w = nullptr, *m = nullptr, *v = nullptr;
    bf16 *Wb[4] = {}, *Wt[4] = {};
    bf16 *XT = nullptr, *H[3] = {}, *HT[3] = {}, *dO = nullptr, *dOT = nullptr, *dZ[2] = {}, *dZT[2] = {};
    float *Z[3] = {};
    float *P[4] = {};
    float *db = nullptr;
    double *loss_part = nullptr, *loss_tmp = nullptr;
    unsigned *status = nullptr;
    int t = 0;  // Adam steps taken
    // inference ping-pong activations for chunks larger than the training
    // batch (allocated by the first inference call that needs them)
    void *inf_arena = nullptr;
    bf16 *IH[2] = {};
    int inf_rows = 0;
    unsigned wait_iters = idm::tc::WAIT_ITERS;  // polls per tensor-core wait (idm_mlp_set_wait_limit)
    char err[256] = {0};
};

namespace {

int mfail(idm_mlp *n, int code, const char *fmt, ...)
{
    if (n) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(n->err, sizeof n->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define MCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return mfail(n, IDM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int round128(int x) { return (x + 127) / 128 * 128; }

// Split-K plan of a weight-gradient GEMM: K = Bp rows of the batch.
void wgrad_plan(int n_sm, int Bp, int m_tiles, int n_tiles, int *splits, int *k_chunk)
{
    int S = std::max(1, 2 * n_sm / std::max(1, m_tiles * n_tiles));
    S = std::min(S, std::max(1, Bp / 256));
    int kc = (Bp + S - 1) / S;
    kc = (kc + 63) / 64 * 64;
    *k_chunk = kc;
    *splits = (Bp + kc - 1) / kc;
}

GemmArgs base_args(idm_mlp *n)
{
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.status = n->status;
    g.wait_iters = n->wait_iters;
    return g;
}

// Forward through the three hidden layers for Bp rows (X rows < B valid).
// store_train: keep Z and the transposed activations for the backward pass
// (outputs in H[0..2]); otherwise the activations alternate between the two
// buffers of out (the last layer's lands in out[0]).
int hidden_forward(idm_mlp *n, const bf16 *X, int B, int Bp, bool store_train, cudaStream_t st,
                   bf16 *const *out = nullptr)
{
    for (int l = 0; l < 3; ++l) {
        bf16 *dst = store_train || !out ? n->H[l] : out[l & 1 ? 1 : 0];
        const bf16 *src = l == 0 ? X : (store_train || !out ? n->H[l - 1] : out[(l - 1) & 1 ? 1 : 0]);
        GemmArgs g = base_args(n);
        g.A = src;
        g.B = n->Wb[l];
        g.M_valid = l == 0 ? B : Bp;
        g.M_rows = Bp;
        g.N = HID;
        g.K = l == 0 ? IN : HID;
        g.BN = 128;
        g.k_chunk = g.K;
        g.bias = n->w + (l == 0 ? OFF_B1 : l == 1 ? OFF_B2 : OFF_B3);
        g.Z = store_train ? n->Z[l] : nullptr;
        g.H = dst;
        g.HT = store_train ? n->HT[l] : nullptr;
        g.ldt = Bp;
        MCK(gemm_batch<GELU_FWD>(g, n->n_sm, st));
    }
    return IDM_OK;
}

// Forward + loss + backward for one batch; leaves the partials and bias
// gradients for update_kernel and the loss in n->loss_tmp (or loss_out).
int fwd_bwd(idm_mlp *n, const bf16 *X, const float *labels, int B, double *loss_out, UpdArgs *u, cudaStream_t st)
{
    const int Bp = round128(B);
    int rc;
    // X^T for dW1
    {
        dim3 grid(Bp / 32, (IN + 31) / 32), block(32, 8);
        idm::mlp::transpose_kernel<<<grid, block, 0, st>>>(X, B, Bp, IN, n->XT);
        MCK(cudaGetLastError());
    }
    if ((rc = hidden_forward(n, X, B, Bp, true, st))) return rc;
    {  // output layer + loss + dO
        GemmArgs g = base_args(n);
        g.A = n->H[2];
        g.B = n->Wb[3];
        g.M_valid = B;
        g.M_rows = Bp;
        g.N = OUTP;
        g.K = HID;
        g.BN = OUTP;
        g.k_chunk = HID;
        g.bias = n->w + OFF_B4;
        g.H = n->dO;
        g.HT = n->dOT;
        g.ldt = Bp;
        g.label = labels;
        g.loss_part = n->loss_part;
        g.scale = 1.0f / (5.0f * (float)B);
        MCK(gemm_batch<OUT_TRAIN>(g, n->n_sm, st));
        idm::mlp::loss_sum_kernel<<<1, 256, 0, st>>>(n->loss_part, Bp / 128 * 4, loss_out ? loss_out : n->loss_tmp,
                                                      n->status);
        MCK(cudaGetLastError());
    }
    // dW4^T = H3^T . dO  (M = 256 hidden units, N = 16, K = Bp)
    int S, kc;
    wgrad_plan(n->n_sm, Bp, 2, 1, &S, &kc);
    {
        GemmArgs g = base_args(n);
        g.A = n->HT[2];
        g.B = n->dOT;
        g.M_valid = HID;
        g.M_rows = HID;
        g.N = OUTP;
        g.K = Bp;
        g.BN = OUTP;
        g.k_chunk = kc;
        g.Cf = n->P[3];
        MCK(gemm<F32_PART>(g, HID, S, st));
        u->S[3] = S;
    }
    idm::mlp::colsum_kernel<<<OUTP, 256, 0, st>>>(n->dOT, Bp, Bp, n->db + 3 * HID);
    MCK(cudaGetLastError());
    // hidden layers, top down: dZ_l = (dZ_{l+1} W_{l+1}) * gelu'(Z_l)
    const bf16 *up = n->dO;  // dZ_{l+1} as [Bp][width]
    int up_width = OUTP;
    for (int l = 2; l >= 0; --l) {
        const int buf = l & 1;
        {
            GemmArgs g = base_args(n);
            g.A = up;
            g.B = n->Wt[l + 1];  // W_{l+1}^T [256][width]
            g.M_valid = Bp;
            g.M_rows = Bp;
            g.N = HID;
            g.K = up_width;
            g.BN = 128;
            g.k_chunk = up_width;
            g.Z = n->Z[l];
            g.H = l > 0 ? n->dZ[buf] : nullptr;
            g.HT = n->dZT[buf];
            g.ldt = Bp;
            MCK(gemm_batch<DGELU>(g, n->n_sm, st));
        }
        // dW_l = dZ_l^T . H_{l-1}  (M = 256, N = fan-in, K = Bp)
        {
            const int fan_in = l == 0 ? IN : HID;
            const int bn = l == 0 ? IN : 64;
            wgrad_plan(n->n_sm, Bp, 2, fan_in / bn, &S, &kc);
            GemmArgs g = base_args(n);
            g.A = n->dZT[buf];
            g.B = l == 0 ? n->XT : n->HT[l - 1];
            g.M_valid = HID;
            g.M_rows = HID;
            g.N = fan_in;
            g.K = Bp;
            g.BN = bn;
            g.k_chunk = kc;
            g.Cf = n->P[l];
            MCK(gemm<F32_PART>(g, HID, S, st));
            u->S[l] = S;
        }
        idm::mlp::colsum_kernel<<<HID, 256, 0, st>>>(n->dZT[buf], Bp, Bp, n->db + l * HID);
        MCK(cudaGetLastError());
        up = n->dZ[buf];
        up_width = HID;
    }
    return IDM_OK;
}

// Rows per inference chunk and the activation buffers for it: the training
// buffers when the chunk fits them, else dedicated ping-pong buffers of
// INFER_CHUNK rows.
constexpr int INFER_CHUNK = 131072;

int infer_buffers(idm_mlp *n, int B, int *chunk, bf16 **buf)
{
    if (B <= n->bp_cap) {
        *chunk = n->max_batch;
        buf[0] = n->H[0];
        buf[1] = n->H[1];
        return IDM_OK;
    }
    if (!n->inf_arena) {
        const size_t bytes = 2 * (size_t)INFER_CHUNK * HID * sizeof(bf16);
        if (cudaMalloc(&n->inf_arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            n->inf_arena = nullptr;
            return mfail(n, IDM_ERR_CUDA, "cannot allocate %zu bytes of inference buffers", bytes);
        }
        n->IH[0] = (bf16 *)n->inf_arena;
        n->IH[1] = n->IH[0] + (size_t)INFER_CHUNK * HID;
        n->inf_rows = INFER_CHUNK;
    }
    *chunk = n->inf_rows;
    buf[0] = n->IH[0];
    buf[1] = n->IH[1];
    return IDM_OK;
}

UpdArgs upd_base(idm_mlp *n)
{
    UpdArgs u;
    memset(&u, 0, sizeof u);
    u.w = n->w;
    u.m = n->m;
    u.v = n->v;
    for (int l = 0; l < 4; ++l) {
        u.P[l] = n->P[l];
        u.Wb[l] = n->Wb[l];
        u.Wt[l] = n->Wt[l];
    }
    u.db = n->db;
    return u;
}

cudaError_t launch_update(const UpdArgs &u, cudaStream_t st)
{
    idm::mlp::update_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(u);
    return cudaGetLastError();
}

int check_batch(idm_mlp *n, const void *X, int B)
{
    if (!X) return mfail(n, IDM_ERR_ARG, "X is required");
    if ((uintptr_t)X & 15) return mfail(n, IDM_ERR_ARG, "X must be 16-byte aligned");
    if (B < 1 || B > n->max_batch) return mfail(n, IDM_ERR_ARG, "B = %d outside [1, %d]", B, n->max_batch);
    return IDM_OK;
}

}  // namespace

extern "C" {

int idm_gemm_bf16(const void *A, const void *B, int32_t M, int32_t N, int32_t K, float *C, uint32_t *status,
                  void *stream)
{
    if (!A || !B || !C || !status) return IDM_ERR_ARG;
    if (M < 1 || N < 16 || N % 16 || K < 16 || K % 16) return IDM_ERR_ARG;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) return IDM_ERR_ARG;
    int bn = 16;
    for (int c = 256; c >= 16; c -= 16)
        if (N % c == 0) {
            bn = c;
            break;
        }
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.A = (const bf16 *)A;
    g.B = (const bf16 *)B;
    g.M_valid = M;
    g.M_rows = M;
    g.N = N;
    g.K = K;
    g.BN = bn;
    g.k_chunk = K;
    g.Cf = C;
    g.status = status;
    g.wait_iters = idm::tc::WAIT_ITERS;
    cudaError_t e = gemm<F32_PART>(g, M, 1, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IDM_ERR_CUDA;
    }
    return IDM_OK;
}

int idm_mlp_gelu_eval(const float *z, float *gelu_out, float *gelu_grad_out, int32_t n, void *stream)
{
    if (n < 0 || (n > 0 && !z)) return IDM_ERR_ARG;
    if (n == 0) return IDM_OK;
    idm::mlp::gelu_eval_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(z, gelu_out, gelu_grad_out, n);
    return cudaGetLastError() == cudaSuccess ? IDM_OK : IDM_ERR_CUDA;
}

int idm_mlp_create(idm_mlp_t **out, int32_t max_batch)
{
    if (!out || max_batch < 1 || max_batch > (1 << 22)) return IDM_ERR_ARG;
    *out = nullptr;
    idm_mlp *n = new idm_mlp();
    if (cudaGetDevice(&n->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&n->n_sm, cudaDevAttrMultiProcessorCount, n->device) != cudaSuccess) {
        delete n;
        return IDM_ERR_CUDA;
    }
    n->max_batch = max_batch;
    const int Bp = round128(max_batch);
    n->bp_cap = Bp;
    // largest split count any weight-gradient GEMM uses at this batch size
    int S = 1;
    for (int tiles : {1, 4}) {
        int s_, k_;
        wgrad_plan(n->n_sm, Bp, 2, tiles, &s_, &k_);
        S = std::max(S, s_);
    }
    n->S_cap = S;
    // carve one arena
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_w = take(4 * (size_t)NPARAM), o_m = take(4 * (size_t)NPARAM), o_v = take(4 * (size_t)NPARAM);
    size_t o_Wb[4], o_Wt[4];
    o_Wb[0] = take(2 * (size_t)HID * IN);
    o_Wb[1] = take(2 * (size_t)HID * HID);
    o_Wb[2] = take(2 * (size_t)HID * HID);
    o_Wb[3] = take(2 * (size_t)OUTP * HID);
    o_Wt[0] = 0;
    o_Wt[1] = take(2 * (size_t)HID * HID);
    o_Wt[2] = take(2 * (size_t)HID * HID);
    o_Wt[3] = take(2 * (size_t)HID * OUTP);
    const size_t o_XT = take(2 * (size_t)IN * Bp);
    size_t o_H[3], o_HT[3], o_Z[3], o_dZ[2], o_dZT[2], o_P[4];
    for (int l = 0; l < 3; ++l) {
        o_H[l] = take(2 * (size_t)Bp * HID);
        o_HT[l] = take(2 * (size_t)Bp * HID);
        o_Z[l] = take(4 * (size_t)Bp * HID);
    }
    const size_t o_dO = take(2 * (size_t)Bp * OUTP), o_dOT = take(2 * (size_t)Bp * OUTP);
    for (int b = 0; b < 2; ++b) {
        o_dZ[b] = take(2 * (size_t)Bp * HID);
        o_dZT[b] = take(2 * (size_t)Bp * HID);
    }
    o_P[0] = take(4 * (size_t)S * HID * IN);
    o_P[1] = take(4 * (size_t)S * HID * HID);
    o_P[2] = take(4 * (size_t)S * HID * HID);
    o_P[3] = take(4 * (size_t)S * HID * OUTP);
    const size_t o_db = take(4 * (size_t)(3 * HID + OUTP));
    const size_t o_lp = take(8 * (size_t)(Bp / 128 * 4)), o_lt = take(8 * 2), o_st = take(16);
    if (cudaMalloc(&n->arena, off) != cudaSuccess) {
        cudaGetLastError();
        delete n;
        return IDM_ERR_CUDA;
    }
    if (cudaMemset(n->arena, 0, off) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(n->arena);
        delete n;
        return IDM_ERR_CUDA;
    }
    char *a = (char *)n->arena;
    n->w = (float *)(a + o_w);
    n->m = (float *)(a + o_m);
    n->v = (float *)(a + o_v);
    for (int l = 0; l < 4; ++l) {
        n->Wb[l] = (bf16 *)(a + o_Wb[l]);
        n->Wt[l] = l ? (bf16 *)(a + o_Wt[l]) : nullptr;
        n->P[l] = (float *)(a + o_P[l]);
    }
    n->XT = (bf16 *)(a + o_XT);
    for (int l = 0; l < 3; ++l) {
        n->H[l] = (bf16 *)(a + o_H[l]);
        n->HT[l] = (bf16 *)(a + o_HT[l]);
        n->Z[l] = (float *)(a + o_Z[l]);
    }
    n->dO = (bf16 *)(a + o_dO);
    n->dOT = (bf16 *)(a + o_dOT);
    for (int b = 0; b < 2; ++b) {
        n->dZ[b] = (bf16 *)(a + o_dZ[b]);
        n->dZT[b] = (bf16 *)(a + o_dZT[b]);
    }
    n->db = (float *)(a + o_db);
    n->loss_part = (double *)(a + o_lp);
    n->loss_tmp = (double *)(a + o_lt);
    n->status = (unsigned *)(a + o_st);
    *out = n;
    return IDM_OK;
}

int idm_mlp_destroy(idm_mlp_t *n)
{
    if (!n) return IDM_OK;
    if (n->arena || n->inf_arena) cudaDeviceSynchronize();
    if (n->arena) cudaFree(n->arena);
    if (n->inf_arena) cudaFree(n->inf_arena);
    delete n;
    return IDM_OK;
}

const char *idm_mlp_last_error(const idm_mlp_t *n) { return n ? n->err : "null network"; }

int idm_mlp_set_weights(idm_mlp_t *n, const float *weights, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    if (!weights) return mfail(n, IDM_ERR_ARG, "weights are required");
    cudaStream_t st = (cudaStream_t)stream;
    MCK(cudaMemcpyAsync(n->w, weights, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st));
    MCK(cudaMemsetAsync(n->m, 0, sizeof(float) * NPARAM, st));
    MCK(cudaMemsetAsync(n->v, 0, sizeof(float) * NPARAM, st));
    n->t = 0;
    UpdArgs u = upd_base(n);
    u.mode = 0;
    MCK(launch_update(u, st));
    return IDM_OK;
}

int idm_mlp_get_weights(idm_mlp_t *n, float *weights, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    if (!weights) return mfail(n, IDM_ERR_ARG, "weights are required");
    MCK(cudaMemcpyAsync(weights, n->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return IDM_OK;
}

int idm_mlp_set_wait_limit(idm_mlp_t *n, uint32_t polls)
{
    if (!n) return IDM_ERR_ARG;
    n->wait_iters = polls == 0 ? idm::tc::WAIT_ITERS : std::min<uint32_t>(polls, idm::tc::WAIT_ITERS);
    return IDM_OK;
}

int idm_mlp_clear_status(idm_mlp_t *n, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    MCK(cudaMemsetAsync(n->status, 0, sizeof(unsigned), (cudaStream_t)stream));
    MCK(cudaStreamSynchronize((cudaStream_t)stream));
    return IDM_OK;
}

int idm_mlp_status(idm_mlp_t *n, void *stream, uint32_t *bits)
{
    if (!n) return IDM_ERR_ARG;
    unsigned h = 0;
    MCK(cudaMemcpyAsync(&h, n->status, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    MCK(cudaStreamSynchronize((cudaStream_t)stream));
    if (bits) *bits = h;
    if (h & IDM_STATUS_TIMEOUT) return mfail(n, IDM_ERR_TIMEOUT, "a tensor-core kernel gave up waiting");
    if (h & IDM_STATUS_NONFINITE) return mfail(n, IDM_ERR_NONFINITE, "non-finite loss");
    return IDM_OK;
}

int idm_mlp_features(const idm_scene_t *sc, const float *p_init, const float *v_init, const idm_sim_t *sim,
                     const float *targets, int32_t obs_stride, const int32_t *perm, int32_t n_rows, void *X,
                     const idm_params_t *label_params, float *labels, const float *box_lo, const float *box_hi,
                     void *stream)
{
    if (!sc || !sim || !sc->lane_off || sc->n_lanes < 1 || sc->n_vehicles < 1) return IDM_ERR_ARG;
    if (!p_init || !v_init || !targets || !X || n_rows < 0) return IDM_ERR_ARG;
    if (obs_stride < 1 || !(sim->dt > 0.0f) || sim->K / obs_stride < PREFIX) return IDM_ERR_ARG;
    if ((label_params == nullptr) != (labels == nullptr)) return IDM_ERR_ARG;
    if (labels) {
        if (!box_lo || !box_hi) return IDM_ERR_ARG;
        if (!label_params->v0 || !label_params->T || !label_params->s0 || !label_params->a_max || !label_params->b)
            return IDM_ERR_ARG;
        for (int q = 0; q < OUT; ++q)
            if (!(box_hi[q] > box_lo[q])) return IDM_ERR_ARG;
    }
    if (((uintptr_t)X) & 15) return IDM_ERR_ARG;
    if (n_rows == 0) return IDM_OK;
    FeatArgs f;
    memset(&f, 0, sizeof f);
    f.lane_off = sc->lane_off;
    f.n_lanes = sc->n_lanes;
    f.N = sc->n_vehicles;
    f.p_init = p_init;
    f.v_init = v_init;
    f.targets = targets;
    f.obs_stride = obs_stride;
    f.dt = sim->dt;
    f.perm = perm;
    f.n_rows = n_rows;
    f.X = (bf16 *)X;
    f.labels = labels;
    if (labels) {
        f.th[0] = label_params->v0;
        f.th[1] = label_params->T;
        f.th[2] = label_params->s0;
        f.th[3] = label_params->a_max;
        f.th[4] = label_params->b;
        for (int q = 0; q < OUT; ++q) {
            f.lo[q] = box_lo[q];
            f.hi[q] = box_hi[q];
        }
    }
    idm::mlp::features_kernel<<<(n_rows + 127) / 128, 128, 0, (cudaStream_t)stream>>>(f);
    if (cudaGetLastError() != cudaSuccess) return IDM_ERR_CUDA;
    return IDM_OK;
}

int idm_mlp_forward(idm_mlp_t *n, const void *X, int32_t B, float *out, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(n, X, B))) return rc;
    if (!out) return mfail(n, IDM_ERR_ARG, "out is required");
    cudaStream_t st = (cudaStream_t)stream;
    const int Bp = round128(B);
    if ((rc = hidden_forward(n, (const bf16 *)X, B, Bp, false, st))) return rc;
    GemmArgs g = base_args(n);
    g.A = n->H[2];
    g.B = n->Wb[3];
    g.M_valid = B;
    g.M_rows = Bp;
    g.N = OUTP;
    g.K = HID;
    g.BN = OUTP;
    g.k_chunk = HID;
    g.bias = n->w + OFF_B4;
    g.out[0] = out;
    MCK(gemm_batch<OUT_INFER>(g, n->n_sm, st));
    return IDM_OK;
}

int idm_mlp_predict_params(idm_mlp_t *n, const void *X, int32_t B, idm_params_t *params, const float *box_lo,
                           const float *box_hi, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    if (!X || B < 1) return mfail(n, IDM_ERR_ARG, "X and B >= 1 are required");
    if ((uintptr_t)X & 15) return mfail(n, IDM_ERR_ARG, "X must be 16-byte aligned");
    if (!params || !params->v0 || !params->T || !params->s0 || !params->a_max || !params->b)
        return mfail(n, IDM_ERR_ARG, "params (v0, T, s0, a_max, b) are required");
    if (!box_lo || !box_hi) return mfail(n, IDM_ERR_ARG, "box_lo and box_hi (host) are required");
    cudaStream_t st = (cudaStream_t)stream;
    float *outs[OUT] = {params->v0, params->T, params->s0, params->a_max, params->b};
    int chunk, rc;
    bf16 *buf[2];
    if ((rc = infer_buffers(n, B, &chunk, buf))) return rc;
    for (int r0 = 0; r0 < B; r0 += chunk) {
        const int b = std::min(chunk, B - r0);
        const int Bp = round128(b);
        const bf16 *Xc = (const bf16 *)X + (size_t)r0 * IN;
        if ((rc = hidden_forward(n, Xc, b, Bp, false, st, buf))) return rc;
        GemmArgs g = base_args(n);
        g.A = buf[0];
        g.B = n->Wb[3];
        g.M_valid = b;
        g.M_rows = Bp;
        g.N = OUTP;
        g.K = HID;
        g.BN = OUTP;
        g.k_chunk = HID;
        g.bias = n->w + OFF_B4;
        for (int q = 0; q < OUT; ++q) {
            g.out[q] = outs[q] + r0;
            g.lo[q] = box_lo[q];
            g.hi[q] = box_hi[q];
        }
        MCK(gemm_batch<OUT_INFER>(g, n->n_sm, st));
    }
    return IDM_OK;
}

int idm_mlp_loss_grad(idm_mlp_t *n, const void *X, const float *labels, int32_t B, double *loss_out, float *grad,
                      void *stream)
{
    if (!n) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(n, X, B))) return rc;
    if (!labels || !grad) return mfail(n, IDM_ERR_ARG, "labels and grad are required");
    cudaStream_t st = (cudaStream_t)stream;
    UpdArgs u = upd_base(n);
    if ((rc = fwd_bwd(n, (const bf16 *)X, labels, B, loss_out, &u, st))) return rc;
    u.mode = 1;
    u.grad_out = grad;
    MCK(launch_update(u, st));
    return IDM_OK;
}

int idm_mlp_train_step(idm_mlp_t *n, const void *X, const float *labels, int32_t B, float lr, double *loss_out,
                       void *stream)
{
    if (!n) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(n, X, B))) return rc;
    if (!labels) return mfail(n, IDM_ERR_ARG, "labels are required");
    if (!(lr >= 0.0f)) return mfail(n, IDM_ERR_ARG, "lr must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    UpdArgs u = upd_base(n);
    if ((rc = fwd_bwd(n, (const bf16 *)X, labels, B, loss_out, &u, st))) return rc;
    u.mode = 2;
    u.lr = lr;
    u.t = ++n->t;
    MCK(launch_update(u, st));
    return IDM_OK;
}

int idm_mlp_train(idm_mlp_t *n, const void *X, const float *labels, int64_t n_samples, int32_t batch,
                  int32_t n_steps, float lr0, float lr1, double *loss_hist, void *stream)
{
    if (!n) return IDM_ERR_ARG;
    int rc;
    if ((rc = check_batch(n, X, batch))) return rc;
    if (!labels) return mfail(n, IDM_ERR_ARG, "labels are required");
    if (n_samples < batch) return mfail(n, IDM_ERR_ARG, "n_samples < batch");
    if (n_steps < 0) return mfail(n, IDM_ERR_ARG, "n_steps must be >= 0");
    if (!(lr0 >= 0.0f) || !(lr1 >= 0.0f)) return mfail(n, IDM_ERR_ARG, "learning rates must be >= 0");
    const int64_t n_batches = n_samples / batch;
    for (int s = 0; s < n_steps; ++s) {
        const int64_t r0 = (s % n_batches) * (int64_t)batch;
        const float lr = n_steps > 1 ? lr0 + (lr1 - lr0) * (float)s / (float)(n_steps - 1) : lr0;
        if ((rc = idm_mlp_train_step(n, (const bf16 *)X + r0 * IN, labels + r0 * OUT, batch, lr,
                                     loss_hist ? loss_hist + s : nullptr, stream)))
            return rc;
    }
    return IDM_OK;
}

}  // extern "C"
