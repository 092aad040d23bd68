// BF16 tensor-core GEMM building blocks for sm_103a (tcgen05 + tensor memory).
//
//   C[m0:m0+128, n0:n0+BN] = sum over k in [kb, ke) of A[m, k] * B[n, k]
//
// A [M x K] and B [N x K] are row-major bf16 with K contiguous (both
// operands K-major), accumulation in FP32.  One CTA of 4 warps owns one
// 128 x BN tile (BN <= 256, a multiple of 16) whose accumulator lives in
// tensor memory.  Tiles of 64 K-columns are staged in shared memory in the
// no-swizzle canonical layout: 8 x 8 core matrices of 16-byte rows stored
// as 128 contiguous bytes; core matrices adjacent in K are LBO = 128 bytes
// apart and 8-row groups SBO = 1024 bytes apart.  Two stages: while the
// tensor core works on stage s, all threads fill stage s^1 with cp.async.
// One thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16 per
// instruction) and signals completion of a stage with tcgen05.commit on that
// stage's mbarrier.  Warp w reads accumulator rows 32w..32w+31 (its tensor
// memory lanes) with tcgen05.ld.
//
// Every mbarrier wait is bounded (iterations and wall time).  A CTA whose
// wait gives up records IDM_STATUS_TIMEOUT, waits (again bounded) for the
// tensor-core work it issued, skips its epilogue and frees its tensor memory.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/idm.h"

namespace idm {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int NTHREADS = 128;
constexpr int MAX_BN = 256;
constexpr int A_STAGE_BYTES = BM * BK * 2;  // 16 KB
constexpr uint32_t WAIT_ITERS = 1u << 26;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s

__host__ __device__ constexpr int b_stage_bytes(int bn) { return bn * BK * 2; }
// Dynamic shared memory of one CTA: two A stages, two B stages, two
// mbarriers and the tensor-memory address slot.
__host__ __device__ constexpr int smem_bytes(int bn) { return 2 * A_STAGE_BYTES + 2 * b_stage_bytes(bn) + 32; }

// Tensor-memory columns to allocate for a BN-wide accumulator (a power of
// two >= 32).
__host__ __device__ inline uint32_t tmem_cols_for(int bn)
{
    uint32_t c = 32;
    while ((int)c < bn) c <<= 1;
    return c;
}

// Byte offset of the 16-byte chunk kc (k = 8 kc .. 8 kc + 7) of row `row`
// inside a staged 64-column tile.
__device__ __forceinline__ uint32_t tile_off(int row, int kc)
{
    return (uint32_t)(((row >> 3) * 8 + kc) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte global -> shared copy; src_bytes = 0 fills the destination with
// zeros (src must still be a valid address).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// Shared-memory matrix descriptor: start address >> 4 in bits 0-13, LBO >> 4
// in bits 16-29, SBO >> 4 in bits 32-45, the fixed value 1 in bits 46-48,
// base offset 0, no swizzling (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Descriptor of a K-major operand tile with the 128-byte swizzle: rows of
// 128 bytes (64 bf16 of K), 8-row groups SBO = 1024 bytes apart, the 16-byte
// chunks of row r at chunk ^ (r & 7) (the layout a TMA box of 64 columns with
// CU_TENSOR_MAP_SWIZZLE_128B writes); swizzling mode 2 in bits 61-63.  The
// tile starts 1024-byte aligned; the K step of 16 columns advances the start
// address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                  // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;       // SBO
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, bits 10-12 = 1), no negation, both operands K-major (bits
// 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ inline uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Wait until the phase with the given parity has completed; false when the
// iteration limit (`limit` polls) or the time limit runs out first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = WAIT_ITERS)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255u) == 255u) {
            const uint64_t t = global_ns();
            if (t0 == 0)
                t0 = t;
            else if (t - t0 > WAIT_NS)
                return false;
        }
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

// mbar_wait that also gives up as soon as another role of the CTA has set
// the shared abort flag, and sets it when it gives up itself.
__device__ __forceinline__ bool mbar_wait_abort(uint32_t bar, uint32_t parity, volatile int *abort,
                                                uint32_t limit = WAIT_ITERS)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255u) == 255u) {
            if (*abort) return false;
            const uint64_t t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > WAIT_NS) {
                *abort = 1;
                return false;
            }
        }
    }
    *abort = 1;
    return false;
}

// mbarrier arrival that also announces `bytes` of asynchronous (TMA)
// transactions the current phase must receive before it completes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// TMA copy of the 2D box at element coordinates (x, y) of the tensor map
// into shared memory at dst; its bytes complete a transaction on `bar`.
// The map (a __grid_constant__ kernel parameter) fixes the box and the
// zero fill of rows or columns outside the tensor.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Whole-warp tensor-memory allocation; the address is written to shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier once every tcgen05 operation this thread issued
// before has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 accumulator columns of this thread's row: one load
// instruction and one wait (the epilogue's exposed tensor-memory latency is
// a quarter of that of four tmem_ld16).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64])
{
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Operands of one CTA tile.
struct TileArgs {
    const __nv_bfloat16 *A;  // [M_valid x K] (rows >= M_valid read as zeros)
    const __nv_bfloat16 *B;  // [>= n0 + BN rows x K]
    int K;                   // row length of A and B (a multiple of 16)
    int M_valid;
    int m0, n0, BN;
    int kb, ke;              // K range (multiples of 16)
};

// Stage the 64-column K tile starting at k0 (width kw) of A and B.
__device__ __forceinline__ void load_stage(const TileArgs &t, int k0, int kw, uint32_t a_buf, uint32_t b_buf)
{
    const int nch = kw >> 3;  // 16-byte chunks per row
    for (int c = threadIdx.x; c < BM * 8; c += NTHREADS) {
        const int row = c >> 3, kc = c & 7;
        if (kc >= nch) continue;
        const int m = t.m0 + row;
        const bool ok = m < t.M_valid;
        const __nv_bfloat16 *src = t.A + (size_t)(ok ? m : 0) * t.K + k0 + kc * 8;
        cp_async16(a_buf + tile_off(row, kc), src, ok ? 16u : 0u);
    }
    for (int c = threadIdx.x; c < t.BN * 8; c += NTHREADS) {
        const int row = c >> 3, kc = c & 7;
        if (kc >= nch) continue;
        cp_async16(b_buf + tile_off(row, kc), t.B + (size_t)(t.n0 + row) * t.K + k0 + kc * 8, 16u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Accumulate the tile into tensor memory at `tmem`.  Every thread of the CTA
// calls it.  Returns false (status recorded, issued work drained) when a
// wait gave up; returns true with *empty set when the K range is empty (the
// accumulator is then not written).  `limit` bounds the polls of each wait
// for the tensor core (WAIT_ITERS normally; the drain after a give-up always
// uses WAIT_ITERS).
__device__ __forceinline__ bool mainloop(const TileArgs &t, uint8_t *smem, uint32_t tmem, unsigned *status,
                                         bool *empty, uint32_t limit = WAIT_ITERS)
{
    const int tid = threadIdx.x;
    const uint32_t sA = smem_u32(smem), sB = sA + 2 * A_STAGE_BYTES;
    const uint32_t bars = sA + 2 * A_STAGE_BYTES + 2 * b_stage_bytes(t.BN);
    const uint32_t idesc = idesc_bf16(BM, t.BN);
    const int nkt = (t.ke - t.kb + BK - 1) / BK;
    *empty = nkt <= 0;
    if (nkt <= 0) return true;

    load_stage(t, t.kb, min(BK, t.ke - t.kb), sA, sB);
    for (int kt = 0; kt < nkt; ++kt) {
        const int buf = kt & 1;
        const int kw = min(BK, t.ke - (t.kb + kt * BK));
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // make the copies visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t a_buf = sA + buf * A_STAGE_BYTES, b_buf = sB + buf * b_stage_bytes(t.BN);
            for (int ks = 0; ks < (kw >> 4); ++ks) {
                const uint64_t ad = smem_desc(a_buf + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(b_buf + ks * 256, 128, 1024);
                mma_bf16(tmem, ad, bd, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(bars + 8 * buf);
        }
        if (kt + 1 < nkt) {
            // stage kt+1 goes to buffer buf^1, last read by the MMAs of tile kt-1
            const int nb = buf ^ 1;
            if (kt >= 1) {
                // every thread takes the same decision, so that no thread
                // leaves while others still wait at a CTA barrier
                const bool done = __syncthreads_and(mbar_wait(bars + 8 * nb, (uint32_t)(((kt - 1) >> 1) & 1), limit));
                if (!done) {
                    if (tid == 0) atomicOr(status, IDM_STATUS_TIMEOUT);
                    mbar_wait(bars + 8 * buf, (uint32_t)((kt >> 1) & 1));  // drain what was issued
                    return false;
                }
            }
            const int k1 = t.kb + (kt + 1) * BK;
            load_stage(t, k1, min(BK, t.ke - k1), sA + nb * A_STAGE_BYTES, sB + nb * b_stage_bytes(t.BN));
        }
    }
    const int last = nkt - 1;
    const bool done = __syncthreads_and(mbar_wait(bars + 8 * (last & 1), (uint32_t)((last >> 1) & 1), limit));
    if (!done) {
        if (tid == 0) atomicOr(status, IDM_STATUS_TIMEOUT);
        mbar_wait(bars + 8 * (last & 1), (uint32_t)((last >> 1) & 1));
        return false;
    }
    fence_after_sync();
    return true;
}

}  // namespace tc
}  // namespace idm
