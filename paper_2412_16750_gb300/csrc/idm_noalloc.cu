// idm_loss_grad_noalloc: the fused loss + gradient of idm_loss_grad for
// callers that cannot allocate device memory: an application whose device
// memory is owned by its own allocator or pool (which a cudaMalloc inside a
// library would bypass and fragment), or one that admits work only against a
// memory budget fixed up front.
//
// All scratch (warp segments, control counters, status word, initial gaps,
// per-warp loss partials, checkpoints, the compensated gradient totals)
// lives in one file-scope device array of IDM_NOALLOC_SCRATCH_BYTES.  Every
// GPU that loads the library holds that array until the process exits.  Host
// code must not pass the array's name to a kernel: on the host the name is
// only a stand-in for the symbol.  The device address is looked up with
// cudaGetSymbolAddress once per CUDA context (keyed by the context's unique
// id, so a device reset, which creates a new context, looks it up again) and
// cached.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/idm.h"
#include "idm_ctx.h"
#include "idm_internal.h"

using idm::ScenDesc;
using idm::Seg;
using idm::SimArgs;
using namespace idm::abi;

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[IDM_NOALLOC_SCRATCH_BYTES];

// Cache of the array's device address per CUDA context.  The runtime has no
// call that names the current context, so the two driver entry points are
// fetched through the runtime (no link against the driver library).
typedef int (*ctx_get_current_fn)(void **ctx);
typedef int (*ctx_get_id_fn)(void *ctx, unsigned long long *id);

constexpr int kCacheSlots = 64;
struct CacheSlot {
    unsigned long long ctx_id;
    void *ptr;
};
CacheSlot g_cache[kCacheSlots] = {};
int g_cache_next = 0;
std::mutex g_cache_mu;

// Unique id of the calling thread's current context, 0 if none is current.
int current_context_id(unsigned long long *id)
{
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return IDM_ERR_CUDA;
        }
        get_current = (ctx_get_current_fn)f1;
        get_id = (ctx_get_id_fn)f2;
    }
    void *ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != 0) return IDM_ERR_CUDA;
    if (ctx && get_id(ctx, id) != 0) return IDM_ERR_CUDA;
    return IDM_OK;
}

// Device address of the scratch array in the current context (set-up on the
// first call in each context: cudaGetSymbolAddress, which also makes the
// device's primary context current when none is).
int scratch_address(void **out)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    unsigned long long id = 0;
    if (current_context_id(&id)) return IDM_ERR_CUDA;
    if (id != 0)
        for (const CacheSlot &c : g_cache)
            if (c.ctx_id == id && c.ptr) {
                *out = c.ptr;
                return IDM_OK;
            }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return IDM_ERR_CUDA;
    }
    if (id == 0 && current_context_id(&id)) return IDM_ERR_CUDA;
    if (id != 0) {
        g_cache[g_cache_next] = CacheSlot{id, p};
        g_cache_next = (g_cache_next + 1) % kCacheSlots;
    }
    *out = p;
    return IDM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int idm_loss_grad_noalloc(const idm_scene_t *sc, const idm_params_t *pr, const float *p_init,
                                     const float *v_init, const idm_sim_t *sim, const float *targets,
                                     int32_t obs_stride, double *loss_out, idm_params_t *grad, float *grad_p_init,
                                     float *grad_v_init, uint32_t *status_out, void *stream)
{
    // launch plan with the context-free default kernel shape; a stack context provides
    // the argument checks and the planning helpers and is never allowed to
    // allocate (its ensure() fails instead)
    idm_ctx c;
    c.no_alloc = 1;
    int rc;
    // the argument checks of idm_loss_grad (host only, nothing launched on failure)
    if ((rc = check_scene(&c, sc)) || (rc = check_params(&c, pr, true, sc->n_vehicles)) || (rc = check_sim(&c, sim)))
        return rc;
    if (obs_stride < 1) return IDM_ERR_ARG;
    if (sc->n_vehicles > 0 && (!p_init || !v_init)) return IDM_ERR_ARG;
    if (sim->K / obs_stride > 0 && sc->n_vehicles > 0 && !targets) return IDM_ERR_ARG;

    if (cudaGetDevice(&c.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess)
        return IDM_ERR_CUDA;
    Prep P;
    if ((rc = pick_shape(&c, sc->max_lane, sc->n_vehicles, sc->n_lanes, &P.vpt, &P.G))) return rc;
    const size_t N = (size_t)sc->n_vehicles, L = (size_t)sc->n_lanes;
    const int G = P.G;
    const int C = std::min(c.C, sim->K);  // as idm_loss_grad: at most the horizon
    const size_t n_ck = (size_t)((sim->K + C - 1) / C);
    const bool totals = sim->K > idm::GSUM_FOLD_STEPS && N > 0;
    const long long cap = 32LL * P.vpt * G;
    const size_t totals_bytes =
        totals ? idm::gsum_bytes((size_t)std::min<long long>((long long)L, 2 * (((long long)N + cap - 1) / cap) +
                                                                               idm::SEG_BUILD_CHUNKS),
                                 (int)cap)
               : 0;

    // scratch layout (256-byte aligned pieces)
    size_t off = 0;
    const size_t o_ctl = off;  off += align256(sizeof(int) * CTL_N);
    const size_t o_stat = off; off += align256(sizeof(unsigned) * 4);
    const size_t o_seg = off;  off += align256(sizeof(Seg) * L);
    const size_t o_g0 = off;   off += align256(sizeof(float) * std::max<size_t>(N, 1));
    const size_t o_part = off; off += align256(sizeof(double) * L * G);
    const size_t o_loss = off; off += align256(sizeof(double) * 2);
    const size_t o_ckpt = off; off += align256(sizeof(float) * idm::STATE_ROWS * n_ck * std::max<size_t>(N, 1));
    const size_t o_gsum = off; off += align256(totals_bytes);
    if (off > (size_t)IDM_NOALLOC_SCRATCH_BYTES) return IDM_ERR_WORKSPACE;

    unsigned char *base = nullptr;
    if ((rc = scratch_address((void **)&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int *ctl = (int *)(base + o_ctl);
    unsigned *status = (unsigned *)(base + o_stat);

    SimArgs &a = P.a;
    memset(&a, 0, sizeof a);
    a.seg = (const Seg *)(base + o_seg);
    a.n_seg = ctl + CTL_NSEG;
    ScenDesc &s0 = a.scen0;
    s0.veh_begin = 0;
    s0.n_veh = (int)N;
    s0.K = sim->K;
    s0.obs_stride = obs_stride;
    s0.n_obs = sim->K / obs_stride;
    s0.dt = sim->dt;
    s0.inv_dt = 1.0f / sim->dt;
    s0.a_min = sim->a_min;
    s0.inv_nobs = s0.n_obs > 0 ? 1.0f / (float)s0.n_obs : 0.0f;
    a.g0 = (const float *)(base + o_g0);
    a.v0 = pr->v0; a.T = pr->T; a.s0 = pr->s0; a.am = pr->a_max; a.b = pr->b; a.delta = pr->delta;
    a.p_init = p_init;
    a.v_init = v_init;
    a.targets = targets;
    a.loss_part = (double *)(base + o_part);
    a.ckpt = (float *)(base + o_ckpt);
    a.C = C;
    a.status = status;
    a.N_total = (int)N;
    a.G = G;
    P.loss_per_seg = G;
    P.k_max = sim->K;
    // the gradient totals come from the scratch array: backward_grid finds
    // them present; any other buffer it would need (sub-checkpoints of a tape
    // shallower than the interval) makes it fail with IDM_ERR_WORKSPACE
    if (totals) {
        c.gsum.p = base + o_gsum;
        c.gsum.n = totals_bytes;
    }
    const bool want_delta = grad && grad->delta;
    if ((rc = forward_grid(&c, &P, (int)L))) return rc;
    if ((rc = backward_grid(&c, &P, false, false, want_delta, (int)L))) return rc;
    if (P.a.tape_T != C) return IDM_ERR_WORKSPACE;

    // the array keeps the previous call's contents: clear counters and status
    if (cudaMemsetAsync(base, 0, o_seg, st) != cudaSuccess) return IDM_ERR_CUDA;
    cudaError_t e = idm::launch_prep_gap(sc->lane_off, (int)L, p_init, sc->length, (int)N, (float *)(base + o_g0),
                                         status, st);
    if (e == cudaSuccess)
        e = idm::launch_build_segments(sc->lane_off, (int)L, nullptr, 0, 32 * P.vpt * G, (int)N, (Seg *)(base + o_seg),
                                       ctl + CTL_NSEG, status, st);
    if (e == cudaSuccess) {
        a.work = ctl + CTL_WORK_F;
        e = idm::launch_forward(P.vpt_f, P.G_f, false, false, true, a, P.grid_f, P.wpb_f, st);
    }
    if (e == cudaSuccess) {
        a.work = ctl + CTL_WORK_B;
        if (grad) {
            a.g_v0 = grad->v0; a.g_T = grad->T; a.g_s0 = grad->s0;
            a.g_am = grad->a_max; a.g_b = grad->b; a.g_delta = grad->delta;
        }
        a.g_p_init = grad_p_init;
        a.g_v_init = grad_v_init;
        e = idm::launch_backward(P.vpt, P.G, false, false, want_delta, a, P.grid_b, P.wpb_b, st);
    }
    if (e == cudaSuccess)
        e = idm::launch_loss_finalize(a.loss_part, a.n_seg, G, loss_out ? loss_out : (double *)(base + o_loss), st);
    if (e == cudaSuccess && status_out)
        e = cudaMemcpyAsync(status_out, status, sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IDM_ERR_CUDA;
    }
    return IDM_OK;
}
