// idm_loss_grad_noalloc: the fused loss + gradient of idm_loss_grad for
// callers that cannot allocate device memory.  Examples are code running inside
// a CUDA-graph capture that forbids cudaMalloc, a host with a custom
// allocator that owns all device memory, or an embedding with a fixed memory
// budget checked up front.
//
// All scratch (warp segments, control counters, status word, initial gaps,
// per-warp loss partials, checkpoints) lives in one file-scope device array of
// IDM_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that
// array until the process exits.  Host code must not pass the array's name
// to a kernel: on the host the name is only a stand-in for the symbol.  The
// device address is obtained once per device with cudaGetSymbolAddress and
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

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IDM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return IDM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return IDM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return IDM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int idm_loss_grad_noalloc(const idm_scene_t *sc, const idm_params_t *pr, const float *p_init,
                                     const float *v_init, const idm_sim_t *sim, const float *targets,
                                     int32_t obs_stride, double *loss_out, idm_params_t *grad, float *grad_p_init,
                                     float *grad_v_init, uint32_t *status_out, void *stream)
{
    // argument checks (host only, nothing launched on failure)
    if (!sc || !pr || !sim) return IDM_ERR_ARG;
    if (sc->n_lanes < 1 || sc->n_vehicles < 0 || !sc->lane_off) return IDM_ERR_ARG;
    if (sc->n_vehicles > 0 && (!sc->length || !p_init || !v_init)) return IDM_ERR_ARG;
    if (sc->max_lane < 0 || sc->max_lane > idm_max_lane_supported()) return IDM_ERR_ARG;
    if (!pr->v0 || !pr->T || !pr->s0 || !pr->a_max || !pr->b || !pr->delta) return IDM_ERR_ARG;
    if (sim->K < 1 || !(sim->dt > 0.0f) || !(sim->a_min < 0.0f)) return IDM_ERR_ARG;
    if (obs_stride < 1) return IDM_ERR_ARG;
    if (sim->K / obs_stride > 0 && sc->n_vehicles > 0 && !targets) return IDM_ERR_ARG;

    // launch plan with the default kernel shape; a stack context provides
    // the planning helpers and is never asked to allocate
    idm_ctx c;
    if (cudaGetDevice(&c.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess)
        return IDM_ERR_CUDA;
    Prep P;
    int rc;
    if ((rc = pick_shape(&c, sc->max_lane, &P.vpt, &P.G))) return rc;
    const size_t N = (size_t)sc->n_vehicles, L = (size_t)sc->n_lanes;
    const int G = P.G;
    const int C = std::min(c.C, sim->K);  // as idm_loss_grad: at most the horizon
    const size_t n_ck = (size_t)((sim->K + C - 1) / C);

    // scratch layout (256-byte aligned pieces)
    size_t off = 0;
    const size_t o_ctl = off;  off += align256(sizeof(int) * CTL_N);
    const size_t o_stat = off; off += align256(sizeof(unsigned) * 4);
    const size_t o_seg = off;  off += align256(sizeof(Seg) * L);
    const size_t o_g0 = off;   off += align256(sizeof(float) * std::max<size_t>(N, 1));
    const size_t o_part = off; off += align256(sizeof(double) * L * G);
    const size_t o_loss = off; off += align256(sizeof(double) * 2);
    const size_t o_ckpt = off; off += align256(sizeof(float) * 4 * n_ck * std::max<size_t>(N, 1));
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
    const bool want_delta = grad && grad->delta;
    if ((rc = forward_grid(&c, &P, (int)L))) return rc;
    if ((rc = backward_grid(&c, &P, false, false, want_delta, (int)L))) return rc;
    if (P.a.tape_T != C) return IDM_ERR_WORKSPACE;  // would need sub-checkpoint scratch

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
