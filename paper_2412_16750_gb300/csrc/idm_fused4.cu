// Single-launch fit kernels with 4 vehicles per thread.
#include "idm_fused.cuh"

namespace idm {

void *fused_fn_vpt4(bool big, bool sub)
{
    if (big) return fused_fn_t<4, true>(sub);
    return fused_fn_t<4, false>(sub);
}

}  // namespace idm
