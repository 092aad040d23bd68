// Single-launch fit kernels with 2 vehicles per thread.
#include "idm_fused.cuh"

namespace idm {

void *fused_fn_vpt2(bool big, bool sub)
{
    (void)big;
    return fused_fn_t<2, false>(sub);
}

}  // namespace idm
