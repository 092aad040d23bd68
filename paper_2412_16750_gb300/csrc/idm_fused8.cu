// Single-launch fit kernels with 8 vehicles per thread.
#include "idm_fused.cuh"

namespace idm {

void *fused_fn_vpt8(bool big, bool sub)
{
    (void)big;
    return fused_fn_t<8, false>(sub);
}

}  // namespace idm
