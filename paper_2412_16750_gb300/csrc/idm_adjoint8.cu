// Adjoint kernels with 8 vehicles per thread.
#include "idm_adjoint.cuh"

namespace idm {

void *backward_fn_vpt8(bool dense, bool adam, bool wd, bool big, bool sub)
{
    (void)big;
    return sub ? backward_fn_t<8, false, true>(dense, adam, wd) : backward_fn_t<8, false, false>(dense, adam, wd);
}

}  // namespace idm
