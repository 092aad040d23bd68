// Adjoint kernels with 2 vehicles per thread.
#include "idm_adjoint.cuh"

namespace idm {

void *backward_fn_vpt2(bool dense, bool adam, bool wd, bool big, bool sub)
{
    (void)big;
    return sub ? backward_fn_t<2, false, true>(dense, adam, wd) : backward_fn_t<2, false, false>(dense, adam, wd);
}

}  // namespace idm
