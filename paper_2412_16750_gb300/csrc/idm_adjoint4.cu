// Adjoint kernels with 4 vehicles per thread.
#include "idm_adjoint.cuh"

namespace idm {

void *backward_fn_vpt4(bool dense, bool adam, bool wd, bool big, bool sub)
{
    if (sub) return big ? backward_fn_t<4, true, true>(dense, adam, wd) : backward_fn_t<4, false, true>(dense, adam, wd);
    return big ? backward_fn_t<4, true, false>(dense, adam, wd) : backward_fn_t<4, false, false>(dense, adam, wd);
}

}  // namespace idm
