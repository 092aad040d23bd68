// Forward, adjoint and single-launch fit kernels with 2 vehicles per thread and 4
// warp(s) per segment.
#include "idm_fused.cuh"

namespace idm {

IDM_DEFINE_SHAPE_KERNELS(2, 4)

}  // namespace idm
