// Forward, adjoint and single-launch fit kernels with 2 vehicles per thread and 2
// warp(s) per segment.
#include "idm_fused.cuh"

namespace idm {

IDM_DEFINE_SHAPE_KERNELS(2, 2)

}  // namespace idm
