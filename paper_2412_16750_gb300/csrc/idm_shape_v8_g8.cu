// Forward, adjoint and single-launch fit kernels with 8 vehicles per thread and 8
// warp(s) per segment.
#include "idm_fused.cuh"

namespace idm {

IDM_DEFINE_SHAPE_KERNELS(8, 8)

}  // namespace idm
