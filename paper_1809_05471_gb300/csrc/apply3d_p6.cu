// 3D apply kernels of order p = 6. Tile (elements): FP64 4, 2, 2, FP32 4, 4, 2.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p6(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 6, 4, 2, 2>() : make_apply3d<float, 6, 4, 4, 2>();
}

}  // namespace igasf
