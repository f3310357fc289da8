// 3D apply kernels of order p = 7. Tile (elements): FP64 2, 2, 2, FP32 4, 2, 2.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p7(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 7, 2, 2, 2>() : make_apply3d<float, 7, 4, 2, 2>();
}

}  // namespace igasf
