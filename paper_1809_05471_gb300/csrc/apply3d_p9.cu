// 3D apply kernels of order p = 9. Tile (elements): FP64 2, 1, 2, FP32 2, 2, 2.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p9(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 9, 2, 1, 2>() : make_apply3d<float, 9, 2, 2, 2>();
}

}  // namespace igasf
