// 3D apply kernels of order p = 2. Tile (elements): FP64 8, 8, 8, FP32 8, 8, 8.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p2(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 2, 8, 8, 8>() : make_apply3d<float, 2, 8, 8, 8>();
}

}  // namespace igasf
