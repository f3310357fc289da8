// 3D apply kernels of order p = 5. Tile (elements): FP64 4, 2, 2, FP32 4, 4, 4.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p5(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 5, 4, 2, 2>() : make_apply3d<float, 5, 4, 4, 4>();
}

}  // namespace igasf
