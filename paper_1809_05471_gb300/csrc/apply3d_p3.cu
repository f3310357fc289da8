// 3D apply kernels of order p = 3. Tile (elements): FP64 8, 4, 4, FP32 8, 8, 4.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p3(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 3, 8, 4, 4>() : make_apply3d<float, 3, 8, 8, 4>();
}

}  // namespace igasf
