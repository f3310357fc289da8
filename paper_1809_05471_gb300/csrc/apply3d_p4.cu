// 3D apply kernels of order p = 4. Tile (elements): FP64 4, 4, 4, FP32 4, 4, 4.
#include "apply3d.cuh"

namespace igasf {

ApplyKernel apply3d_p4(int prec) {
  return prec == IGASF_FP64 ? make_apply3d<double, 4, 4, 4, 4>() : make_apply3d<float, 4, 4, 4, 4>();
}

}  // namespace igasf
