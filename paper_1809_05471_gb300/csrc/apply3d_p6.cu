// 3D apply kernels of order p = 6. FP64: scalar kernel, tile 4, 2, 2 elements.
// FP32: packed FP32x2 kernel; tiles (4, 4, 2); (2, 2, 4), the first the default
// (fastest in a sweep of the shapes below on the order-sweep workload); more
// shapes are compiled under IGASF_TILE_SEARCH for such sweeps.
#include "apply3d.cuh"
#include "apply3d_f32.cuh"

namespace igasf {

int apply3d_p6(int prec, ApplyKernel *out, int max_out) {
  int n = 0;
  if (prec == IGASF_FP64) {
    if (n < max_out) out[n++] = make_apply3d<double, 6, 4, 2, 2>();
    return n;
  }
  if (n < max_out) out[n++] = make_apply3d_f32<6, 4, 4, 2>();
  if (n < max_out) out[n++] = make_apply3d_f32<6, 2, 2, 4>();
#ifdef IGASF_TILE_SEARCH
  if (n < max_out) out[n++] = make_apply3d_f32<6, 4, 2, 2>();
  if (n < max_out) out[n++] = make_apply3d_f32<6, 2, 2, 2>();
  if (n < max_out) out[n++] = make_apply3d_f32<6, 4, 4, 1>();
#endif
  return n;
}

}  // namespace igasf
