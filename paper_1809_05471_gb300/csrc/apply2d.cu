// 2D apply kernels for p = 2..9 (FP64, FP32, and FP32 with bfloat16-stored
// factors); tile = 8 x 8 elements.
#include "apply2d.cuh"

namespace igasf {

template <int P>
static ApplyKernel get2(int prec) {
  if (prec == IGASF_FP64) return make_apply2d<double, P, 8, 8>();
  if (prec == IGASF_FP32) return make_apply2d<float, P, 8, 8>();
  return make_apply2d<float, P, 8, 8, __nv_bfloat16>();
}

ApplyKernel apply2d_any(int p, int prec) {
  switch (p) {
    case 2: return get2<2>(prec);
    case 3: return get2<3>(prec);
    case 4: return get2<4>(prec);
    case 5: return get2<5>(prec);
    case 6: return get2<6>(prec);
    case 7: return get2<7>(prec);
    case 8: return get2<8>(prec);
    default: return get2<9>(prec);
  }
}

}  // namespace igasf
