// 2D apply kernels for p = 6..9 (candidate lists in apply2d_list.cuh).
#include "apply2d_list.cuh"

namespace igasf {

int apply2d_list_hi(int p, int prec, ApplyKernel *out, int max_out) {
  switch (p) {
    case 6: return apply2d_candidates<6, 32, 4, 16, 8>(prec, out, max_out);
    case 7: return apply2d_candidates<7, 32, 4, 16, 4>(prec, out, max_out);
    case 8: return apply2d_candidates<8, 16, 4, 8, 4>(prec, out, max_out);
    default: return apply2d_candidates<9, 32, 4, 16, 4, true>(prec, out, max_out);
  }
}

}  // namespace igasf
