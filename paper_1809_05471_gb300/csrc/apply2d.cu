// 2D apply kernels for p = 2..5 (candidate lists in apply2d_list.cuh); the
// dispatch over all orders.
#include "apply2d_list.cuh"

namespace igasf {

int apply2d_list_hi(int p, int prec, ApplyKernel *out, int max_out);

int apply2d_list(int p, int prec, ApplyKernel *out, int max_out) {
  switch (p) {
    case 2: return apply2d_candidates<2, 32, 8, 64, 8>(prec, out, max_out);
    case 3: return apply2d_candidates<3, 64, 8, 32, 8>(prec, out, max_out);
    case 4: return apply2d_candidates<4, 16, 8, 32, 8>(prec, out, max_out);
    case 5: return apply2d_candidates<5, 32, 8, 64, 4>(prec, out, max_out);
    default: return apply2d_list_hi(p, prec, out, max_out);
  }
}

}  // namespace igasf
