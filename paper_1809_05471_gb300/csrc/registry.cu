// Lookup of the compiled apply kernels by (d, p, precision).
#include "igasf_internal.h"

namespace igasf {

ApplyKernel apply3d_p2(int prec);
ApplyKernel apply3d_p3(int prec);
ApplyKernel apply3d_p4(int prec);
ApplyKernel apply3d_p5(int prec);
ApplyKernel apply3d_p6(int prec);
ApplyKernel apply3d_p7(int prec);
ApplyKernel apply3d_p8(int prec);
ApplyKernel apply3d_p9(int prec);
ApplyKernel apply2d_any(int p, int prec);

bool find_apply_kernel(int d, int p, int prec, ApplyKernel *out) {
  if (prec != IGASF_FP64 && prec != IGASF_FP32) return false;
  if (p < 2 || p > IGASF_MAX_ORDER) return false;
  if (d == 2) {
    *out = apply2d_any(p, prec);
    return true;
  }
  if (d != 3) return false;
  switch (p) {
    case 2: *out = apply3d_p2(prec); return true;
    case 3: *out = apply3d_p3(prec); return true;
    case 4: *out = apply3d_p4(prec); return true;
    case 5: *out = apply3d_p5(prec); return true;
    case 6: *out = apply3d_p6(prec); return true;
    case 7: *out = apply3d_p7(prec); return true;
    case 8: *out = apply3d_p8(prec); return true;
    case 9: *out = apply3d_p9(prec); return true;
  }
  return false;
}

}  // namespace igasf
