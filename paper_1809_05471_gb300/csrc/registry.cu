// Lookup of the compiled apply kernels by (d, p, precision, tile shape).
#include "igasf_internal.h"

namespace igasf {

int apply3d_p2(int prec, ApplyKernel *out, int max_out);
int apply3d_p3(int prec, ApplyKernel *out, int max_out);
int apply3d_p4(int prec, ApplyKernel *out, int max_out);
int apply3d_p5(int prec, ApplyKernel *out, int max_out);
int apply3d_p6(int prec, ApplyKernel *out, int max_out);
int apply3d_p7(int prec, ApplyKernel *out, int max_out);
int apply3d_p8(int prec, ApplyKernel *out, int max_out);
int apply3d_p9(int prec, ApplyKernel *out, int max_out);
int apply3d_p2_geo(ApplyKernel *out, int max_out);
int apply3d_p3_geo(ApplyKernel *out, int max_out);
int apply3d_p4_geo(ApplyKernel *out, int max_out);
int apply3d_p5_geo(ApplyKernel *out, int max_out);
int apply3d_p6_geo(ApplyKernel *out, int max_out);
int apply3d_p7_geo(ApplyKernel *out, int max_out);
int apply3d_p8_geo(ApplyKernel *out, int max_out);
int apply3d_p9_geo(ApplyKernel *out, int max_out);
int apply2d_list(int p, int prec, ApplyKernel *out, int max_out);

int list_apply_kernels(int d, int p, int prec, ApplyKernel *out, int max_out) {
  if (prec < 0 || prec >= kNumPrec) return 0;
  if (p < 2 || p > IGASF_MAX_ORDER || max_out < 1) return 0;
  if (d == 2) return tensor_core_prec(prec) ? 0 : apply2d_list(p, prec, out, max_out);
  if (d != 3) return 0;
  switch (p) {
    case 2: return apply3d_p2(prec, out, max_out);
    case 3: return apply3d_p3(prec, out, max_out);
    case 4: return apply3d_p4(prec, out, max_out);
    case 5: return apply3d_p5(prec, out, max_out);
    case 6: return apply3d_p6(prec, out, max_out);
    case 7: return apply3d_p7(prec, out, max_out);
    case 8: return apply3d_p8(prec, out, max_out);
    case 9: return apply3d_p9(prec, out, max_out);
  }
  return 0;
}

bool find_apply_kernel(int d, int p, int prec, const int *tile, int variant, ApplyKernel *out) {
  ApplyKernel cand[kMaxCandidates];
  const int n = list_apply_kernels(d, p, prec, cand, kMaxCandidates);
  if (n == 0) return false;
  bool any = false;
  for (int a = 0; a < d; ++a) any = any || (tile && tile[a] != 0);
  any = any || variant != 0;
  if (!any) {
    *out = cand[0];
    return true;
  }
  for (int i = 0; i < n; ++i) {
    bool ok = variant == 0 || variant == cand[i].variant;
    for (int a = 0; a < d && tile; ++a)
      if (tile[a] != 0 && tile[a] != cand[i].S[a]) ok = false;
    if (ok) {
      *out = cand[i];
      return true;
    }
  }
  return false;
}

int list_geometry_kernels(int p, ApplyKernel *out, int max_out) {
  if (max_out < 1) return 0;
  switch (p) {
    case 2: return apply3d_p2_geo(out, max_out);
    case 3: return apply3d_p3_geo(out, max_out);
    case 4: return apply3d_p4_geo(out, max_out);
    case 5: return apply3d_p5_geo(out, max_out);
    case 6: return apply3d_p6_geo(out, max_out);
    case 7: return apply3d_p7_geo(out, max_out);
    case 8: return apply3d_p8_geo(out, max_out);
    case 9: return apply3d_p9_geo(out, max_out);
  }
  return 0;
}

bool find_geometry_kernel(int p, const int *tile, ApplyKernel *out) {
  ApplyKernel cand[kMaxCandidates];
  const int n = list_geometry_kernels(p, cand, kMaxCandidates);
  for (int i = 0; i < n; ++i) {
    bool ok = true;
    for (int a = 0; a < 3 && tile; ++a)
      if (tile[a] != 0 && tile[a] != cand[i].S[a]) ok = false;
    if (ok) {
      *out = cand[i];
      return true;
    }
  }
  return false;
}

}  // namespace igasf
