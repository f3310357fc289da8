// Candidate lists of the 2D kernels (apply2d.cu, apply2d_hi.cu). FP64: the
// scalar kernel, tile 8 x 8 elements. FP32 and BF16 (bfloat16-stored factors):
// the packed FP32x2 kernel with two tile shapes per order (the first the
// default: wide along direction 1 so a block holds at least one warp of pencil
// pairs), then the scalar kernel (first at p = 9).
#pragma once

#include "apply2d.cuh"
#include "apply2d_f32.cuh"

namespace igasf {

// SCALAR_FIRST: the scalar kernel is the default (measured faster at p = 9).
template <int P, int A1, int A2, int B1, int B2, bool SCALAR_FIRST = false>
int apply2d_candidates(int prec, ApplyKernel *out, int max_out) {
  int n = 0;
  if (prec == IGASF_FP64) {
    if (n < max_out) out[n++] = make_apply2d<double, P, 8, 8>();
    return n;
  }
  const bool bf = prec == IGASF_BF16;
  auto scalar = [&]() {
    if (n < max_out)
      out[n++] = bf ? make_apply2d<float, P, 8, 8, __nv_bfloat16>() : make_apply2d<float, P, 8, 8>();
  };
  if (SCALAR_FIRST) scalar();
  if (n < max_out) out[n++] = bf ? make_apply2d_f32<P, A1, A2, true>() : make_apply2d_f32<P, A1, A2>();
  if (n < max_out) out[n++] = bf ? make_apply2d_f32<P, B1, B2, true>() : make_apply2d_f32<P, B1, B2>();
  if (!SCALAR_FIRST) scalar();
  return n;
}

}  // namespace igasf
