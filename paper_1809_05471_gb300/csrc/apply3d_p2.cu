// 3D apply kernels of order p = 2. FP64: scalar kernel, tile 8, 8, 8 elements.
// FP32 (packed FP32x2) candidates, the first the default (fastest in a sweep
// of tile shapes and factor-stream variants on the order-sweep workload);
// BF16 (bfloat16-stored factors) uses the same candidates unless a line names both:
//   register prefetch, tile 8, 8, 4
//   register prefetch, tile 8, 8, 2
//   TMA ring, tile 16, 8, 4
//   register prefetch, tile 2, 2, 1
// Register-prefetch kernels request their tile's factors into L2 at entry: FP32 no, BF16 no.
// IGASF_TILE_SEARCH compiles every listed shape in both variants.
// Tensor-core kernels (IGASF_TF32, IGASF_BF16_MMA): tile 8, 8, 4, 8 warps; tile 8, 8, 2, 8 warps.
// Factors evaluated on the fly (FP32): tile 8, 8, 2 first, then 8, 4, 4.
#include "apply3d.cuh"
#include "apply3d_f32.cuh"
#include "apply3d_f32g.cuh"
#include "apply3d_f32r.cuh"
#include "apply3d_tc.cuh"

namespace igasf {

int apply3d_p2(int prec, ApplyKernel *out, int max_out) {
  int n = 0;
  if (prec == IGASF_FP64) {
    if (n < max_out) out[n++] = make_apply3d<double, 2, 8, 8, 8>();
    return n;
  }
  if (tensor_core_prec(prec)) {
    const bool b = prec == IGASF_BF16_MMA;
    if (n < max_out) out[n++] = b ? make_apply3d_tc<2, 8, 8, 4, TC_BF16, 8, 2>() : make_apply3d_tc<2, 8, 8, 4, TC_TF32, 8, 2>();
    if (n < max_out) out[n++] = b ? make_apply3d_tc<2, 8, 8, 2, TC_BF16, 8, 2>() : make_apply3d_tc<2, 8, 8, 2, TC_TF32, 8, 2>();
    return n;
  }
  const bool bf = prec == IGASF_BF16;
#ifndef IGASF_TILE_SEARCH
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 8, 4, true, 2, 0, 0>() : make_apply3d_f32r<2, 8, 8, 4, false, 2, 0, 0>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 8, 2, true, 2, 0, 0>() : make_apply3d_f32r<2, 8, 8, 2, false, 2, 0, 0>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 16, 8, 4, true>() : make_apply3d_f32<2, 16, 8, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 2, 2, 1, true, 2, 0, 0>() : make_apply3d_f32r<2, 2, 2, 1, false, 2, 0, 0>();
#else
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 8, 4, true, 2, 0, 0>() : make_apply3d_f32r<2, 8, 8, 4, false, 2, 0, 0>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 8, 2, true>() : make_apply3d_f32r<2, 8, 8, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 16, 8, 4, true>() : make_apply3d_f32r<2, 16, 8, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 4, 8, true>() : make_apply3d_f32r<2, 8, 4, 8>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 8, 8, 8, true>() : make_apply3d_f32r<2, 8, 8, 8>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<2, 16, 8, 2, true>() : make_apply3d_f32r<2, 16, 8, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 8, 8, 2, true>() : make_apply3d_f32<2, 8, 8, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 8, 8, 4, true>() : make_apply3d_f32<2, 8, 8, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 16, 8, 4, true>() : make_apply3d_f32<2, 16, 8, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 8, 4, 8, true>() : make_apply3d_f32<2, 8, 4, 8>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 8, 8, 8, true>() : make_apply3d_f32<2, 8, 8, 8>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<2, 16, 8, 2, true>() : make_apply3d_f32<2, 16, 8, 2>();
#endif
  return n;
}

int apply3d_p2_geo(ApplyKernel *out, int max_out) {
  int n = 0;
  if (n < max_out) out[n++] = make_apply3d_f32g<2, 8, 8, 2, true>();
  if (n < max_out) out[n++] = make_apply3d_f32g<2, 8, 4, 4, true>();
  return n;
}

}  // namespace igasf
