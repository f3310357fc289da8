// 3D apply kernels of order p = 7. FP64: scalar kernel, tile 2, 2, 2 elements.
// FP32 (packed FP32x2) candidates, the first the default (fastest in a sweep
// of tile shapes and factor-stream variants on the order-sweep workload);
// BF16 (bfloat16-stored factors) uses the same candidates unless a line names both:
//   FP32: register prefetch, tile 2, 2, 8, registers capped for 3 resident blocks, tables reloaded for the transposed sweep; BF16: register prefetch, tile 2, 2, 8
//   FP32: register prefetch, tile 2, 2, 6, registers capped for 3 resident blocks, tables reloaded for the transposed sweep; BF16: register prefetch, tile 2, 2, 6
//   TMA ring, tile 2, 2, 4, tables reloaded for the transposed sweep
//   register prefetch, tile 4, 2, 2
// Register-prefetch kernels request their tile's factors into L2 at entry: FP32 yes, BF16 yes.
// IGASF_TILE_SEARCH compiles every listed shape in both variants.
// Tensor-core kernels (IGASF_TF32, IGASF_BF16_MMA): tile 2, 2, 8, 7 warps; tile 2, 2, 6, 7 warps.
// Factors evaluated on the fly (FP32): tile 2, 2, 2 first, then 2, 2, 1.
#include "apply3d.cuh"
#include "apply3d_f32.cuh"
#include "apply3d_f32g.cuh"
#include "apply3d_f32r.cuh"
#include "apply3d_tc.cuh"

namespace igasf {

int apply3d_p7(int prec, ApplyKernel *out, int max_out) {
  int n = 0;
  if (prec == IGASF_FP64) {
    if (n < max_out) out[n++] = make_apply3d<double, 7, 2, 2, 2>();
    return n;
  }
  if (tensor_core_prec(prec)) {
    const bool b = prec == IGASF_BF16_MMA;
    if (n < max_out) out[n++] = b ? make_apply3d_tc<7, 2, 2, 8, TC_BF16, 7, 2>() : make_apply3d_tc<7, 2, 2, 8, TC_TF32, 7, 2>();
    if (n < max_out) out[n++] = b ? make_apply3d_tc<7, 2, 2, 6, TC_BF16, 7, 2>() : make_apply3d_tc<7, 2, 2, 6, TC_TF32, 7, 2>();
    return n;
  }
  const bool bf = prec == IGASF_BF16;
#ifndef IGASF_TILE_SEARCH
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 8, true, 2, 0, 2>() : make_apply3d_f32r<7, 2, 2, 8, false, 2, 3, 3>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 6, true, 2, 0, 2>() : make_apply3d_f32r<7, 2, 2, 6, false, 2, 3, 3>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 2, 2, 4, true, true>() : make_apply3d_f32<7, 2, 2, 4, false, true>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 4, 2, 2, true, 2, 0, 2>() : make_apply3d_f32r<7, 4, 2, 2, false, 2, 0, 2>();
#else
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 8, true, 2, 0, 2>() : make_apply3d_f32r<7, 2, 2, 8, false, 2, 3, 3>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 6, true>() : make_apply3d_f32r<7, 2, 2, 6>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 4, true>() : make_apply3d_f32r<7, 2, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 4, 2, 4, true>() : make_apply3d_f32r<7, 4, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 4, 2, 2, true>() : make_apply3d_f32r<7, 4, 2, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<7, 2, 2, 2, true>() : make_apply3d_f32r<7, 2, 2, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 2, 2, 8, true>() : make_apply3d_f32<7, 2, 2, 8>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 2, 2, 6, true>() : make_apply3d_f32<7, 2, 2, 6>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 2, 2, 4, true>() : make_apply3d_f32<7, 2, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 4, 2, 4, true>() : make_apply3d_f32<7, 4, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 4, 2, 2, true>() : make_apply3d_f32<7, 4, 2, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<7, 2, 2, 2, true>() : make_apply3d_f32<7, 2, 2, 2>();
#endif
  return n;
}

int apply3d_p7_geo(ApplyKernel *out, int max_out) {
  int n = 0;
  if (n < max_out) out[n++] = make_apply3d_f32g<7, 2, 2, 2, false>();
  if (n < max_out) out[n++] = make_apply3d_f32g<7, 2, 2, 1, false>();
  return n;
}

}  // namespace igasf
