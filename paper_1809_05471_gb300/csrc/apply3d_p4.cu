// 3D apply kernels of order p = 4. FP64: scalar kernel, tile 4, 4, 4 elements.
// FP32 (packed FP32x2) candidates, the first the default (fastest in a sweep
// of tile shapes and factor-stream variants on the order-sweep workload);
// BF16 (bfloat16-stored factors) uses the same candidates unless a line names both:
//   FP32: register prefetch, tile 4, 4, 4, registers capped for 4 resident blocks (mass 6, FP32), tables reloaded for the transposed sweep; BF16: register prefetch, tile 4, 4, 8
//   FP32: register prefetch, tile 4, 4, 8, registers capped for 4 resident blocks (mass 6, FP32), tables reloaded for the transposed sweep; BF16: register prefetch, tile 4, 4, 4
//   TMA ring, tile 8, 4, 2
//   TMA ring, tile 4, 4, 4
//   register prefetch, tile 4, 4, 1
// Register-prefetch kernels request their tile's factors into L2 at entry: FP32 no, BF16 yes.
// IGASF_TILE_SEARCH compiles every listed shape in both variants.
// Tensor-core kernels (IGASF_TF32, IGASF_BF16_MMA): tile 4, 4, 4, 8 warps; tile 4, 4, 8, 8 warps.
// Factors evaluated on the fly (FP32): tile 4, 4, 2 first, then 4, 4, 4.
#include "apply3d.cuh"
#include "apply3d_f32.cuh"
#include "apply3d_f32g.cuh"
#include "apply3d_f32r.cuh"
#include "apply3d_tc.cuh"

namespace igasf {

int apply3d_p4(int prec, ApplyKernel *out, int max_out) {
  int n = 0;
  if (prec == IGASF_FP64) {
    if (n < max_out) out[n++] = make_apply3d<double, 4, 4, 4, 4>();
    return n;
  }
  if (tensor_core_prec(prec)) {
    const bool b = prec == IGASF_BF16_MMA;
    if (n < max_out) out[n++] = b ? make_apply3d_tc<4, 4, 4, 4, TC_BF16, 8, 2>() : make_apply3d_tc<4, 4, 4, 4, TC_TF32, 8, 2>();
    if (n < max_out) out[n++] = b ? make_apply3d_tc<4, 4, 4, 8, TC_BF16, 8, 2>() : make_apply3d_tc<4, 4, 4, 8, TC_TF32, 8, 2>();
    return n;
  }
  const bool bf = prec == IGASF_BF16;
#ifndef IGASF_TILE_SEARCH
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 4, 8, true, 2, 0, 2>() : make_apply3d_f32r<4, 4, 4, 4, false, 2, 4, 1, 6>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 4, 4, true, 2, 0, 2>() : make_apply3d_f32r<4, 4, 4, 8, false, 2, 4, 1, 6>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 8, 4, 2, true>() : make_apply3d_f32<4, 8, 4, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 4, 4, 4, true>() : make_apply3d_f32<4, 4, 4, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 4, 1, true, 2, 0, 2>() : make_apply3d_f32r<4, 4, 4, 1, false, 2, 0, 0>();
#else
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 4, 8, true, 2, 0, 2>() : make_apply3d_f32r<4, 4, 4, 4, false, 2, 4, 1, 6>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 2, 4, true>() : make_apply3d_f32r<4, 4, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 8, 4, 4, true>() : make_apply3d_f32r<4, 8, 4, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 8, 4, 2, true>() : make_apply3d_f32r<4, 8, 4, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 2, 2, 4, true>() : make_apply3d_f32r<4, 2, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32r<4, 4, 4, 2, true>() : make_apply3d_f32r<4, 4, 4, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 4, 4, 4, true>() : make_apply3d_f32<4, 4, 4, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 4, 2, 4, true>() : make_apply3d_f32<4, 4, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 8, 4, 4, true>() : make_apply3d_f32<4, 8, 4, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 8, 4, 2, true>() : make_apply3d_f32<4, 8, 4, 2>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 2, 2, 4, true>() : make_apply3d_f32<4, 2, 2, 4>();
  if (n < max_out) out[n++] = bf ? make_apply3d_f32<4, 4, 4, 2, true>() : make_apply3d_f32<4, 4, 4, 2>();
#endif
  return n;
}

int apply3d_p4_geo(ApplyKernel *out, int max_out) {
  int n = 0;
  if (n < max_out) out[n++] = make_apply3d_f32g<4, 4, 4, 2, true>();
  if (n < max_out) out[n++] = make_apply3d_f32g<4, 4, 4, 4, true>();
  return n;
}

}  // namespace igasf
