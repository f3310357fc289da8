// The plan behind an igasf_handle (shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "igasf_internal.h"

namespace igasf {

// Kernel, layout, tables and workspace of one stored precision.
struct Variant {
  bool present = false;
  ApplyKernel k{};
  FactorLayout L{};
  void *tabB[kMaxDim] = {nullptr, nullptr, nullptr};
  void *tabD[kMaxDim] = {nullptr, nullptr, nullptr};
  int T[kMaxDim] = {1, 1, 1};
  int Qpad[kMaxDim] = {0, 0, 0};
  int ntiles = 0;
  size_t bytesM = 0, bytesK = 0;
  void *vpart = nullptr;
  size_t vpart_bytes = 0;
  void *u_stage = nullptr, *v_stage = nullptr;
  void *u_stage2 = nullptr;                 // second input buffer of igasf_apply_host_async
  int2 *gtab[kMaxDim] = {nullptr, nullptr, nullptr};   // gather tables, see gather_table
  // factors evaluated on the fly (FP32 only): no stored factors
  bool on_the_fly = false;
  float *ctrl32 = nullptr;                            // SoA [3][N]
  float *wq32[kMaxDim] = {nullptr, nullptr, nullptr}; // [Qpad]
};

}  // namespace igasf

struct igasf_plan {
  int d = 0, p = 0, device = 0;
  // Elements are all knot spans [t_k, t_k+1), k = p-1 .. nk-p-1, empty ones
  // included, so that the first function of element e is e in every
  // direction; an empty span has zero weights, tables and factors and adds
  // nothing. K, Q and Qtot count these elements; the API's quadrature points
  // (num_quad_points, tables, factors, points, per-point coefficients) are
  // those of the non-empty spans only: Ke per direction, Qapi in all, with
  // elem[a][i] the element of the i-th non-empty span.
  int N[igasf::kMaxDim] = {1, 1, 1}, K[igasf::kMaxDim] = {1, 1, 1}, Q[igasf::kMaxDim] = {1, 1, 1};
  int64_t Ntot = 0, Qtot = 0;
  int Ke[igasf::kMaxDim] = {1, 1, 1};
  int64_t Qapi = 0;
  bool empty_spans = false;
  std::vector<int> elem[igasf::kMaxDim];
  std::vector<unsigned char> nonempty[igasf::kMaxDim];   // per element: 1 if its span is non-empty
  double *knots[igasf::kMaxDim] = {nullptr, nullptr, nullptr};
  int *span[igasf::kMaxDim] = {nullptr, nullptr, nullptr};
  double *nodes[igasf::kMaxDim] = {nullptr, nullptr, nullptr};
  double *weights[igasf::kMaxDim] = {nullptr, nullptr, nullptr};
  double *tabB[igasf::kMaxDim] = {nullptr, nullptr, nullptr};  // FP64 [j][Q]
  double *tabD[igasf::kMaxDim] = {nullptr, nullptr, nullptr};
  double *ctrl64 = nullptr;              // control points, device, N x d (for igasf_quad_points)
  int default_prec = IGASF_FP64;
  igasf::Variant var[igasf::kNumPrec];
  unsigned int *status = nullptr;        // device status word (bounded waits)
  long long wait_limit = 2000000000LL;   // about one second at 2 GHz
  int skip_slab = -1;                    // test hook, see igasf_set_test_fault
  std::vector<cudaEvent_t> prof_events;  // 3 per timed apply
  int prof_next = 0;                     // applies recorded so far
  // igasf_apply_host_async: copies into the two input buffers run on their own
  // stream, ordered against the applies by events
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int stage_next = 0;
  double *dinv64 = nullptr;              // inverse Jacobi diagonal of K (solver), lazily
  float *dinv32 = nullptr;
  int coef_kind = IGASF_COEF_CONSTANT;   // for factors evaluated on the fly
  double coef_constant = 1.0, coef_alpha = 0.0;
};

namespace igasf {
// Arguments of one tile-kernel launch of the plan's precision `var` (capi.cu).
void make_apply_params(const igasf_plan *h, const Variant &var, int op, const void *u, void *vpart,
                       ApplyParams *prm);
}  // namespace igasf
