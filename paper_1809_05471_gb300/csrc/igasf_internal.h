// Internal declarations shared by the CUDA translation units of libigasf.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "igasf.h"

namespace igasf {

// Records the message of the last error (thread-local) and returns code.
int set_error(int code, const char *msg);

// C-ABI entry points that use standard containers end in this handler of a
// function-try-block, so that a failed host allocation returns IGASF_ERR_OOM
// instead of letting an exception cross the C boundary.
#define IGASF_CATCH_HOST                                                          \
  catch (const std::bad_alloc &) {                                                \
    return igasf::set_error(IGASF_ERR_OOM, "host allocation failed");             \
  }                                                                               \
  catch (...) {                                                                   \
    return igasf::set_error(IGASF_ERR_INVALID_ARG, "unexpected host exception");  \
  }

constexpr int kMaxDim = 3;
constexpr int kNumPrec = 5;        // FP64, FP32, BF16, TF32, BF16_MMA
constexpr int kFieldsK3 = 6;       // 11 12 13 22 23 33
constexpr int kFieldsK2 = 3;       // 11 12 22

inline int num_fields(int d, int op) { return op == IGASF_MASS ? 1 : (d == 3 ? kFieldsK3 : kFieldsK2); }

// Vectors and tables are double for FP64 and float otherwise; factors are
// stored as double, float or bfloat16.
inline bool vectors_are_float(int prec) { return prec != IGASF_FP64; }
inline size_t vector_bytes(int prec) { return prec == IGASF_FP64 ? 8 : 4; }
inline int factor_bytes(int prec) {
  return prec == IGASF_FP64 ? 8 : ((prec == IGASF_FP32 || prec == IGASF_TF32) ? 4 : 2);
}
// Precisions whose direction-3 contractions run on the tensor cores (3D only).
inline bool tensor_core_prec(int prec) { return prec == IGASF_TF32 || prec == IGASF_BF16_MMA; }

#ifdef __CUDACC__
// Programmatic dependent launch: a tile kernel lets the gather that follows it
// on the stream be scheduled once every tile block has started; the gather
// waits for the tile kernel's completion (and its memory) before reading.
// Both are no-ops when the launch carries no programmatic dependency.
__device__ __forceinline__ void pdl_allow_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_primary() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Arguments of one apply launch; pointers are device addresses in the
// precision of the kernel (float or double).
struct ApplyParams {
  const void *u;
  void *vpart;                // per-tile partial v, [tile][E_d]..[E_1]
  const void *D;              // factors of the op, tile-major (see FactorLayout)
  const void *tabB[kMaxDim];  // per direction [j][Qpad]: values of active function j
  const void *tabD[kMaxDim];  // derivatives, same layout
  int N[kMaxDim];             // dofs per direction
  int K[kMaxDim];             // elements per direction
  int T[kMaxDim];             // tiles per direction
  int Qpad[kMaxDim];          // T * S * p: row stride of the tables
  int ntiles;
  unsigned int *status;       // device word: bit 0 set when a bounded wait ran out
  long long wait_limit;       // clock cycles a kernel may wait on one mbarrier phase
  int skip_slab;              // test hook: tile 0 never fills this factor slab (-1: off)
  // factors evaluated on the fly (D unused): control points SoA [3][N],
  // Gauss weights per direction padded like the tables, coefficient
  const float *ctrl;
  const float *wq[kMaxDim];
  int coef_kind;              // IGASF_COEF_CONSTANT or IGASF_COEF_EXP_SIN_COS
  float coef_a;               // the constant, or alpha
};

// Many patches' tiles in one launch (device arrays): params[patch], and for
// every block its patch and the patch's first block.
struct BatchParams {
  const ApplyParams *params;
  const int *block_patch;
  const int *first_block;
};

// A compiled apply kernel for one (d, p, precision) and its tile shape.
struct ApplyKernel {
  int S[kMaxDim];             // elements per tile
  int threads;                // block size
  size_t smem[2];             // dynamic shared memory, [op]
  int plane;                  // padded pencils per slab (the factor layout's row length)
  int lanes;                  // pencils per thread (1, or 2 for packed FP32x2)
  int variant;                // IGASF_KERNEL_* (which factor-stream scheme)
  cudaError_t (*launch[2])(const ApplyParams &, cudaStream_t);
  // batched launch over `blocks` tiles of several patches (nullptr if not built)
  cudaError_t (*launch_batched[2])(const BatchParams &, int blocks, cudaStream_t);
  cudaError_t (*prepare)();   // raise the dynamic shared memory limit once
};

constexpr int kMaxCandidates = 16;  // compiled shapes per (d, p, precision)

// The compiled kernels for (d, p, prec), default first; returns how many.
int list_apply_kernels(int d, int p, int prec, ApplyKernel *out, int max_out);
// The default kernel (tile all zero or NULL, variant 0) or the first one whose
// tile matches every non-zero entry of `tile` and whose variant matches a
// non-zero `variant`; false if none is built.
bool find_apply_kernel(int d, int p, int prec, const int *tile, int variant, ApplyKernel *out);
// FP32 3D kernels that evaluate the factors on the fly (default first).
int list_geometry_kernels(int p, ApplyKernel *out, int max_out);
bool find_geometry_kernel(int p, const int *tile, ApplyKernel *out);

// Tile-major layout of the factors (see layout.h for the exact order).
struct FactorLayout {
  int d, p;
  int S[kMaxDim];
  int T[kMaxDim];
  int plane;
  int lanes;
  int elem_bytes;             // 8 (double), 4 (float) or 2 (bfloat16)
  void *DM;                   // mass factors (1 field)
  void *DK;                   // stiffness factors (num_fields)
};

struct GeometryParams {
  int d, p;
  int N[kMaxDim], K[kMaxDim];
  const double *ctrl;                 // N x d
  const double *tabB[kMaxDim];        // FP64 [j][K*p]
  const double *tabD[kMaxDim];
  const double *wq[kMaxDim];          // [K*p]
  int coef_kind;
  double coef_const, coef_alpha;
  const double *coef_values;          // device, lexicographic quadrature order
  int nout;
  FactorLayout out[kNumPrec];
  unsigned int *bad_det;              // set to 1 if det J <= 0 somewhere
  double *min_det;                    // unused if NULL
  double *xq_out;                     // if not NULL: G(x_q), [Qtot][d] lexicographic
};

// setup kernels (setup.cu)
cudaError_t launch_tables(int p, int K, const double *knots, const int *span, double *nodes,
                          double *weights, double *tabB, double *tabD, cudaStream_t s);
cudaError_t launch_geometry(const GeometryParams &g, cudaStream_t s);
cudaError_t launch_pad_tables(int p, int K, int Qpad, const double *src, void *dst, int to_float,
                              cudaStream_t s);
cudaError_t launch_export_factors(const FactorLayout &L, int op, int64_t Qtot, const int *Q,
                                  double *out, cudaStream_t s);
// gtab: per direction the table of gather_table (device, N_a entries; one
// entry {0, 1 << 16} for directions beyond d)
cudaError_t launch_gather(int d, int float_vectors, const void *vpart, void *v, const int *N,
                          const int *T, const int *S, int p, int2 *const *gtab, cudaStream_t s);
void gather_table(int N, int S, int E, int T, std::vector<int2> &out);
// The persistent batch kernel (batch_persistent.cu): the tile shape it runs for
// order p in precision prec (false if none), its grid on the current device,
// and its launch over a work list of (patch, tile) items.
bool persistent_tile(int p, int prec, int *S);
cudaError_t prepare_persistent(int op, int prec, int *grid);
cudaError_t launch_persistent(int op, int prec, const ApplyParams *params, const int *order,
                              const int2 *items, int nitems, int grid, cudaStream_t s);
// Locate the static scratch array of igasf_apply_noalloc on `device` (current)
// and cache its address (noalloc.cu).
void noalloc_prepare(int device);

}  // namespace igasf
