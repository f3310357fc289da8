// One persistent launch for a whole batch of patches (the multipatch setting of
// Sec. 4, patches kept independent), as an alternative to the graph of one
// launch per tile kernel in batch.cu.
//
// The kernel runs blocks of kPersistentThreads threads, as many as fit on the
// GPU at once, and each block walks a work list of (patch, tile) items with a
// stride of the grid size. An item runs the register-prefetch FP32 (or
// bfloat16-stored) tile body of its patch's order on that patch's parameters,
// so a patch must have been set up with the persistent tile shape of its order
// (persistent_tile): the factor layout depends on the tile shape. The block
// covers the pencil pairs of every order's tile (phase C uses one thread per
// pair, phases A, B, D and E every thread). Items are ordered by decreasing
// order, so the expensive tiles are spread over all blocks first and the cheap
// ones fill the tail. Each tile writes the same per-tile partial results, in
// the same arithmetic order, as the single-patch register-prefetch kernel of
// that shape, so the batch apply with the common gather equals the individual
// applies of plans set up with that kernel bit for bit.
#include <cuda_runtime.h>

#include "apply3d_f32r.cuh"
#include "igasf_internal.h"

namespace igasf {

namespace {

// the block covers the 200 pencil pairs of the order-5 tile
constexpr int kPersistentThreads = 224;
constexpr int kPersistentMinP = 2, kPersistentMaxP = 6;
// tile shape per order p = 2..6: the register-prefetch candidates of each order
constexpr int kPersTile[5][3] = {{8, 8, 4}, {8, 4, 4}, {4, 4, 4}, {4, 4, 4}, {2, 2, 8}};

#define IGASF_PERS_BODY(P, S1, S2, S3) \
  apply3d_f32r_body<P, S1, S2, S3, STIFF, 2, BF, kReloadTables, kPersistentThreads>(prm, w.y)

// One resident block per SM guaranteed to the register allocator: the tile
// bodies of orders 5 and 6 keep about 12 (S3 + p - 1) registers of per-pencil
// state in phase C, more than a two-block budget (128 per thread) holds
// without spilling.
constexpr int kPersistentMinBlocks = 1;

template <bool STIFF, bool BF>
__global__ void __launch_bounds__(kPersistentThreads, kPersistentMinBlocks)
apply3d_persistent_kernel(const ApplyParams *params, const int *order, const int2 *items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];               // (patch, tile)
    const ApplyParams &prm = params[w.x];
    switch (order[w.x]) {
      case 2: IGASF_PERS_BODY(2, 8, 8, 4); break;
      case 3: IGASF_PERS_BODY(3, 8, 4, 4); break;
      case 4: IGASF_PERS_BODY(4, 4, 4, 4); break;
      case 5: IGASF_PERS_BODY(5, 4, 4, 4); break;
      case 6: IGASF_PERS_BODY(6, 2, 2, 8); break;
      default: break;
    }
    __syncthreads();   // the next item's staging overwrites this item's shared memory
  }
}

#undef IGASF_PERS_BODY

template <int P, int S1, int S2, int S3>
constexpr size_t body_smem(bool stiff) {
  return TileF2R<P, S1, S2, S3>::smem_floats(stiff) * sizeof(float);
}

size_t persistent_smem(bool stiff) {
  size_t m = body_smem<2, 8, 8, 4>(stiff);
  m = m > body_smem<3, 8, 4, 4>(stiff) ? m : body_smem<3, 8, 4, 4>(stiff);
  m = m > body_smem<4, 4, 4, 4>(stiff) ? m : body_smem<4, 4, 4, 4>(stiff);
  m = m > body_smem<5, 4, 4, 4>(stiff) ? m : body_smem<5, 4, 4, 4>(stiff);
  m = m > body_smem<6, 2, 2, 8>(stiff) ? m : body_smem<6, 2, 2, 8>(stiff);
  return m;
}

template <bool STIFF, bool BF>
cudaError_t prepare_one(int *blocks_per_sm) {
  const size_t sh = persistent_smem(STIFF);
  cudaError_t e = cudaFuncSetAttribute(apply3d_persistent_kernel<STIFF, BF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, apply3d_persistent_kernel<STIFF, BF>,
                                                      kPersistentThreads, sh);
  return e;
}

}  // namespace

bool persistent_tile(int p, int prec, int *S) {
  if (p < kPersistentMinP || p > kPersistentMaxP) return false;
  if (prec != IGASF_FP32 && prec != IGASF_BF16) return false;
  for (int a = 0; a < 3; ++a) S[a] = kPersTile[p - kPersistentMinP][a];
  return true;
}

// Raise the shared-memory limit and return the grid size (resident blocks on
// the current device).
cudaError_t prepare_persistent(int op, int prec, int *grid) {
  int per_sm = 0, dev = 0, sms = 0;
  const bool stiff = op == IGASF_STIFFNESS, bf = prec == IGASF_BF16;
  cudaError_t e = stiff ? (bf ? prepare_one<true, true>(&per_sm) : prepare_one<true, false>(&per_sm))
                        : (bf ? prepare_one<false, true>(&per_sm) : prepare_one<false, false>(&per_sm));
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  *grid = per_sm * sms;
  return e;
}

cudaError_t launch_persistent(int op, int prec, const ApplyParams *params, const int *order,
                              const int2 *items, int nitems, int grid, cudaStream_t s) {
  const bool stiff = op == IGASF_STIFFNESS, bf = prec == IGASF_BF16;
  const size_t sh = persistent_smem(stiff);
  const int g = grid < nitems ? grid : (nitems > 0 ? nitems : 1);
  if (stiff) {
    if (bf) apply3d_persistent_kernel<true, true><<<g, kPersistentThreads, sh, s>>>(params, order, items, nitems);
    else apply3d_persistent_kernel<true, false><<<g, kPersistentThreads, sh, s>>>(params, order, items, nitems);
  } else {
    if (bf) apply3d_persistent_kernel<false, true><<<g, kPersistentThreads, sh, s>>>(params, order, items, nitems);
    else apply3d_persistent_kernel<false, false><<<g, kPersistentThreads, sh, s>>>(params, order, items, nitems);
  }
  return cudaGetLastError();
}

}  // namespace igasf
