// Tile-major layout of the stored factors w F (host and device).
//
// A tile of S_1 x .. x S_d elements has Q_a = S_a p quadrature points per
// direction. Its "slabs" are the quadrature indices along the last direction;
// inside a slab the points of the other directions are "pencils", numbered
// lexicographically (q_1 fastest) and padded to `plane` (a multiple of 32).
// Consecutive pencils are grouped into units of `lanes` pencils (1 or 2) that
// one thread of the tile kernel handles. The NF fields of a unit form V = NF *
// lanes values ordered (field, lane); they are cut into chunks of CE values, CE
// the largest power of two dividing V with CE * sizeof(T) <= 16. Within a slab
// the layout is chunk-major: [chunk][unit][CE], so every warp-wide load of one
// chunk is contiguous.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define IGASF_HD __host__ __device__ __forceinline__
#else
#define IGASF_HD inline
#endif

namespace igasf {

IGASF_HD int chunk_elems(int nf, int lanes, int elem_bytes) {
  const int V = nf * lanes;
  int ce = 16 / elem_bytes;
  while (ce > 1 && (V % ce) != 0) ce >>= 1;
  return ce;
}

// Index of (tile, slab, pencil, field) in a layout with `plane` pencils per
// slab row, `qlast` slabs per tile, nf fields and `lanes` pencils per unit.
IGASF_HD int64_t factor_index(int64_t tile, int slab, int pen, int f, int nf, int plane,
                              int qlast, int lanes, int elem_bytes) {
  const int ce = chunk_elems(nf, lanes, elem_bytes);
  const int units = plane / lanes;
  const int unit = pen / lanes, lane = pen - unit * lanes;
  const int v = f * lanes + lane;
  const int ch = v / ce, w = v - ch * ce;
  const int nch = nf * lanes / ce;
  return (((tile * qlast + slab) * nch + ch) * (int64_t)units + unit) * ce + w;
}

// Index of field f at the quadrature point with per-direction global indices
// qg[0..d-1], in the layout of tiles of S[a] elements, T[a] tiles per
// direction: the tile, the pencil inside the tile's slab (directions before
// the last, first fastest) and the slab (the last direction's local index).
IGASF_HD int64_t layout_index_q(int d, int p, const int *S, const int *T, int plane, int lanes,
                                int elem_bytes, int nf, int f, const int *qg) {
  int64_t tile = 0, stride = 1;
  int pen = 0, pstride = 1, slab = 0;
  for (int a = 0; a < d; ++a) {
    const int t = qg[a] / p / S[a];
    const int ql = qg[a] - t * S[a] * p;
    tile += t * stride;
    stride *= T[a];
    if (a < d - 1) {
      pen += ql * pstride;
      pstride *= S[a] * p;
    } else {
      slab = ql;
    }
  }
  return factor_index(tile, slab, pen, f, nf, plane, S[d - 1] * p, lanes, elem_bytes);
}

}  // namespace igasf
