// FP32 tile kernel, register-prefetch variant: the same packed FP32x2 sweeps as
// apply3d_f32.cuh, but each thread loads its own factors straight from HBM into
// registers, PD slabs ahead (the first PD slabs at kernel entry; PD scaled up
// for the narrow slabs of the mass). No producer
// warp and no shared-memory ring: fewer instructions and no barrier waits,
// fewer bytes in flight. Which variant is faster depends on the order and the
// tile (both are tile-search candidates).
//
// Each thread owns a PAIR of neighbouring quadrature pencils
// (q1 = 2k, 2k+1 at one q2), so every per-pencil quantity is a float2 and one
// FFMA2 advances both pencils. Same sweeps as the scalar kernel (Alg. 3, the
// product with w F, Alg. 2, localized per Sec. 4):
//
//   A  X0 = B1 u, X1 = B1' u                      [n3][n2][k]  float2, shared
//   B  Y00 = B2 X0, Y01 = B2' X0, Y10 = B2 X1     [n3][q2][k]  float2, shared
//      (each item holds the p dofs of one element in registers, emits its p q2)
//   C  per pencil pair, in registers: d3 u = B3' Y00, d2 u = B3 Y01,
//      d1 u = B3 Y10; g = D grad u; W3 = B3'^T g3, W2 = B3^T g2, W1 = B3^T g1
//   D  Ya = B2^T W3 + B2'^T W2, Yb = B2^T W1      (register-blocked over q2)
//   E  v_D = B1^T Ya + B1'^T Yb                   (register-blocked over q1)
//
// The factors of the first PD slabs are requested at kernel entry, before
// phases A and B, so their HBM latency overlaps the first two sweeps; in
// phase C every slab's loads are issued PD slabs ahead of their use.
// Tables of directions 2 and 3 are held in shared memory as duplicated pairs
// {b, b} so that one 128-bit load feeds two FFMA2 table operands.
// BF (template flag): the factors are stored in bfloat16, so each prefetched
// slab takes half the bytes and half the registers; they are widened to FP32
// at use.
#pragma once

#include "apply3d_f32.cuh"
#include "igasf_internal.h"
#include "layout.h"

namespace igasf {


// Streaming (evict-first) loads of one factor chunk.
__device__ __forceinline__ float4 ldg_stream(const float4 *p) {
  float4 r;
  asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ float2 ldg_stream(const float2 *p) {
  float2 r;
  asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}

__device__ __forceinline__ uint2 ldg_stream(const uint2 *p) {
  uint2 r;
  asm volatile("ld.global.cs.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}

__device__ __forceinline__ uint32_t ldg_stream(const uint32_t *p) {
  uint32_t r;
  asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(r) : "l"(p));
  return r;
}

// Flags of the register-prefetch kernel (template parameter RL).
constexpr int kReloadTables = 1;
constexpr int kL2Prefetch = 2;

template <int P, int S1, int S2, int S3>
struct TileF2R {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1, E3 = S3 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P, Q3 = S3 * P;
  static_assert(Q1 % 2 == 0, "pencil pairs need an even number of q1 points per tile");
  static constexpr int H1 = Q1 / 2;                 // pencil pairs per q1 row
  static constexpr int NPEN = Q1 * Q2;
  // plane (pencils), the layout row length: padded to a multiple of 8 so that
  // every slab is a whole number of 16-byte units in each storage format
  static constexpr int PL = (NPEN + 7) / 8 * 8;
  static constexpr int UNITS = PL / 2;              // pairs per layout row
  static constexpr int NPAIR = H1 * Q2;
  static constexpr int NT = (NPAIR + 31) / 32 * 32;
  static constexpr int PP = P + (P & 1);            // j padded to even for 128-bit loads
  static constexpr int T2 = 4 * PP * Q2;            // dup tables of dir 2 (B, B'), floats
  static constexpr int T3 = 4 * PP * Q3;
  static constexpr int T1 = 2 * P * Q1;             // dir-1 tables [j][q1] (B, B')
  static constexpr int VOL = E1 * E2 * E3;
  static constexpr int X = E3 * E2 * Q1;            // floats
  static constexpr int Y = E3 * Q2 * Q1;            // floats
  static constexpr size_t smem_floats(bool stiff) {
    return (size_t)T2 + T3 + T1 + (stiff ? 2 : 1) * X + (stiff ? 3 : 1) * Y + VOL;
  }
};

// NTX: block size when it is not the tile's own (0); a persistent kernel that
// runs tiles of several orders in blocks of one size passes its block size,
// which must cover the tile's pencil pairs.
template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int NTX = 0>
__device__ __forceinline__ void apply3d_f32r_body(const ApplyParams &prm, const int tile) {
  using G = TileF2R<P, S1, S2, S3>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int H1 = G::H1, PP = G::PP, NPAIR = G::NPAIR, UNITS = G::UNITS;
  constexpr int NT = NTX ? NTX : G::NT;
  static_assert(NT >= NPAIR, "the block must cover the tile's pencil pairs");
  constexpr int NCH = STIFF ? 3 : 1;   // chunks of a pencil pair per slab
  using Chunk = typename FactorChunk<STIFF, BF>::type;
  // Slabs in flight per thread. PD counts slabs of FP32 stiffness factors (48
  // bytes per thread and slab); the mass's single-field slabs (8 or 4 bytes)
  // are requested proportionally further ahead, so that they keep about the
  // same bytes in flight (at most the tile's Q3 slabs). The bfloat16 stiffness
  // keeps PD: twice as many slabs ahead raised its registers to 154 and cost a
  // resident block per SM (64^3, p = 4: 61 -> 67 us).
  constexpr int SLABB = NCH * (int)sizeof(Chunk);
  constexpr int PDX = STIFF ? PD : cmin(Q3, cmax(PD, PD * 48 / SLABB));
  constexpr bool L2P = (RL & kL2Prefetch) != 0;

  extern __shared__ __align__(16) unsigned char smem_f32r[];
  float *sm = reinterpret_cast<float *>(smem_f32r);
  float *t2b = sm, *t2d = t2b + 2 * PP * Q2;        // [q2][PP] float2 {b, b}
  float *t3b = t2d + 2 * PP * Q2, *t3d = t3b + 2 * PP * Q3;
  float *t1b = t3d + 2 * PP * Q3, *t1d = t1b + P * Q1; // [j][q1]
  float2 *X0 = reinterpret_cast<float2 *>(t1d + P * Q1);
  float2 *X1 = X0 + G::X / 2;
  float2 *Y0 = STIFF ? X1 + G::X / 2 : X0 + G::X / 2;
  float2 *Y1 = Y0 + G::Y / 2, *Y2 = Y1 + G::Y / 2;
  float *us = reinterpret_cast<float *>(STIFF ? Y2 + G::Y / 2 : Y0 + G::Y / 2);

  const int tid = threadIdx.x;
  const int t1 = tile % prm.T[0];
  const int t2 = (tile / prm.T[0]) % prm.T[1];
  const int t3 = tile / (prm.T[0] * prm.T[1]);
  const int e01 = t1 * S1, e02 = t2 * S2, e03 = t3 * S3;
  const int ke3 = min(S3, prm.K[2] - e03);
  const int nslab = ke3 * P;

  // ---- with L2P, the tile's factors (up to about 96 KB of them) into L2 now,
  // as evict-first lines: the stream from DRAM runs during staging and phases
  // A and B, and the register loads of phase C hit L2; then the first PDX
  // slabs into registers (consumed in phase C)
  const bool has_pair = tid < NPAIR;
  Chunk dq[PDX][NCH];
  const Chunk *Dc = reinterpret_cast<const Chunk *>(prm.D) + (size_t)tile * Q3 * NCH * UNITS + tid;
  if constexpr (L2P) {
    constexpr uint32_t SLAB_ROW = (uint32_t)(NCH * UNITS * sizeof(Chunk));   // one slab, all pairs
    prefetch_factor_slabs(Dc - tid, SLAB_ROW, 0, min(l2_window_slabs((int)SLAB_ROW, Q3), nslab), tid, NT);
  }
#pragma unroll
  for (int s = 0; s < PDX; ++s) {
    if (has_pair && s < nslab) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) dq[s][c] = ldg_stream(Dc + ((size_t)s * NCH + c) * UNITS);
    }
  }

  // ---- stage tables and the u tile
  stage_tile_f32<P, S1, S2, S3, NT, STIFF>(prm, tid, e01, e02, e03, t1b, t1d, t2b, t2d, t3b, t3d, us);
  __syncthreads();

  // ---- A: direction 1, X0 = B1 u, X1 = B1' u, one pencil pair per item
  for (int i = tid; i < E3 * E2 * H1; i += NT) {
    const int k = i % H1, r = i / H1;
    const int qa = 2 * k;
    const int ea = qa / P, eb = (qa + 1) / P;
    const float *ur = us + r * E1;
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const float2 uu = make_float2(ur[ea + j], ur[eb + j]);
      a0 = ffma2(*reinterpret_cast<const float2 *>(t1b + j * Q1 + qa), uu, a0);
      if (STIFF) a1 = ffma2(*reinterpret_cast<const float2 *>(t1d + j * Q1 + qa), uu, a1);
    }
    X0[i] = a0;
    if (STIFF) X1[i] = a1;
  }
  __syncthreads();

  // ---- B: direction 2, one (n3, element e2, pair) per item: p inputs -> p outputs
  for (int i = tid; i < E3 * S2 * H1; i += NT) {
    const int k = i % H1, t = i / H1;
    const int e2 = t % S2, n3 = t / S2;
    float2 xa[P], xb[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      xa[j] = X0[(n3 * E2 + e2 + j) * H1 + k];
      if (STIFF) xb[j] = X1[(n3 * E2 + e2 + j) * H1 + k];
    }
#pragma unroll
    for (int qq = 0; qq < P; ++qq) {
      const int q2 = e2 * P + qq;
      const float4 *b4 = reinterpret_cast<const float4 *>(t2b + q2 * 2 * PP);
      const float4 *d4 = reinterpret_cast<const float4 *>(t2d + q2 * 2 * PP);
      float2 y00 = make_float2(0.f, 0.f), y01 = y00, y10 = y00;
#pragma unroll
      for (int jj = 0; jj < PP / 2; ++jj) {
        const float4 bb = b4[jj];
        const int j0 = 2 * jj, j1 = 2 * jj + 1;
        y00 = ffma2(make_float2(bb.x, bb.y), xa[j0], y00);
        if (STIFF) {
          const float4 dd = d4[jj];
          y01 = ffma2(make_float2(dd.x, dd.y), xa[j0], y01);
          y10 = ffma2(make_float2(bb.x, bb.y), xb[j0], y10);
          if (j1 < P) {
            y01 = ffma2(make_float2(dd.z, dd.w), xa[j1], y01);
            y10 = ffma2(make_float2(bb.z, bb.w), xb[j1], y10);
          }
        }
        if (j1 < P) y00 = ffma2(make_float2(bb.z, bb.w), xa[j1], y00);
      }
      const int idx = (n3 * Q2 + q2) * H1 + k;
      Y0[idx] = y00;
      if (STIFF) {
        Y1[idx] = y01;
        Y2[idx] = y10;
      }
    }
  }
  __syncthreads();

  // ---- C: pencil pairs: direction-3 sweep, product with D, transposed sweep.
  // Element e3 reads y[e3 .. e3 + P - 1] and adds to z[e3 .. e3 + P - 1], so
  // y[n] is read from shared memory when element n - P + 1 first needs it and
  // z[n] written back as soon as element n has added to it: P live values per
  // array instead of E3 (the same arithmetic in the same order).
  if (has_pair) {
    float2 y0[E3], y1[E3], y2[E3], z0[E3], z1[E3], z2[E3];
#pragma unroll
    for (int n = 0; n < P - 1; ++n) {
      y0[n] = Y0[n * NPAIR + tid];
      z0[n] = make_float2(0.f, 0.f);
      if (STIFF) {
        y1[n] = Y1[n * NPAIR + tid];
        y2[n] = Y2[n * NPAIR + tid];
        z1[n] = z0[n];
        z2[n] = z0[n];
      }
    }
#pragma unroll
    for (int e3 = 0; e3 < S3; ++e3) {
      {
        const int n = e3 + P - 1;
        y0[n] = Y0[n * NPAIR + tid];
        z0[n] = make_float2(0.f, 0.f);
        if (STIFF) {
          y1[n] = Y1[n * NPAIR + tid];
          y2[n] = Y2[n * NPAIR + tid];
          z1[n] = z0[n];
          z2[n] = z0[n];
        }
      }
      if (e3 < ke3) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q3 = e3 * P + qq;
          // factors of this slab, then request slab q3 + PDX into the freed slot
          float4 dc[NCH] = {};
          float2 dm = make_float2(0.f, 0.f);
          if constexpr (STIFF) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) dc[c] = widen(dq[q3 % PDX][c]);
          } else {
            dm = widen(dq[q3 % PDX][0]);
          }
          if (q3 + PDX < nslab) {
#pragma unroll
            for (int c = 0; c < NCH; ++c)
              dq[q3 % PDX][c] = ldg_stream(Dc + ((size_t)(q3 + PDX) * NCH + c) * UNITS);
          }
          float2 b[PP], db[PP];
          {
            const float4 *b4 = reinterpret_cast<const float4 *>(t3b + q3 * 2 * PP);
            const float4 *d4 = reinterpret_cast<const float4 *>(t3d + q3 * 2 * PP);
#pragma unroll
            for (int jj = 0; jj < PP / 2; ++jj) {
              const float4 bb = b4[jj];
              b[2 * jj] = make_float2(bb.x, bb.y);
              b[2 * jj + 1] = make_float2(bb.z, bb.w);
              if (STIFF) {
                const float4 dd = d4[jj];
                db[2 * jj] = make_float2(dd.x, dd.y);
                db[2 * jj + 1] = make_float2(dd.z, dd.w);
              }
            }
          }
          if (STIFF) {
            float2 d1 = make_float2(0.f, 0.f), d2 = d1, d3 = d1;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              d3 = ffma2(db[j], y0[e3 + j], d3);
              d2 = ffma2(b[j], y1[e3 + j], d2);
              d1 = ffma2(b[j], y2[e3 + j], d1);
            }
            const float2 D11 = make_float2(dc[0].x, dc[0].y), D12 = make_float2(dc[0].z, dc[0].w);
            const float2 D13 = make_float2(dc[1].x, dc[1].y), D22 = make_float2(dc[1].z, dc[1].w);
            const float2 D23 = make_float2(dc[2].x, dc[2].y), D33 = make_float2(dc[2].z, dc[2].w);
            const float2 g1 = ffma2(D13, d3, ffma2(D12, d2, fmul2(D11, d1)));
            const float2 g2 = ffma2(D23, d3, ffma2(D22, d2, fmul2(D12, d1)));
            const float2 g3 = ffma2(D33, d3, ffma2(D23, d2, fmul2(D13, d1)));
            if constexpr ((RL & kReloadTables) != 0) {
              // read the tables again (volatile shared loads) instead of
              // keeping them live across the product: fewer registers
              const float4 *b4 = reinterpret_cast<const float4 *>(t3b + q3 * 2 * PP);
              const float4 *d4 = reinterpret_cast<const float4 *>(t3d + q3 * 2 * PP);
#pragma unroll
              for (int jj = 0; jj < PP / 2; ++jj) {
                const float4 bb = lds_volatile4(b4 + jj), dd = lds_volatile4(d4 + jj);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int j = 2 * jj + h;
                  if (j < P) {
                    const float2 bj = h ? make_float2(bb.z, bb.w) : make_float2(bb.x, bb.y);
                    const float2 dj = h ? make_float2(dd.z, dd.w) : make_float2(dd.x, dd.y);
                    z0[e3 + j] = ffma2(dj, g3, z0[e3 + j]);
                    z1[e3 + j] = ffma2(bj, g2, z1[e3 + j]);
                    z2[e3 + j] = ffma2(bj, g1, z2[e3 + j]);
                  }
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < P; ++j) {
                z0[e3 + j] = ffma2(db[j], g3, z0[e3 + j]);   // W3
                z1[e3 + j] = ffma2(b[j], g2, z1[e3 + j]);    // W2
                z2[e3 + j] = ffma2(b[j], g1, z2[e3 + j]);    // W1
              }
            }
          } else {
            float2 uq = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = ffma2(b[j], y0[e3 + j], uq);
            const float2 w = fmul2(dm, uq);
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e3 + j] = ffma2(b[j], w, z0[e3 + j]);
          }
        }
      }
      Y0[e3 * NPAIR + tid] = z0[e3];   // complete: no later element adds to z[e3]
      if (STIFF) {
        Y1[e3 * NPAIR + tid] = z1[e3];
        Y2[e3 * NPAIR + tid] = z2[e3];
      }
    }
#pragma unroll
    for (int n = S3; n < E3; ++n) {
      Y0[n * NPAIR + tid] = z0[n];
      if (STIFF) {
        Y1[n * NPAIR + tid] = z1[n];
        Y2[n * NPAIR + tid] = z2[n];
      }
    }
  }
  __syncthreads();

  // ---- D: transposed direction 2, register-blocked over all q2 of the tile
  for (int i = tid; i < E3 * H1; i += NT) {
    const int k = i % H1, n3 = i / H1;
    float2 ya[E2], yb[E2];
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      ya[n] = make_float2(0.f, 0.f);
      yb[n] = ya[n];
    }
#pragma unroll
    for (int q2 = 0; q2 < Q2; ++q2) {
      const int e2 = q2 / P;
      const int idx = (n3 * Q2 + q2) * H1 + k;
      const float2 w3 = Y0[idx];
      float2 w2 = make_float2(0.f, 0.f), w1 = w2;
      if (STIFF) {
        w2 = Y1[idx];
        w1 = Y2[idx];
      }
      const float4 *b4 = reinterpret_cast<const float4 *>(t2b + q2 * 2 * PP);
      const float4 *d4 = reinterpret_cast<const float4 *>(t2d + q2 * 2 * PP);
#pragma unroll
      for (int jj = 0; jj < PP / 2; ++jj) {
        const float4 bb = b4[jj];
        const float4 dd = STIFF ? d4[jj] : bb;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * jj + h;
          if (j < P) {
            const float2 bj = h ? make_float2(bb.z, bb.w) : make_float2(bb.x, bb.y);
            ya[e2 + j] = ffma2(bj, w3, ya[e2 + j]);
            if (STIFF) {
              const float2 dj = h ? make_float2(dd.z, dd.w) : make_float2(dd.x, dd.y);
              ya[e2 + j] = ffma2(dj, w2, ya[e2 + j]);
              yb[e2 + j] = ffma2(bj, w1, yb[e2 + j]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      X0[(n3 * E2 + n) * H1 + k] = ya[n];
      if (STIFF) X1[(n3 * E2 + n) * H1 + k] = yb[n];
    }
  }
  __syncthreads();

  // ---- E: transposed direction 1, one (n3, n2) row per item, all q1 in registers
  float *vp = static_cast<float *>(prm.vpart) + (size_t)tile * G::VOL;
  for (int r = tid; r < E3 * E2; r += NT) {
    float2 acc[E1];
#pragma unroll
    for (int n = 0; n < E1; ++n) acc[n] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < H1; ++k) {
      const int qa = 2 * k, ea = qa / P, eb = (qa + 1) / P;
      const float2 ya = X0[r * H1 + k];
      const float2 yb = STIFF ? X1[r * H1 + k] : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const float2 bt = *reinterpret_cast<const float2 *>(t1b + j * Q1 + qa);
        const float2 dt = STIFF ? *reinterpret_cast<const float2 *>(t1d + j * Q1 + qa) : bt;
        if (ea == eb) {
          acc[ea + j] = ffma2(bt, ya, acc[ea + j]);
          if (STIFF) acc[ea + j] = ffma2(dt, yb, acc[ea + j]);
        } else {
          acc[ea + j].x = fmaf(bt.x, ya.x, acc[ea + j].x);
          acc[eb + j].y = fmaf(bt.y, ya.y, acc[eb + j].y);
          if (STIFF) {
            acc[ea + j].x = fmaf(dt.x, yb.x, acc[ea + j].x);
            acc[eb + j].y = fmaf(dt.y, yb.y, acc[eb + j].y);
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < E1; ++n) vp[r * E1 + n] = acc[n].x + acc[n].y;
  }
}

// Two kernel entry points per configuration: without a minimum of resident
// blocks (the register allocator's own choice) and with one (MINB > 0 caps the
// registers per thread at 65536 / (MINB * threads)); the launch picks by MINB.
template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL>
__global__ void __launch_bounds__(TileF2R<P, S1, S2, S3>::NT)
apply3d_f32r_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_f32r_body<P, S1, S2, S3, STIFF, PD, BF, RL>(prm, blockIdx.x);
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int MINB>
__global__ void __launch_bounds__(TileF2R<P, S1, S2, S3>::NT, MINB)
apply3d_f32r_kernel_mb(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_f32r_body<P, S1, S2, S3, STIFF, PD, BF, RL>(prm, blockIdx.x);
}

// Many patches in one launch: block b works on tile b - first_block[patch] of
// patch = block_patch[b], with that patch's parameters.
template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL>
__global__ void __launch_bounds__(TileF2R<P, S1, S2, S3>::NT)
apply3d_f32r_batched(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  apply3d_f32r_body<P, S1, S2, S3, STIFF, PD, BF, RL>(bp.params[patch], blockIdx.x - bp.first_block[patch]);
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int MINB>
__global__ void __launch_bounds__(TileF2R<P, S1, S2, S3>::NT, MINB)
apply3d_f32r_batched_mb(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  apply3d_f32r_body<P, S1, S2, S3, STIFF, PD, BF, RL>(bp.params[patch], blockIdx.x - bp.first_block[patch]);
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int MINB>
cudaError_t launch_apply3d_f32r(const ApplyParams &prm, cudaStream_t s) {
  using G = TileF2R<P, S1, S2, S3>;
  const size_t sh = G::smem_floats(STIFF) * sizeof(float);
  if constexpr (MINB > 0)
    apply3d_f32r_kernel_mb<P, S1, S2, S3, STIFF, PD, BF, RL, MINB><<<prm.ntiles, G::NT, sh, s>>>(prm);
  else
    apply3d_f32r_kernel<P, S1, S2, S3, STIFF, PD, BF, RL><<<prm.ntiles, G::NT, sh, s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int MINB>
cudaError_t launch_apply3d_f32r_batched(const BatchParams &bp, int blocks, cudaStream_t s) {
  using G = TileF2R<P, S1, S2, S3>;
  const size_t sh = G::smem_floats(STIFF) * sizeof(float);
  if constexpr (MINB > 0)
    apply3d_f32r_batched_mb<P, S1, S2, S3, STIFF, PD, BF, RL, MINB><<<blocks, G::NT, sh, s>>>(bp);
  else
    apply3d_f32r_batched<P, S1, S2, S3, STIFF, PD, BF, RL><<<blocks, G::NT, sh, s>>>(bp);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF, int RL, int MINB>
cudaError_t prepare_apply3d_f32r_op() {
  using G = TileF2R<P, S1, S2, S3>;
  const int sh = (int)(G::smem_floats(STIFF) * sizeof(float));
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if constexpr (MINB > 0) {
    e = cudaFuncSetAttribute(apply3d_f32r_kernel_mb<P, S1, S2, S3, STIFF, PD, BF, RL, MINB>, a, sh);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32r_batched_mb<P, S1, S2, S3, STIFF, PD, BF, RL, MINB>, a, sh);
  } else {
    e = cudaFuncSetAttribute(apply3d_f32r_kernel<P, S1, S2, S3, STIFF, PD, BF, RL>, a, sh);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32r_batched<P, S1, S2, S3, STIFF, PD, BF, RL>, a, sh);
  }
  return e;
}

template <int P, int S1, int S2, int S3, int PD, bool BF, int RL, int MINB, int MINBM>
cudaError_t prepare_apply3d_f32r() {
  cudaError_t e = prepare_apply3d_f32r_op<P, S1, S2, S3, false, PD, BF, RL, MINBM>();
  if (e == cudaSuccess) e = prepare_apply3d_f32r_op<P, S1, S2, S3, true, PD, BF, RL, MINB>();
  return e;
}

// BF: bfloat16-stored factors. PD: slabs prefetched ahead. MINB: minimum
// resident blocks per SM asked of the register allocator (0: its own choice).
// RL: flags; kReloadTables: phase C reads the direction-3 tables again for the
// transposed sweep instead of keeping them live across the product;
// kL2Prefetch: the tile requests its factors into L2 at entry. MINBM: the
// mass kernel's minimum resident blocks where it differs from MINB (0: the
// same); the mass keeps fewer values per thread and fits more blocks.
template <int P, int S1, int S2, int S3, bool BF = false, int PD = 2, int MINB = 0, int RL = 0,
          int MINBM = 0>
ApplyKernel make_apply3d_f32r() {
  constexpr int MB_MASS = MINBM ? MINBM : MINB;
  using G = TileF2R<P, S1, S2, S3>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  static_assert(G::smem_floats(true) * sizeof(float) <= 227 * 1024, "tile exceeds shared memory");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = S3;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_floats(false) * sizeof(float);
  k.smem[IGASF_STIFFNESS] = G::smem_floats(true) * sizeof(float);
  k.plane = G::PL;
  k.lanes = 2;
  k.variant = IGASF_KERNEL_REGISTERS;
  k.launch[IGASF_MASS] = &launch_apply3d_f32r<P, S1, S2, S3, false, PD, BF, RL, MB_MASS>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d_f32r<P, S1, S2, S3, true, PD, BF, RL, MINB>;
  k.launch_batched[IGASF_MASS] = &launch_apply3d_f32r_batched<P, S1, S2, S3, false, PD, BF, RL, MB_MASS>;
  k.launch_batched[IGASF_STIFFNESS] = &launch_apply3d_f32r_batched<P, S1, S2, S3, true, PD, BF, RL, MINB>;
  k.prepare = &prepare_apply3d_f32r<P, S1, S2, S3, PD, BF, RL, MINB, MB_MASS>;
  return k;
}

}  // namespace igasf
