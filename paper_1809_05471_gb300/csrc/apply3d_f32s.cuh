// FP32 tile kernel, split variant: the sweeps and the factor prefetch of the
// register-prefetch kernel (apply3d_f32r.cuh), but phase C of the stiffness
// spreads each pencil pair over three lanes of a warp, one per derivative
// stream: lane k holds only its stream's dof values and accumulators
// (2 x (S3 + p - 1) float2 instead of 6 x) and one of the three 16-byte factor
// chunks of a slab. Per slab each lane contracts its stream with the
// direction-3 table (B3' for d3 u, B3 for d2 u and d1 u), the three partial
// derivatives and the missing factors are exchanged by warp shuffles, each
// lane forms its row of g = D grad u and runs its transposed sweep. Ten pairs
// fill 30 lanes of a warp. Less state per thread gives more resident warps at
// high orders, where the other variants are occupancy-bound. The mass apply
// keeps one pencil pair per thread.
#pragma once

#include "apply3d_f32.cuh"
#include "apply3d_f32r.cuh"
#include "igasf_internal.h"
#include "layout.h"

namespace igasf {

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <int P, int S1, int S2, int S3>
struct TileF2S {
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
  // stiffness: three lanes per pencil pair in phase C, 10 pairs per warp
  static constexpr int NW3 = (NPAIR + 9) / 10;
  static constexpr int NT = NW3 * 32 > (NPAIR + 31) / 32 * 32 ? NW3 * 32 : (NPAIR + 31) / 32 * 32;
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

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF>
__device__ __forceinline__ void apply3d_f32s_body(const ApplyParams &prm, const int tile) {
  using G = TileF2S<P, S1, S2, S3>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int H1 = G::H1, PP = G::PP, NT = G::NT, NPAIR = G::NPAIR, UNITS = G::UNITS;
  constexpr int NCH = STIFF ? 3 : 1;   // chunks of a pencil pair per slab
  using Chunk = typename FactorChunk<STIFF, BF>::type;

  extern __shared__ __align__(16) unsigned char smem_f32s[];
  float *sm = reinterpret_cast<float *>(smem_f32s);
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

  // ---- request the first PD slabs of factors now (consumed in phase C).
  // Stiffness: lane 3i + k of a warp (i < 10) serves stream k of pencil pair
  // 10 w + i (w the warp) and reads one 16-byte chunk per slab: role k reads
  // chunk 2 - k, so role 0 holds (D23, D33), role 1 (D13, D22), role 2 (D11, D12).
  // Mass: one pencil pair per thread, as in the register-prefetch kernel.
  const int lane = tid & 31;
  const int grp = lane / 3, role = lane - 3 * grp;
  const int pr = STIFF ? (tid >> 5) * 10 + grp : tid;
  const bool has_pair = STIFF ? (lane < 30 && pr < NPAIR) : tid < NPAIR;
  const int ch = STIFF ? 2 - role : 0;
  Chunk dq[PD];
  const Chunk *Dc = reinterpret_cast<const Chunk *>(prm.D) + (size_t)tile * Q3 * NCH * UNITS +
                    (size_t)ch * UNITS + pr;
#pragma unroll
  for (int s = 0; s < PD; ++s) {
    dq[s] = Chunk{};
    if (has_pair && s < nslab) dq[s] = ldg_stream(Dc + (size_t)s * NCH * UNITS);
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

  // ---- C: direction-3 sweep, product with D, transposed sweep
  if constexpr (STIFF) {
    // this lane's stream: role 0 Y00 (d3 u, table B3'), role 1 Y01 (d2 u, B3),
    // role 2 Y10 (d1 u, B3); the three partial derivatives and the factors
    // a lane lacks come from the other two lanes of its group by shuffles
    float2 *Ys = role == 0 ? Y0 : (role == 1 ? Y1 : Y2);
    const float2 *ts = reinterpret_cast<const float2 *>(role == 0 ? t3d : t3b);
    const int base = lane - role;
    const float2 zero = make_float2(0.f, 0.f);
    float2 y[E3], z[E3];
#pragma unroll
    for (int n = 0; n < E3; ++n) {
      y[n] = has_pair ? Ys[n * NPAIR + pr] : zero;
      z[n] = zero;
    }
#pragma unroll
    for (int e3 = 0; e3 < S3; ++e3) {
      if (e3 < ke3) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q3 = e3 * P + qq;
          const float4 c4 = widen(dq[q3 % PD]);
          if (has_pair && q3 + PD < nslab) dq[q3 % PD] = ldg_stream(Dc + (size_t)(q3 + PD) * NCH * UNITS);
          float2 t[P];
#pragma unroll
          for (int j = 0; j < P; ++j) t[j] = ts[q3 * PP + j];
          float2 d = zero;
#pragma unroll
          for (int j = 0; j < P; ++j) d = ffma2(t[j], y[e3 + j], d);
          const float2 du3 = shfl2(d, base), du2 = shfl2(d, base + 1), du1 = shfl2(d, base + 2);
          const float2 A = make_float2(c4.x, c4.y), B = make_float2(c4.z, c4.w);
          const float2 A0 = shfl2(A, base), A1 = shfl2(A, base + 1), B2 = shfl2(B, base + 2);
          // role 0: g3 = D13 du1 + D23 du2 + D33 du3; role 1: g2 = D12 du1 + D22 du2 + D23 du3;
          // role 2: g1 = D11 du1 + D12 du2 + D13 du3
          const float2 c1 = role == 0 ? A1 : (role == 1 ? B2 : A);
          const float2 c2 = role == 0 ? A : B;
          const float2 c3 = role == 0 ? B : (role == 1 ? A0 : A1);
          const float2 g = ffma2(c3, du3, ffma2(c2, du2, fmul2(c1, du1)));
#pragma unroll
          for (int j = 0; j < P; ++j) z[e3 + j] = ffma2(t[j], g, z[e3 + j]);
        }
      }
    }
    if (has_pair) {
#pragma unroll
      for (int n = 0; n < E3; ++n) Ys[n * NPAIR + pr] = z[n];
    }
  } else {
    if (has_pair) {
      float2 y0[E3], z0[E3];
#pragma unroll
      for (int n = 0; n < E3; ++n) {
        y0[n] = Y0[n * NPAIR + tid];
        z0[n] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int e3 = 0; e3 < S3; ++e3) {
        if (e3 < ke3) {
#pragma unroll
          for (int qq = 0; qq < P; ++qq) {
            const int q3 = e3 * P + qq;
            const float2 dm = widen(dq[q3 % PD]);
            if (q3 + PD < nslab) dq[q3 % PD] = ldg_stream(Dc + (size_t)(q3 + PD) * UNITS);
            const float2 *b3 = reinterpret_cast<const float2 *>(t3b) + q3 * PP;
            float2 uq = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = ffma2(b3[j], y0[e3 + j], uq);
            const float2 w = fmul2(dm, uq);
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e3 + j] = ffma2(b3[j], w, z0[e3 + j]);
          }
        }
      }
#pragma unroll
      for (int n = 0; n < E3; ++n) Y0[n * NPAIR + tid] = z0[n];
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

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF>
__global__ void __launch_bounds__(TileF2S<P, S1, S2, S3>::NT)
apply3d_f32s_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_f32s_body<P, S1, S2, S3, STIFF, PD, BF>(prm, blockIdx.x);
}

// Many patches in one launch: block b works on tile b - first_block[patch] of
// patch = block_patch[b], with that patch's parameters.
template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF>
__global__ void __launch_bounds__(TileF2S<P, S1, S2, S3>::NT)
apply3d_f32s_batched(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  apply3d_f32s_body<P, S1, S2, S3, STIFF, PD, BF>(bp.params[patch], blockIdx.x - bp.first_block[patch]);
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF>
cudaError_t launch_apply3d_f32s(const ApplyParams &prm, cudaStream_t s) {
  using G = TileF2S<P, S1, S2, S3>;
  apply3d_f32s_kernel<P, S1, S2, S3, STIFF, PD, BF>
      <<<prm.ntiles, G::NT, G::smem_floats(STIFF) * sizeof(float), s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool STIFF, int PD, bool BF>
cudaError_t launch_apply3d_f32s_batched(const BatchParams &bp, int blocks, cudaStream_t s) {
  using G = TileF2S<P, S1, S2, S3>;
  apply3d_f32s_batched<P, S1, S2, S3, STIFF, PD, BF>
      <<<blocks, G::NT, G::smem_floats(STIFF) * sizeof(float), s>>>(bp);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, int PD, bool BF>
cudaError_t prepare_apply3d_f32s() {
  using G = TileF2S<P, S1, S2, S3>;
  const int sm = (int)(G::smem_floats(false) * sizeof(float));
  const int sk = (int)(G::smem_floats(true) * sizeof(float));
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(apply3d_f32s_kernel<P, S1, S2, S3, false, PD, BF>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32s_kernel<P, S1, S2, S3, true, PD, BF>, a, sk);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32s_batched<P, S1, S2, S3, false, PD, BF>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32s_batched<P, S1, S2, S3, true, PD, BF>, a, sk);
  return e;
}

// BF: bfloat16-stored factors. PD: slabs prefetched ahead.
template <int P, int S1, int S2, int S3, bool BF = false, int PD = 2>
ApplyKernel make_apply3d_f32s() {
  using G = TileF2S<P, S1, S2, S3>;
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
  k.variant = IGASF_KERNEL_SPLIT;
  k.launch[IGASF_MASS] = &launch_apply3d_f32s<P, S1, S2, S3, false, PD, BF>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d_f32s<P, S1, S2, S3, true, PD, BF>;
  k.launch_batched[IGASF_MASS] = &launch_apply3d_f32s_batched<P, S1, S2, S3, false, PD, BF>;
  k.launch_batched[IGASF_STIFFNESS] = &launch_apply3d_f32s_batched<P, S1, S2, S3, true, PD, BF>;
  k.prepare = &prepare_apply3d_f32s<P, S1, S2, S3, PD, BF>;
  return k;
}

}  // namespace igasf
