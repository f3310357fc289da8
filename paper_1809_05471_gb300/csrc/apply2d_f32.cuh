// FP32 tile kernel of the 2D apply with packed FP32x2 arithmetic: each thread
// owns a PAIR of neighbouring quadrature pencils (q1 = 2k, 2k+1) running along
// direction 2 through the tile, so every per-pencil quantity is a float2 and
// one FFMA2 advances both. Same sweeps as the scalar 2D kernel (Alg. 3, the
// product with w F, Alg. 2, localized per Sec. 4):
//
//   A  X0 = B1 u, X1 = B1' u                 [n2][k] float2, shared
//   C  per pencil pair, in registers: d2 u = B2' X0, d1 u = B2 X1;
//      g = D grad u; W2 = B2'^T g2, W1 = B2^T g1
//   E  v_D = B1^T W2 + B1'^T W1              one output dof per item
//
// The factors of a slab (one q2) are three 8-byte chunks per pencil pair (D11,
// D12, D22 of both pencils; bfloat16: 4-byte chunks), loaded into registers PD
// slabs ahead, the first PD at kernel entry. Staging loads are issued before
// the first shared-memory store. Direction-2 tables are held as duplicated
// pairs {b, b}.
#pragma once

#include "apply3d_f32.cuh"
#include "apply3d_f32r.cuh"
#include "igasf_internal.h"

namespace igasf {

template <int P, int S1, int S2>
struct Tile2F2 {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P;
  static_assert(Q1 % 2 == 0, "pencil pairs need an even number of q1 points per tile");
  static constexpr int H1 = Q1 / 2;                 // pencil pairs
  static constexpr int PL = (Q1 + 7) / 8 * 8;       // plane (pencils), layout row length
  static constexpr int UNITS = PL / 2;
  static constexpr int NT = (H1 + 31) / 32 * 32;
  static constexpr int PP = P + (P & 1);
  static constexpr int T1 = 2 * P * Q1;             // [j][q1] (B, B')
  static constexpr int T2 = 4 * PP * Q2;            // [q2][PP] dup pairs (B, B')
  static constexpr int VOL = E1 * E2;
  static constexpr int XF = E2 * Q1;                // floats per X array
  __host__ __device__ static constexpr size_t smem_floats(bool stiff) {
    return (size_t)T1 + T2 + (VOL + (VOL & 1)) + (stiff ? 2 : 1) * XF;
  }
};

template <int P, int S1, int S2, bool STIFF, bool BF, int PD>
__global__ void __launch_bounds__(Tile2F2<P, S1, S2>::NT)
apply2d_f32_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  using G = Tile2F2<P, S1, S2>;
  constexpr int E1 = G::E1, E2 = G::E2, Q1 = G::Q1, Q2 = G::Q2;
  constexpr int H1 = G::H1, NT = G::NT, PP = G::PP, UNITS = G::UNITS, VOL = G::VOL;
  constexpr int NCH = STIFF ? 3 : 1;
  using Chunk = typename FactorChunk<false, BF>::type;   // one field of both pencils

  extern __shared__ __align__(16) unsigned char smem_2f[];
  float *sm = reinterpret_cast<float *>(smem_2f);
  float *t1b = sm, *t1d = t1b + P * Q1;                 // [j][q1]
  float *t2b = t1d + P * Q1, *t2d = t2b + 2 * PP * Q2;  // [q2][PP] float2 {b, b}
  float *us = t2d + 2 * PP * Q2;                        // [n2][n1]
  float2 *X0 = reinterpret_cast<float2 *>(us + VOL + (VOL & 1));
  float2 *X1 = X0 + G::XF / 2;

  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int t1 = tile % prm.T[0], t2 = tile / prm.T[0];
  const int e01 = t1 * S1, e02 = t2 * S2;
  const int ke2 = min(S2, prm.K[1] - e02);
  const int nslab = ke2 * P;
  const bool has_pair = tid < H1;

  // ---- first PD slabs of factors, requested now (consumed in phase C)
  Chunk dq[PD][NCH];
  const Chunk *Dc = reinterpret_cast<const Chunk *>(prm.D) + (size_t)tile * Q2 * NCH * UNITS + tid;
#pragma unroll
  for (int s = 0; s < PD; ++s) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      dq[s][c] = Chunk{};
      if (has_pair && s < nslab) dq[s][c] = ldg_stream(Dc + ((size_t)s * NCH + c) * UNITS);
    }
  }

  // ---- stage tables and the u box: every global load before any shared store
  {
    constexpr int A1 = (P * Q1 + NT - 1) / NT, A2 = (PP * Q2 + NT - 1) / NT, AU = (VOL + NT - 1) / NT;
    const float *gb1 = static_cast<const float *>(prm.tabB[0]), *gd1 = static_cast<const float *>(prm.tabD[0]);
    const float *gb2 = static_cast<const float *>(prm.tabB[1]), *gd2 = static_cast<const float *>(prm.tabD[1]);
    const float *u = static_cast<const float *>(prm.u);
    const int N1 = prm.N[0], N2 = prm.N[1];
    float b1[A1], d1[A1], b2[A2], d2[A2], uv[AU];
#pragma unroll
    for (int k = 0; k < A1; ++k) {
      const int i = tid + k * NT;
      b1[k] = 0.f;
      d1[k] = 0.f;
      if (i < P * Q1) {
        const int j = i / Q1, q = i - j * Q1, g = j * prm.Qpad[0] + e01 * P + q;
        b1[k] = __ldg(gb1 + g);
        if (STIFF) d1[k] = __ldg(gd1 + g);
      }
    }
#pragma unroll
    for (int k = 0; k < A2; ++k) {
      const int i = tid + k * NT;
      const int q = i / PP, j = i - q * PP;
      b2[k] = 0.f;
      d2[k] = 0.f;
      if (i < PP * Q2 && j < P) {
        const int g = j * prm.Qpad[1] + e02 * P + q;
        b2[k] = __ldg(gb2 + g);
        if (STIFF) d2[k] = __ldg(gd2 + g);
      }
    }
#pragma unroll
    for (int k = 0; k < AU; ++k) {
      const int i = tid + k * NT;
      const int n1 = i % E1, n2 = i / E1;
      uv[k] = 0.f;
      if (i < VOL && e01 + n1 < N1 && e02 + n2 < N2)
        uv[k] = __ldg(u + (int64_t)(e02 + n2) * N1 + e01 + n1);
    }
#pragma unroll
    for (int k = 0; k < A1; ++k) {
      const int i = tid + k * NT;
      if (i < P * Q1) {
        t1b[i] = b1[k];
        if (STIFF) t1d[i] = d1[k];
      }
    }
#pragma unroll
    for (int k = 0; k < A2; ++k) {
      const int i = tid + k * NT;
      if (i < PP * Q2) {
        reinterpret_cast<float2 *>(t2b)[i] = make_float2(b2[k], b2[k]);
        if (STIFF) reinterpret_cast<float2 *>(t2d)[i] = make_float2(d2[k], d2[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < AU; ++k) {
      const int i = tid + k * NT;
      if (i < VOL) us[i] = uv[k];
    }
  }
  __syncthreads();

  // ---- A: direction 1, X0 = B1 u, X1 = B1' u, one (n2, pair) per item
  for (int i = tid; i < E2 * H1; i += NT) {
    const int k = i % H1, n2 = i / H1;
    const int qa = 2 * k, ea = qa / P, eb = (qa + 1) / P;
    const float *ur = us + n2 * E1;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
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

  // ---- C: pencil pairs: direction-2 sweep, product with D, transposed sweep
  if (has_pair) {
    float2 y0[E2], y1[E2], z0[E2], z1[E2];
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      y0[n] = X0[n * H1 + tid];
      z0[n] = make_float2(0.f, 0.f);
      if (STIFF) {
        y1[n] = X1[n * H1 + tid];
        z1[n] = z0[n];
      }
    }
#pragma unroll
    for (int e2 = 0; e2 < S2; ++e2) {
      if (e2 < ke2) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q2 = e2 * P + qq;
          float2 dc[NCH];
#pragma unroll
          for (int c = 0; c < NCH; ++c) dc[c] = widen(dq[q2 % PD][c]);
          if (q2 + PD < nslab) {
#pragma unroll
            for (int c = 0; c < NCH; ++c)
              dq[q2 % PD][c] = ldg_stream(Dc + ((size_t)(q2 + PD) * NCH + c) * UNITS);
          }
          const float2 *b2 = reinterpret_cast<const float2 *>(t2b) + q2 * PP;
          const float2 *d2 = reinterpret_cast<const float2 *>(t2d) + q2 * PP;
          if (STIFF) {
            float2 du2 = make_float2(0.f, 0.f), du1 = du2;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              du2 = ffma2(d2[j], y0[e2 + j], du2);
              du1 = ffma2(b2[j], y1[e2 + j], du1);
            }
            const float2 g1 = ffma2(dc[1], du2, fmul2(dc[0], du1));   // D11 d1 + D12 d2
            const float2 g2 = ffma2(dc[2], du2, fmul2(dc[1], du1));   // D12 d1 + D22 d2
#pragma unroll
            for (int j = 0; j < P; ++j) {
              z0[e2 + j] = ffma2(d2[j], g2, z0[e2 + j]);   // W2, goes with B1^T
              z1[e2 + j] = ffma2(b2[j], g1, z1[e2 + j]);   // W1, goes with B1'^T
            }
          } else {
            float2 uq = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = ffma2(b2[j], y0[e2 + j], uq);
            const float2 w = fmul2(dc[0], uq);
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e2 + j] = ffma2(b2[j], w, z0[e2 + j]);
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      X0[n * H1 + tid] = z0[n];
      if (STIFF) X1[n * H1 + tid] = z1[n];
    }
  }
  __syncthreads();

  // ---- E: transposed direction 1, one output dof per item
  float *vp = static_cast<float *>(prm.vpart) + (size_t)tile * VOL;
  const float *x0 = reinterpret_cast<const float *>(X0);
  const float *x1 = reinterpret_cast<const float *>(X1);
  for (int i = tid; i < VOL; i += NT) {
    const int n1 = i % E1, n2 = i / E1;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int e1 = n1 - j;
      if (e1 >= 0 && e1 < S1) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q1 = e1 * P + qq;
          acc = fmaf(t1b[j * Q1 + q1], x0[n2 * Q1 + q1], acc);
          if (STIFF) acc = fmaf(t1d[j * Q1 + q1], x1[n2 * Q1 + q1], acc);
        }
      }
    }
    vp[i] = acc;
  }
}

template <int P, int S1, int S2, bool STIFF, bool BF, int PD>
cudaError_t launch_apply2d_f32(const ApplyParams &prm, cudaStream_t s) {
  using G = Tile2F2<P, S1, S2>;
  apply2d_f32_kernel<P, S1, S2, STIFF, BF, PD>
      <<<prm.ntiles, G::NT, G::smem_floats(STIFF) * sizeof(float), s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, bool BF, int PD>
cudaError_t prepare_apply2d_f32() {
  using G = Tile2F2<P, S1, S2>;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(apply2d_f32_kernel<P, S1, S2, false, BF, PD>, a,
                                       (int)(G::smem_floats(false) * sizeof(float)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply2d_f32_kernel<P, S1, S2, true, BF, PD>, a,
                             (int)(G::smem_floats(true) * sizeof(float)));
  return e;
}

// BF: bfloat16-stored factors. PD: slabs prefetched ahead.
template <int P, int S1, int S2, bool BF = false, int PD = 2>
ApplyKernel make_apply2d_f32() {
  using G = Tile2F2<P, S1, S2>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  static_assert(G::smem_floats(true) * sizeof(float) <= 227 * 1024, "tile exceeds shared memory");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = 1;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_floats(false) * sizeof(float);
  k.smem[IGASF_STIFFNESS] = G::smem_floats(true) * sizeof(float);
  k.plane = G::PL;
  k.lanes = 2;
  k.variant = IGASF_KERNEL_REGISTERS;
  k.launch[IGASF_MASS] = &launch_apply2d_f32<P, S1, S2, false, BF, PD>;
  k.launch[IGASF_STIFFNESS] = &launch_apply2d_f32<P, S1, S2, true, BF, PD>;
  k.launch_batched[IGASF_MASS] = nullptr;
  k.launch_batched[IGASF_STIFFNESS] = nullptr;
  k.prepare = &prepare_apply2d_f32<P, S1, S2, BF, PD>;
  return k;
}

}  // namespace igasf
