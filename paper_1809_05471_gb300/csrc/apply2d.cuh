// Matrix-free sum-factorized apply of the 2D mass / stiffness operator on one
// macro-element tile of S1 x S2 elements per thread block (Alg. 3, product with
// the factors, Alg. 2; localized per Sec. 4). One thread owns the pencil of a
// fixed q1 along all q2 of the tile.
//
// Stiffness:
//   X0 = B1 u, X1 = B1' u                 [n2][q1] shared
//   d2u = B2' X0, d1u = B2 X1             registers (pencil)
//   g = D grad u (3 stored entries)
//   W2 = B2'^T g2, W1 = B2^T g1           registers -> shared
//   v = B1^T W2 + B1'^T W1                -> per-tile partial v
// T is the arithmetic type (double or float), TF the stored factor type (T,
// or bfloat16 with float arithmetic).
#pragma once

#include <cuda_bf16.h>

#include "igasf_internal.h"

namespace igasf {

template <typename T>
__device__ __forceinline__ T load_factor(const T *p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ T load_factor(const __nv_bfloat16 *p) { return (T)__bfloat162float(__ldcs(p)); }

template <int P, int S1, int S2>
struct Tile2 {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P;
  static constexpr int NPEN = Q1;
  static constexpr int PL = (NPEN + 31) / 32 * 32;
  static constexpr int NT = PL;
  static constexpr int VOL = E1 * E2;
  static constexpr int X = E2 * Q1;
  static constexpr int TAB = P * (Q1 + Q2);
  static constexpr size_t smem_words(bool stiff) { return 2 * TAB + VOL + (stiff ? 2 : 1) * X; }
};

template <typename T, typename TF, int P, int S1, int S2, bool STIFF>
__global__ void __launch_bounds__(Tile2<P, S1, S2>::NT)
apply2d_kernel(const ApplyParams prm) {
  using G = Tile2<P, S1, S2>;
  constexpr int E1 = G::E1, E2 = G::E2, Q1 = G::Q1, Q2 = G::Q2;
  constexpr int NPEN = G::NPEN, PL = G::PL, NT = G::NT;
  constexpr int NF = STIFF ? 3 : 1;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *tb1 = sm, *td1 = tb1 + P * Q1, *tb2 = td1 + P * Q1, *td2 = tb2 + P * Q2;
  T *us = td2 + P * Q2;
  T *X0 = us + G::VOL, *X1 = X0 + G::X;

  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int t1 = tile % prm.T[0], t2 = tile / prm.T[0];
  const int e01 = t1 * S1, e02 = t2 * S2;
  const int N1 = prm.N[0], N2 = prm.N[1];
  {
    const T *gb1 = static_cast<const T *>(prm.tabB[0]), *gd1 = static_cast<const T *>(prm.tabD[0]);
    const T *gb2 = static_cast<const T *>(prm.tabB[1]), *gd2 = static_cast<const T *>(prm.tabD[1]);
    for (int i = tid; i < P * Q1; i += NT) {
      const int j = i / Q1, q = i - j * Q1;
      tb1[i] = gb1[j * prm.Qpad[0] + e01 * P + q];
      if (STIFF) td1[i] = gd1[j * prm.Qpad[0] + e01 * P + q];
    }
    for (int i = tid; i < P * Q2; i += NT) {
      const int j = i / Q2, q = i - j * Q2;
      tb2[i] = gb2[j * prm.Qpad[1] + e02 * P + q];
      if (STIFF) td2[i] = gd2[j * prm.Qpad[1] + e02 * P + q];
    }
    const T *u = static_cast<const T *>(prm.u);
    for (int i = tid; i < G::VOL; i += NT) {
      const int n1 = i % E1, n2 = i / E1;
      const int g1 = e01 + n1, g2 = e02 + n2;
      us[i] = (g1 < N1 && g2 < N2) ? u[(int64_t)g2 * N1 + g1] : T(0);
    }
  }
  __syncthreads();

  for (int i = tid; i < G::X; i += NT) {
    const int q1 = i % Q1, n2 = i / Q1;
    const T *ur = us + n2 * E1 + q1 / P;
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      a0 = fma(tb1[j * Q1 + q1], ur[j], a0);
      if (STIFF) a1 = fma(td1[j * Q1 + q1], ur[j], a1);
    }
    X0[i] = a0;
    if (STIFF) X1[i] = a1;
  }
  __syncthreads();

  if (tid < NPEN) {
    const int q1 = tid;
    const bool valid = (e01 + q1 / P < prm.K[0]);
    const int ke2 = min(S2, prm.K[1] - e02);
    const TF *Dt = static_cast<const TF *>(prm.D) + (size_t)tile * Q2 * NF * PL + tid;
    T y0[E2], y1[E2], z0[E2], z1[E2];
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      y0[n] = X0[n * Q1 + q1];
      z0[n] = T(0);
      if (STIFF) {
        y1[n] = X1[n * Q1 + q1];
        z1[n] = T(0);
      }
    }
#pragma unroll
    for (int e2 = 0; e2 < S2; ++e2) {
      if (e2 < ke2) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q2 = e2 * P + qq;
          const TF *Dq = Dt + (size_t)q2 * NF * PL;
          if (STIFF) {
            T D11 = T(0), D12 = T(0), D22 = T(0);
            if (valid) {
              D11 = load_factor<T>(Dq);
              D12 = load_factor<T>(Dq + PL);
              D22 = load_factor<T>(Dq + 2 * PL);
            }
            T d1 = T(0), d2 = T(0);
#pragma unroll
            for (int j = 0; j < P; ++j) {
              d2 = fma(td2[j * Q2 + q2], y0[e2 + j], d2);
              d1 = fma(tb2[j * Q2 + q2], y1[e2 + j], d1);
            }
            const T g1 = D11 * d1 + D12 * d2;
            const T g2 = D12 * d1 + D22 * d2;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              z0[e2 + j] = fma(td2[j * Q2 + q2], g2, z0[e2 + j]);  // W2 (goes with B1^T)
              z1[e2 + j] = fma(tb2[j * Q2 + q2], g1, z1[e2 + j]);  // W1 (goes with B1'^T)
            }
          } else {
            const T Dm = valid ? load_factor<T>(Dq) : T(0);
            T uq = T(0);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = fma(tb2[j * Q2 + q2], y0[e2 + j], uq);
            const T w = Dm * uq;
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e2 + j] = fma(tb2[j * Q2 + q2], w, z0[e2 + j]);
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < E2; ++n) {
      X0[n * Q1 + q1] = z0[n];
      if (STIFF) X1[n * Q1 + q1] = z1[n];
    }
  }
  __syncthreads();

  T *vp = static_cast<T *>(prm.vpart) + (size_t)tile * G::VOL;
  for (int i = tid; i < G::VOL; i += NT) {
    const int n1 = i % E1, n2 = i / E1;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int e1 = n1 - j;
      if (e1 >= 0 && e1 < S1) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q1 = e1 * P + qq;
          acc = fma(tb1[j * Q1 + q1], X0[n2 * Q1 + q1], acc);
          if (STIFF) acc = fma(td1[j * Q1 + q1], X1[n2 * Q1 + q1], acc);
        }
      }
    }
    vp[i] = acc;
  }
}

template <typename T, typename TF, int P, int S1, int S2, bool STIFF>
cudaError_t launch_apply2d(const ApplyParams &prm, cudaStream_t s) {
  using G = Tile2<P, S1, S2>;
  apply2d_kernel<T, TF, P, S1, S2, STIFF><<<prm.ntiles, G::NT, G::smem_words(STIFF) * sizeof(T), s>>>(prm);
  return cudaGetLastError();
}

template <typename T, typename TF, int P, int S1, int S2>
cudaError_t prepare_apply2d() {
  using G = Tile2<P, S1, S2>;
  cudaError_t e = cudaFuncSetAttribute(apply2d_kernel<T, TF, P, S1, S2, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(G::smem_words(false) * sizeof(T)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(apply2d_kernel<T, TF, P, S1, S2, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(G::smem_words(true) * sizeof(T)));
}

template <typename T, int P, int S1, int S2, typename TF = T>
ApplyKernel make_apply2d() {
  using G = Tile2<P, S1, S2>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = 1;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_words(false) * sizeof(T);
  k.smem[IGASF_STIFFNESS] = G::smem_words(true) * sizeof(T);
  k.plane = G::PL;
  k.lanes = 1;
  k.variant = IGASF_KERNEL_REGISTERS;
  k.launch[IGASF_MASS] = &launch_apply2d<T, TF, P, S1, S2, false>;
  k.launch[IGASF_STIFFNESS] = &launch_apply2d<T, TF, P, S1, S2, true>;
  k.launch_batched[IGASF_MASS] = nullptr;
  k.launch_batched[IGASF_STIFFNESS] = nullptr;
  k.prepare = &prepare_apply2d<T, TF, P, S1, S2>;
  return k;
}

}  // namespace igasf
