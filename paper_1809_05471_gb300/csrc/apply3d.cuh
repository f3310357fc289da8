// Matrix-free sum-factorized apply of the 3D mass / stiffness operator on one
// macro-element tile per thread block (Alg. 3, then the pointwise product
// with the factors, then Alg. 2; localized per Sec. 4, eq. loc-basis-change).
//
// Tile = S1 x S2 x S3 elements; its dofs are the (S+p-1)^3 functions active on
// it (element e carries functions e..e+p-1: every knot span is an element, the
// empty spans of repeated knots included with zero weight), its quadrature
// points the (S p)^3 Gauss points. One thread owns one "pencil": a fixed
// (q1, q2) quadrature index in the tile, along all q3.
//
// Stiffness, with B / B' the 1D value / derivative tables of each direction:
//   forward (dofs -> quadrature points):
//     X0 = B1 u, X1 = B1' u                            [n3][n2][q1]  shared
//     Y00 = B2 X0, Y01 = B2' X0, Y10 = B2 X1           [n3][q2][q1]  shared
//     d3u = B3' Y00, d2u = B3 Y01, d1u = B3 Y10        registers, per pencil
//   pointwise: g = D grad u, D = w F (6 stored entries, streamed from HBM)
//   transposed (quadrature points -> dofs):
//     W3 = B3'^T g3, W2 = B3^T g2, W1 = B3^T g1        registers -> shared
//     Ya = B2^T W3 + B2'^T W2, Yb = B2^T W1            [n3][n2][q1]  shared
//     v  = B1^T Ya + B1'^T Yb                          -> per-tile partial v
// The last forward sweep, the product and the first transposed sweep run in
// the registers of the pencil's thread, so the p^3-times-larger quadrature
// point arrays never leave registers and the factors are read exactly once.
#pragma once

#include "igasf_internal.h"

namespace igasf {

template <int P, int S1, int S2, int S3>
struct Tile3 {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1, E3 = S3 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P, Q3 = S3 * P;
  static constexpr int NPEN = Q1 * Q2;
  static constexpr int PL = (NPEN + 31) / 32 * 32;   // factor row length (padded)
  static constexpr int NT = PL;                      // threads per block
  static constexpr int VOL = E1 * E2 * E3;
  static constexpr int X = E3 * E2 * Q1;             // first-sweep array size
  static constexpr int Y = E3 * NPEN;                // second-sweep array size
  static constexpr int TAB = P * (Q1 + Q2 + Q3);
  static constexpr size_t smem_words(bool stiff) {
    return 2 * TAB + VOL + (stiff ? 2 : 1) * X + (stiff ? 3 : 1) * Y;
  }
};

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }

// Two neighbouring values of one factor chunk in one load (a chunk holds two
// values and starts at an even index, so the pair is aligned).
template <typename T> struct Pair2;
template <> struct Pair2<double> { using type = double2; };
template <> struct Pair2<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ typename Pair2<T>::type ld_stream2(const T *p) {
  return __ldcs(reinterpret_cast<const typename Pair2<T>::type *>(p));
}

template <typename T, int P, int S1, int S2, int S3, bool STIFF>
__device__ __forceinline__ void apply3d_body(const ApplyParams &prm, const int tile) {
  using G = Tile3<P, S1, S2, S3>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int NPEN = G::NPEN, PL = G::PL, NT = G::NT;
  constexpr int NF = STIFF ? 6 : 1;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *tb1 = sm, *td1 = tb1 + P * Q1;
  T *tb2 = td1 + P * Q1, *td2 = tb2 + P * Q2;
  T *tb3 = td2 + P * Q2, *td3 = tb3 + P * Q3;
  T *us = td3 + P * Q3;
  T *X0 = us + G::VOL;
  T *X1 = X0 + G::X;                        // stiffness only
  T *Y0 = STIFF ? X1 + G::X : X0 + G::X;
  T *Y1 = Y0 + G::Y, *Y2 = Y1 + G::Y;       // stiffness only

  const int tid = threadIdx.x;
  const int t1 = tile % prm.T[0];
  const int t2 = (tile / prm.T[0]) % prm.T[1];
  const int t3 = tile / (prm.T[0] * prm.T[1]);
  const int e01 = t1 * S1, e02 = t2 * S2, e03 = t3 * S3;
  const int N1 = prm.N[0], N2 = prm.N[1], N3 = prm.N[2];

  // ---- stage tables and the u tile (selection S_D u of eq. loc-basis-change)
  {
    const T *gb1 = static_cast<const T *>(prm.tabB[0]), *gd1 = static_cast<const T *>(prm.tabD[0]);
    const T *gb2 = static_cast<const T *>(prm.tabB[1]), *gd2 = static_cast<const T *>(prm.tabD[1]);
    const T *gb3 = static_cast<const T *>(prm.tabB[2]), *gd3 = static_cast<const T *>(prm.tabD[2]);
    for (int i = tid; i < P * Q1; i += NT) {
      const int j = i / Q1, q = i - j * Q1;
      const int g = j * prm.Qpad[0] + e01 * P + q;
      tb1[i] = gb1[g];
      if (STIFF) td1[i] = gd1[g];
    }
    for (int i = tid; i < P * Q2; i += NT) {
      const int j = i / Q2, q = i - j * Q2;
      const int g = j * prm.Qpad[1] + e02 * P + q;
      tb2[i] = gb2[g];
      if (STIFF) td2[i] = gd2[g];
    }
    for (int i = tid; i < P * Q3; i += NT) {
      const int j = i / Q3, q = i - j * Q3;
      const int g = j * prm.Qpad[2] + e03 * P + q;
      tb3[i] = gb3[g];
      if (STIFF) td3[i] = gd3[g];
    }
    const T *u = static_cast<const T *>(prm.u);
    for (int i = tid; i < G::VOL; i += NT) {
      const int n1 = i % E1, r = i / E1;
      const int n2 = r % E2, n3 = r / E2;
      const int g1 = e01 + n1, g2 = e02 + n2, g3 = e03 + n3;
      T val = T(0);
      if (g1 < N1 && g2 < N2 && g3 < N3) val = u[((int64_t)g3 * N2 + g2) * N1 + g1];
      us[i] = val;
    }
  }
  __syncthreads();

  // ---- forward sweep, direction 1: X0 = B1 u, X1 = B1' u
  for (int i = tid; i < G::X; i += NT) {
    const int q1 = i % Q1, r = i / Q1;
    const T *ur = us + r * E1 + q1 / P;
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const T uv = ur[j];
      a0 = fma(tb1[j * Q1 + q1], uv, a0);
      if (STIFF) a1 = fma(td1[j * Q1 + q1], uv, a1);
    }
    X0[i] = a0;
    if (STIFF) X1[i] = a1;
  }
  __syncthreads();

  // ---- forward sweep, direction 2
  for (int i = tid; i < G::Y; i += NT) {
    const int q1 = i % Q1, r = i / Q1;
    const int q2 = r % Q2, n3 = r / Q2;
    const int base = (n3 * E2 + q2 / P) * Q1 + q1;
    T y00 = T(0), y01 = T(0), y10 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const T b = tb2[j * Q2 + q2];
      const T x0 = X0[base + j * Q1];
      y00 = fma(b, x0, y00);
      if (STIFF) {
        y01 = fma(td2[j * Q2 + q2], x0, y01);
        y10 = fma(b, X1[base + j * Q1], y10);
      }
    }
    Y0[i] = y00;
    if (STIFF) {
      Y1[i] = y01;
      Y2[i] = y10;
    }
  }
  __syncthreads();

  // ---- pencil: direction-3 sweep, pointwise product, transposed direction-3 sweep
  if (tid < NPEN) {
    const int q1 = tid % Q1, q2 = tid / Q1;
    const bool valid = (e01 + q1 / P < prm.K[0]) && (e02 + q2 / P < prm.K[1]);
    const int ke3 = min(S3, prm.K[2] - e03);
    // layout.h with one pencil per unit: mass [slab][pencil]; stiffness
    // [slab][chunk c][pencil] with chunks (11,12), (13,22), (23,33) of two values
    const T *Dt = static_cast<const T *>(prm.D) + (size_t)tile * Q3 * NF * PL + (STIFF ? 2 : 1) * tid;
    T y0[E3], y1[E3], y2[E3], z0[E3], z1[E3], z2[E3];
#pragma unroll
    for (int n = 0; n < E3; ++n) {
      y0[n] = Y0[n * NPEN + tid];
      z0[n] = T(0);
      if (STIFF) {
        y1[n] = Y1[n * NPEN + tid];
        y2[n] = Y2[n * NPEN + tid];
        z1[n] = T(0);
        z2[n] = T(0);
      }
    }
#pragma unroll
    for (int e3 = 0; e3 < S3; ++e3) {
      if (e3 < ke3) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q3 = e3 * P + qq;
          const T *Dq = Dt + (size_t)q3 * NF * PL;
          if (STIFF) {
            T D11 = T(0), D12 = T(0), D13 = T(0), D22 = T(0), D23 = T(0), D33 = T(0);
            if (valid) {
              const auto c0 = ld_stream2(Dq), c1 = ld_stream2(Dq + 2 * PL), c2 = ld_stream2(Dq + 4 * PL);
              D11 = c0.x;
              D12 = c0.y;
              D13 = c1.x;
              D22 = c1.y;
              D23 = c2.x;
              D33 = c2.y;
            }
            T d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const T b = tb3[j * Q3 + q3], db = td3[j * Q3 + q3];
              d3 = fma(db, y0[e3 + j], d3);
              d2 = fma(b, y1[e3 + j], d2);
              d1 = fma(b, y2[e3 + j], d1);
            }
            const T g1 = D11 * d1 + D12 * d2 + D13 * d3;
            const T g2 = D12 * d1 + D22 * d2 + D23 * d3;
            const T g3 = D13 * d1 + D23 * d2 + D33 * d3;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const T b = tb3[j * Q3 + q3], db = td3[j * Q3 + q3];
              z0[e3 + j] = fma(db, g3, z0[e3 + j]);   // W3
              z1[e3 + j] = fma(b, g2, z1[e3 + j]);    // W2
              z2[e3 + j] = fma(b, g1, z2[e3 + j]);    // W1
            }
          } else {
            const T Dm = valid ? ld_stream(Dq) : T(0);
            T uq = T(0);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = fma(tb3[j * Q3 + q3], y0[e3 + j], uq);
            const T w = Dm * uq;
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e3 + j] = fma(tb3[j * Q3 + q3], w, z0[e3 + j]);
          }
        }
      }
    }
#pragma unroll
    for (int n = 0; n < E3; ++n) {
      Y0[n * NPEN + tid] = z0[n];
      if (STIFF) {
        Y1[n * NPEN + tid] = z1[n];
        Y2[n * NPEN + tid] = z2[n];
      }
    }
  }
  __syncthreads();

  // ---- transposed sweep, direction 2: Ya = B2^T W3 + B2'^T W2, Yb = B2^T W1
  for (int i = tid; i < G::X; i += NT) {
    const int q1 = i % Q1, r = i / Q1;
    const int n2 = r % E2, n3 = r / E2;
    T ya = T(0), yb = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int e2 = n2 - j;
      if (e2 >= 0 && e2 < S2) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q2 = e2 * P + qq;
          const int idx = n3 * NPEN + q2 * Q1 + q1;
          const T b = tb2[j * Q2 + q2];
          ya = fma(b, Y0[idx], ya);
          if (STIFF) {
            ya = fma(td2[j * Q2 + q2], Y1[idx], ya);
            yb = fma(b, Y2[idx], yb);
          }
        }
      }
    }
    X0[i] = ya;
    if (STIFF) X1[i] = yb;
  }
  __syncthreads();

  // ---- transposed sweep, direction 1: v_D = B1^T Ya + B1'^T Yb
  T *vp = static_cast<T *>(prm.vpart) + (size_t)tile * G::VOL;
  for (int i = tid; i < G::VOL; i += NT) {
    const int n1 = i % E1, r = i / E1;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int e1 = n1 - j;
      if (e1 >= 0 && e1 < S1) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q1 = e1 * P + qq;
          acc = fma(tb1[j * Q1 + q1], X0[r * Q1 + q1], acc);
          if (STIFF) acc = fma(td1[j * Q1 + q1], X1[r * Q1 + q1], acc);
        }
      }
    }
    vp[i] = acc;
  }
}

template <typename T, int P, int S1, int S2, int S3, bool STIFF>
__global__ void __launch_bounds__(Tile3<P, S1, S2, S3>::NT)
apply3d_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_body<T, P, S1, S2, S3, STIFF>(prm, blockIdx.x);
}

// Many patches in one launch: block b works on tile b - first_block[patch] of
// patch = block_patch[b], with that patch's parameters.
template <typename T, int P, int S1, int S2, int S3, bool STIFF>
__global__ void __launch_bounds__(Tile3<P, S1, S2, S3>::NT)
apply3d_batched(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  apply3d_body<T, P, S1, S2, S3, STIFF>(bp.params[patch], blockIdx.x - bp.first_block[patch]);
}

template <typename T, int P, int S1, int S2, int S3, bool STIFF>
cudaError_t launch_apply3d(const ApplyParams &prm, cudaStream_t s) {
  using G = Tile3<P, S1, S2, S3>;
  const size_t smem = G::smem_words(STIFF) * sizeof(T);
  apply3d_kernel<T, P, S1, S2, S3, STIFF><<<prm.ntiles, G::NT, smem, s>>>(prm);
  return cudaGetLastError();
}

template <typename T, int P, int S1, int S2, int S3>
cudaError_t prepare_apply3d() {
  using G = Tile3<P, S1, S2, S3>;
  cudaError_t e = cudaFuncSetAttribute(apply3d_kernel<T, P, S1, S2, S3, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(G::smem_words(false) * sizeof(T)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply3d_kernel<T, P, S1, S2, S3, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(G::smem_words(true) * sizeof(T)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply3d_batched<T, P, S1, S2, S3, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(G::smem_words(false) * sizeof(T)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(apply3d_batched<T, P, S1, S2, S3, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(G::smem_words(true) * sizeof(T)));
}

template <typename T, int P, int S1, int S2, int S3, bool STIFF>
cudaError_t launch_apply3d_batched(const BatchParams &bp, int blocks, cudaStream_t s) {
  using G = Tile3<P, S1, S2, S3>;
  apply3d_batched<T, P, S1, S2, S3, STIFF><<<blocks, G::NT, G::smem_words(STIFF) * sizeof(T), s>>>(bp);
  return cudaGetLastError();
}

template <typename T, int P, int S1, int S2, int S3>
ApplyKernel make_apply3d() {
  using G = Tile3<P, S1, S2, S3>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  static_assert(G::smem_words(true) * sizeof(T) <= 227 * 1024, "tile exceeds shared memory");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = S3;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_words(false) * sizeof(T);
  k.smem[IGASF_STIFFNESS] = G::smem_words(true) * sizeof(T);
  k.plane = G::PL;
  k.lanes = 1;
  k.variant = IGASF_KERNEL_REGISTERS;
  k.launch[IGASF_MASS] = &launch_apply3d<T, P, S1, S2, S3, false>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d<T, P, S1, S2, S3, true>;
  k.launch_batched[IGASF_MASS] = &launch_apply3d_batched<T, P, S1, S2, S3, false>;
  k.launch_batched[IGASF_STIFFNESS] = &launch_apply3d_batched<T, P, S1, S2, S3, true>;
  k.prepare = &prepare_apply3d<T, P, S1, S2, S3>;
  return k;
}

}  // namespace igasf
