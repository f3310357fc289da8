// FP32 tile kernel of the 3D apply that evaluates the factors w F itself
// (Sec. 6.2: each component of G = sum_n c_n phi_n, and its derivatives, by
// the same sum factorization as u; then det J, the cofactor matrix C of J and
// the coefficient at G(x)) instead of reading stored factors from HBM. With
// J^-1 = C^T / det J:
//
//     mass:       w |det J|
//     stiffness:  w a(G(x)) |det J| J^-1 J^-T = w a(G(x)) C^T C / |det J|.
//
// The sweeps of u are those of the register-prefetch kernel (apply3d_f32r.cuh:
// phases A, B, the per-pencil-pair phase C, then D and E), with packed FP32x2
// arithmetic and a pair of quadrature pencils per thread. The geometry is
// evaluated slab by slab inside phase C, direction 3 first:
//
//   Z  (all threads)  Z0_c = B3(q3) c_c, Z1_c = B3'(q3) c_c     [c][n2][n1]
//   X  (all threads)  X0_c = B1 Z0_c, X1_c = B1' Z0_c, X2_c = B1 Z1_c  [c][n2][k]
//   per pencil pair   G_c = B2 X0_c, dG_c/dxi_1 = B2 X1_c,
//                     dG_c/dxi_2 = B2' X0_c, dG_c/dxi_3 = B2 X2_c
//
// ZALL: Z of every slab is computed before phase C (one barrier), otherwise
// per slab into a double buffer. X is double-buffered, so a slab costs one
// (ZALL) or two block barriers. Quadrature points of elements beyond the patch
// (ragged tiles) get zero factors.
#pragma once

#include "apply3d_f32.cuh"
#include "igasf_internal.h"

namespace igasf {

template <int P, int S1, int S2, int S3, bool ZALL>
struct TileF2G {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1, E3 = S3 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P, Q3 = S3 * P;
  static_assert(Q1 % 2 == 0, "pencil pairs need an even number of q1 points per tile");
  static constexpr int H1 = Q1 / 2;
  static constexpr int NPAIR = H1 * Q2;
  static constexpr int NT = (NPAIR + 31) / 32 * 32;
  static constexpr int PP = P + (P & 1);
  static constexpr int T2 = 4 * PP * Q2, T3 = 4 * PP * Q3, T1 = 2 * P * Q1;
  static constexpr int VOL = E1 * E2 * E3;
  __host__ __device__ static constexpr int EV(int x) { return x + (x & 1); }
  static constexpr int WQ = EV(Q1 + Q2 + Q3);        // weights w1, w2, w3
  static constexpr int XU = E3 * E2 * Q1;            // floats per u X array
  static constexpr int YU = E3 * Q2 * Q1;            // floats per u Y array
  static constexpr int ZS = 6 * E2 * E1;             // floats of one slab's Z
  static constexpr int XG = 9 * E2 * Q1;             // floats of one slab's X (float2 pairs)
  static constexpr int NZ = ZALL ? Q3 : 2;
  __host__ __device__ static constexpr size_t smem_floats(bool stiff) {
    return (size_t)T2 + T3 + T1 + WQ + EV(VOL) + EV(3 * VOL) + (stiff ? 2 : 1) * XU +
           (stiff ? 3 : 1) * YU + (size_t)NZ * ZS + 2 * XG;
  }
};

template <int P, int S1, int S2, int S3, bool STIFF, bool ZALL>
__device__ __forceinline__ void apply3d_f32g_body(const ApplyParams &prm, const int tile) {
  using G = TileF2G<P, S1, S2, S3, ZALL>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int H1 = G::H1, PP = G::PP, NT = G::NT, NPAIR = G::NPAIR;
  constexpr int VOL = G::VOL, E21 = E2 * E1;

  extern __shared__ __align__(16) unsigned char smem_f32g[];
  float *sm = reinterpret_cast<float *>(smem_f32g);
  float *t2b = sm, *t2d = t2b + 2 * PP * Q2;        // [q2][PP] float2 {b, b}
  float *t3b = t2d + 2 * PP * Q2, *t3d = t3b + 2 * PP * Q3;
  float *t1b = t3d + 2 * PP * Q3, *t1d = t1b + P * Q1; // [j][q1]
  float *w1s = t1d + P * Q1, *w2s = w1s + Q1, *w3s = w2s + Q2;
  float *us = sm + G::T2 + G::T3 + G::T1 + G::WQ;
  float *cs = us + G::EV(VOL);                         // [c][n3][n2][n1]
  float2 *X0 = reinterpret_cast<float2 *>(cs + G::EV(3 * VOL));
  float2 *X1 = X0 + G::XU / 2;
  float2 *Y0 = STIFF ? X1 + G::XU / 2 : X0 + G::XU / 2;
  float2 *Y1 = Y0 + G::YU / 2, *Y2 = Y1 + G::YU / 2;
  float *Zs = reinterpret_cast<float *>(STIFF ? Y2 + G::YU / 2 : Y0 + G::YU / 2);
  float2 *Xg = reinterpret_cast<float2 *>(Zs + G::NZ * G::ZS);   // 2 buffers of XG floats

  const int tid = threadIdx.x;
  const int t1 = tile % prm.T[0];
  const int t2 = (tile / prm.T[0]) % prm.T[1];
  const int t3 = tile / (prm.T[0] * prm.T[1]);
  const int e01 = t1 * S1, e02 = t2 * S2, e03 = t3 * S3;
  const int ke3 = min(S3, prm.K[2] - e03);

  // ---- stage tables (the derivative tables too: the geometry needs them for
  // the mass as well), u, control points and weights
  stage_tile_f32<P, S1, S2, S3, NT, true>(prm, tid, e01, e02, e03, t1b, t1d, t2b, t2d, t3b, t3d, us);
  {
    constexpr int AC = (3 * VOL + NT - 1) / NT, AW = (Q1 + Q2 + Q3 + NT - 1) / NT;
    const int N1 = prm.N[0], N2 = prm.N[1], N3 = prm.N[2];
    const int64_t Ntot = (int64_t)N1 * N2 * N3;
    float cv[AC], wv[AW];
#pragma unroll
    for (int k = 0; k < AC; ++k) {
      const int i = tid + k * NT;
      const int c = i / VOL, l = i - c * VOL;
      const int n1 = l % E1, r = l / E1;
      const int n2 = r % E2, n3 = r / E2;
      const int g1 = e01 + n1, g2 = e02 + n2, g3 = e03 + n3;
      cv[k] = 0.f;
      if (i < 3 * VOL && g1 < N1 && g2 < N2 && g3 < N3)
        cv[k] = __ldg(prm.ctrl + c * Ntot + ((int64_t)g3 * N2 + g2) * N1 + g1);
    }
#pragma unroll
    for (int k = 0; k < AW; ++k) {
      const int i = tid + k * NT;
      wv[k] = 0.f;
      if (i < Q1) wv[k] = __ldg(prm.wq[0] + e01 * P + i);
      else if (i < Q1 + Q2) wv[k] = __ldg(prm.wq[1] + e02 * P + (i - Q1));
      else if (i < Q1 + Q2 + Q3) wv[k] = __ldg(prm.wq[2] + e03 * P + (i - Q1 - Q2));
    }
#pragma unroll
    for (int k = 0; k < AC; ++k) {
      const int i = tid + k * NT;
      if (i < 3 * VOL) cs[i] = cv[k];
    }
#pragma unroll
    for (int k = 0; k < AW; ++k) {
      const int i = tid + k * NT;
      if (i < Q1 + Q2 + Q3) w1s[i] = wv[k];
    }
  }
  __syncthreads();

  // Z of one slab: Z0_c = B3(q3) c_c, Z1_c = B3'(q3) c_c over the slab's p layers
  auto z_step = [&](const int q3, float *Z) {
    const int e3 = q3 / P;
    for (int i = tid; i < 3 * E21; i += NT) {
      const int c = i / E21, l = i - c * E21;
      const float *cp = cs + c * VOL + e3 * E21 + l;
      float z0 = 0.f, z1 = 0.f;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const float cv = cp[j * E21];
        z0 = fmaf(t3b[2 * (q3 * PP + j)], cv, z0);
        z1 = fmaf(t3d[2 * (q3 * PP + j)], cv, z1);
      }
      Z[2 * c * E21 + l] = z0;
      Z[(2 * c + 1) * E21 + l] = z1;
    }
  };

  if constexpr (ZALL) {
    for (int q3 = 0; q3 < ke3 * P; ++q3) z_step(q3, Zs + q3 * G::ZS);
  }

  // ---- A: direction 1, X0 = B1 u, X1 = B1' u
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

  // ---- B: direction 2, one (n3, element e2, pair) per item
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
      const float2 *b2 = reinterpret_cast<const float2 *>(t2b) + q2 * PP;
      const float2 *d2 = reinterpret_cast<const float2 *>(t2d) + q2 * PP;
      float2 y00 = make_float2(0.f, 0.f), y01 = y00, y10 = y00;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        y00 = ffma2(b2[j], xa[j], y00);
        if (STIFF) {
          y01 = ffma2(d2[j], xa[j], y01);
          y10 = ffma2(b2[j], xb[j], y10);
        }
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

  // ---- C: per slab, the geometry (Z, X cooperatively; J per pencil pair), the
  // factors, the direction-3 sweep of u, the product and the transposed sweep
  {
    const bool has_pair = tid < NPAIR;
    const int kk = tid % H1, q2 = tid / H1;
    const int e2 = q2 / P;
    // lanes in elements beyond the patch get zero factors
    const bool ok2 = e02 + e2 < prm.K[1];
    const bool oka = ok2 && e01 + (2 * kk) / P < prm.K[0];
    const bool okb = ok2 && e01 + (2 * kk + 1) / P < prm.K[0];
    float2 w12 = make_float2(0.f, 0.f);
    if (has_pair) w12 = make_float2(oka ? w1s[2 * kk] * w2s[q2] : 0.f, okb ? w1s[2 * kk + 1] * w2s[q2] : 0.f);
    float2 y0[E3], y1[E3], y2[E3], z0[E3], z1[E3], z2[E3];
#pragma unroll
    for (int n = 0; n < E3; ++n) {
      const float2 zero = make_float2(0.f, 0.f);
      y0[n] = has_pair ? Y0[n * NPAIR + tid] : zero;
      z0[n] = zero;
      if (STIFF) {
        y1[n] = has_pair ? Y1[n * NPAIR + tid] : zero;
        y2[n] = has_pair ? Y2[n * NPAIR + tid] : zero;
        z1[n] = zero;
        z2[n] = zero;
      }
    }
    const bool coef_var = STIFF && prm.coef_kind == IGASF_COEF_EXP_SIN_COS;
#pragma unroll
    for (int e3 = 0; e3 < S3; ++e3) {
      if (e3 < ke3) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq) {
          const int q3 = e3 * P + qq;
          const float *Z = ZALL ? Zs + q3 * G::ZS : Zs + (q3 & 1) * G::ZS;
          float2 *Xq = Xg + (q3 & 1) * (G::XG / 2);
          if constexpr (!ZALL) {
            z_step(q3, Zs + (q3 & 1) * G::ZS);
            __syncthreads();
          }
          // X: direction 1 of the slab's Z, one (c, n2, pair) per item
          for (int i = tid; i < 3 * E2 * H1; i += NT) {
            const int k = i % H1, r = i / H1;
            const int n2 = r % E2, c = r / E2;
            const int qa = 2 * k, ea = qa / P, eb = (qa + 1) / P;
            const float *zr0 = Z + 2 * c * E21 + n2 * E1;
            const float *zr1 = zr0 + E21;
            float2 x0 = make_float2(0.f, 0.f), x1 = x0, x2 = x0;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const float2 tb = *reinterpret_cast<const float2 *>(t1b + j * Q1 + qa);
              const float2 td = *reinterpret_cast<const float2 *>(t1d + j * Q1 + qa);
              const float2 v0 = make_float2(zr0[ea + j], zr0[eb + j]);
              const float2 v1 = make_float2(zr1[ea + j], zr1[eb + j]);
              x0 = ffma2(tb, v0, x0);
              x1 = ffma2(td, v0, x1);
              x2 = ffma2(tb, v1, x2);
            }
            Xq[(3 * c + 0) * E2 * H1 + n2 * H1 + k] = x0;
            Xq[(3 * c + 1) * E2 * H1 + n2 * H1 + k] = x1;
            Xq[(3 * c + 2) * E2 * H1 + n2 * H1 + k] = x2;
          }
          __syncthreads();
          if (!has_pair) continue;
          // J (and G) of the pencil pair: direction 2 of X
          const float2 *b2 = reinterpret_cast<const float2 *>(t2b) + q2 * PP;
          const float2 *d2 = reinterpret_cast<const float2 *>(t2d) + q2 * PP;
          float2 J[3][3], Gv[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 *x0 = Xq + (3 * c + 0) * E2 * H1 + e2 * H1 + kk;
            const float2 *x1 = Xq + (3 * c + 1) * E2 * H1 + e2 * H1 + kk;
            const float2 *x2 = Xq + (3 * c + 2) * E2 * H1 + e2 * H1 + kk;
            float2 g = make_float2(0.f, 0.f), j1 = g, j2 = g, j3 = g;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const float2 v0 = x0[j * H1];
              j1 = ffma2(b2[j], x1[j * H1], j1);
              j2 = ffma2(d2[j], v0, j2);
              j3 = ffma2(b2[j], x2[j * H1], j3);
              if (c < 2) g = ffma2(b2[j], v0, g);
            }
            J[c][0] = j1;
            J[c][1] = j2;
            J[c][2] = j3;
            if (c < 2) Gv[c] = g;
          }
          // cofactors C_ij of J, det J = sum_j J_0j C_0j
          auto cof = [](float2 a, float2 b, float2 c, float2 d) {   // a d - b c
            return ffma2(make_float2(-b.x, -b.y), c, fmul2(a, d));
          };
          const float2 C00 = cof(J[1][1], J[1][2], J[2][1], J[2][2]);
          const float2 C01 = cof(J[1][2], J[1][0], J[2][2], J[2][0]);
          const float2 C02 = cof(J[1][0], J[1][1], J[2][0], J[2][1]);
          const float2 det = ffma2(J[0][2], C02, ffma2(J[0][1], C01, fmul2(J[0][0], C00)));
          const float w3 = w3s[q3];
          const float2 w = make_float2(w12.x * w3, w12.y * w3);
          // b (basis values of direction 3) for the sweeps of u
          const float2 *b3 = reinterpret_cast<const float2 *>(t3b) + q3 * PP;
          const float2 *d3 = reinterpret_cast<const float2 *>(t3d) + q3 * PP;
          if (STIFF) {
            const float2 C10 = cof(J[0][2], J[0][1], J[2][2], J[2][1]);
            const float2 C11 = cof(J[0][0], J[0][2], J[2][0], J[2][2]);
            const float2 C12 = cof(J[0][1], J[0][0], J[2][1], J[2][0]);
            const float2 C20 = cof(J[0][1], J[0][2], J[1][1], J[1][2]);
            const float2 C21 = cof(J[0][2], J[0][0], J[1][2], J[1][0]);
            const float2 C22 = cof(J[0][0], J[0][1], J[1][0], J[1][1]);
            float2 a = make_float2(prm.coef_a, prm.coef_a);
            if (coef_var) {
              // fast hardware sine, cosine and exponential; the period is taken
              // out exactly first (x - rint(x) in [-1/2, 1/2]), so the sine and
              // cosine see arguments in [-pi, pi], where their absolute error
              // (~1e-6) is far inside the FP32 tolerance
              constexpr float twopi = 6.28318530717958647692f;
              const float sx = __sinf(twopi * (Gv[0].x - rintf(Gv[0].x)));
              const float sy = __sinf(twopi * (Gv[0].y - rintf(Gv[0].y)));
              const float cx = __cosf(twopi * (Gv[1].x - rintf(Gv[1].x)));
              const float cy = __cosf(twopi * (Gv[1].y - rintf(Gv[1].y)));
              a.x = __expf(prm.coef_a * sx * cx);
              a.y = __expf(prm.coef_a * sy * cy);
            }
            const float2 s = make_float2(w.x > 0.f ? __fdividef(w.x * a.x, fabsf(det.x)) : 0.f,
                                         w.y > 0.f ? __fdividef(w.y * a.y, fabsf(det.y)) : 0.f);
            const float2 D11 = fmul2(s, ffma2(C20, C20, ffma2(C10, C10, fmul2(C00, C00))));
            const float2 D12 = fmul2(s, ffma2(C20, C21, ffma2(C10, C11, fmul2(C00, C01))));
            const float2 D13 = fmul2(s, ffma2(C20, C22, ffma2(C10, C12, fmul2(C00, C02))));
            const float2 D22 = fmul2(s, ffma2(C21, C21, ffma2(C11, C11, fmul2(C01, C01))));
            const float2 D23 = fmul2(s, ffma2(C21, C22, ffma2(C11, C12, fmul2(C01, C02))));
            const float2 D33 = fmul2(s, ffma2(C22, C22, ffma2(C12, C12, fmul2(C02, C02))));
            float2 g1 = make_float2(0.f, 0.f), g2 = g1, g3 = g1;
            {
              float2 du1 = make_float2(0.f, 0.f), du2 = du1, du3 = du1;
#pragma unroll
              for (int j = 0; j < P; ++j) {
                du3 = ffma2(d3[j], y0[e3 + j], du3);
                du2 = ffma2(b3[j], y1[e3 + j], du2);
                du1 = ffma2(b3[j], y2[e3 + j], du1);
              }
              g1 = ffma2(D13, du3, ffma2(D12, du2, fmul2(D11, du1)));
              g2 = ffma2(D23, du3, ffma2(D22, du2, fmul2(D12, du1)));
              g3 = ffma2(D33, du3, ffma2(D23, du2, fmul2(D13, du1)));
            }
#pragma unroll
            for (int j = 0; j < P; ++j) {
              z0[e3 + j] = ffma2(d3[j], g3, z0[e3 + j]);
              z1[e3 + j] = ffma2(b3[j], g2, z1[e3 + j]);
              z2[e3 + j] = ffma2(b3[j], g1, z2[e3 + j]);
            }
          } else {
            const float2 dm = make_float2(w.x * fabsf(det.x), w.y * fabsf(det.y));
            float2 uq = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < P; ++j) uq = ffma2(b3[j], y0[e3 + j], uq);
            const float2 wv = fmul2(dm, uq);
#pragma unroll
            for (int j = 0; j < P; ++j) z0[e3 + j] = ffma2(b3[j], wv, z0[e3 + j]);
          }
        }
      }
    }
    __syncthreads();   // every X buffer read before phase D reuses X0 / X1
    if (has_pair) {
#pragma unroll
      for (int n = 0; n < E3; ++n) {
        Y0[n * NPAIR + tid] = z0[n];
        if (STIFF) {
          Y1[n * NPAIR + tid] = z1[n];
          Y2[n * NPAIR + tid] = z2[n];
        }
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
      const float2 *b2 = reinterpret_cast<const float2 *>(t2b) + q2 * PP;
      const float2 *d2 = reinterpret_cast<const float2 *>(t2d) + q2 * PP;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        ya[e2 + j] = ffma2(b2[j], w3, ya[e2 + j]);
        if (STIFF) {
          ya[e2 + j] = ffma2(d2[j], w2, ya[e2 + j]);
          yb[e2 + j] = ffma2(b2[j], w1, yb[e2 + j]);
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

  // ---- E: transposed direction 1, one (n3, n2) row per item
  float *vp = static_cast<float *>(prm.vpart) + (size_t)tile * VOL;
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

template <int P, int S1, int S2, int S3, bool STIFF, bool ZALL>
__global__ void __launch_bounds__(TileF2G<P, S1, S2, S3, ZALL>::NT)
apply3d_f32g_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_f32g_body<P, S1, S2, S3, STIFF, ZALL>(prm, blockIdx.x);
}

template <int P, int S1, int S2, int S3, bool STIFF, bool ZALL>
cudaError_t launch_apply3d_f32g(const ApplyParams &prm, cudaStream_t s) {
  using G = TileF2G<P, S1, S2, S3, ZALL>;
  apply3d_f32g_kernel<P, S1, S2, S3, STIFF, ZALL>
      <<<prm.ntiles, G::NT, G::smem_floats(STIFF) * sizeof(float), s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool ZALL>
cudaError_t prepare_apply3d_f32g() {
  using G = TileF2G<P, S1, S2, S3, ZALL>;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(apply3d_f32g_kernel<P, S1, S2, S3, false, ZALL>, a,
                                       (int)(G::smem_floats(false) * sizeof(float)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply3d_f32g_kernel<P, S1, S2, S3, true, ZALL>, a,
                             (int)(G::smem_floats(true) * sizeof(float)));
  return e;
}

template <int P, int S1, int S2, int S3, bool ZALL = true>
ApplyKernel make_apply3d_f32g() {
  using G = TileF2G<P, S1, S2, S3, ZALL>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  static_assert(G::smem_floats(true) * sizeof(float) <= 227 * 1024, "tile exceeds shared memory");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = S3;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_floats(false) * sizeof(float);
  k.smem[IGASF_STIFFNESS] = G::smem_floats(true) * sizeof(float);
  k.plane = 0;
  k.lanes = 2;
  k.variant = IGASF_KERNEL_ON_THE_FLY;
  k.launch[IGASF_MASS] = &launch_apply3d_f32g<P, S1, S2, S3, false, ZALL>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d_f32g<P, S1, S2, S3, true, ZALL>;
  k.launch_batched[IGASF_MASS] = nullptr;
  k.launch_batched[IGASF_STIFFNESS] = nullptr;
  k.prepare = &prepare_apply3d_f32g<P, S1, S2, S3, ZALL>;
  return k;
}

}  // namespace igasf
