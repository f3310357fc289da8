// FP32 tile kernel whose direction-3 sweeps run on the tensor cores.
//
// Same five phases as the packed FP32 kernels (apply3d_f32r.cuh: Alg. 3, the
// product with w F, Alg. 2, localized per Sec. 4), but phase C, the last
// forward sweep, the product and the first transposed sweep, which carry about
// three quarters of the multiply-adds at p >= 6, are small dense products per
// warp (the Kronecker form of Sec. 5: along direction 3 the operator factor is
// the banded 1D matrix B3 or B3', dense inside a window of p consecutive dofs
// per element):
//
//   forward     d[16 pencils x 8 q3]  = Y[16 pencils x window of dofs j3] B3^T[window x 8 q3]
//   transposed  W[16 pencils x 8 j3] += g[16 pencils x 8 (or 16) q3] B3[q3 x 8 j3]
//
// issued as mma.sync with FP32 accumulation, in one of two operand formats:
//   MK = TC_TF32: m16n8k8 with TF32 operands (11 significant bits, round to
//                 nearest, ties away) for the FP32-stored factors (IGASF_TF32);
//   MK = TC_BF16: m16n8k16 with bfloat16 operands (8 significant bits, round to
//                 nearest even) for the bfloat16-stored factors (IGASF_BF16_MMA).
// The operands rounded to the narrow format are the direction-2 results Y, the
// products g and the direction-3 tables; accumulation, the other sweeps (phases
// A, B, D, E on the FP32 FMA pipe, packed FFMA2) and the product with w F stay
// FP32.
//
// Fragment bookkeeping. A warp owns m-tiles of 16 pencils = 8 consecutive pencil
// pairs of the factor layout (layout.h, lanes = 2): fragment rows g and g + 8
// (g = lane / 4) are the two pencils of pair 8 mt + g. The accumulator of a
// forward product holds, per thread, rows g, g + 8 at quadrature columns
// 2t, 2t + 1 (t = lane % 4) of its n-tile: exactly the two pencils of one pair
// at two consecutive factor slabs, so each thread reads its factors as the
// chunks of its pair in two slabs (128-bit loads, 128 contiguous bytes per slab
// and warp) and the product needs no data exchange. The accumulator then serves
// as the A operand of the transposed product: for BF16 the k16 A fragment of
// two consecutive n-tiles is the two accumulators side by side; for TF32 the
// k8 fragment takes the columns in the order 2t, 2t + 1 -> t, t + 4, a
// permutation of the contraction index that the B fragment (the table, built in
// shared memory at staging in the same permuted order) mirrors.
// The direction-3 tables are staged once per tile as ready-made B fragments
// (rounded to the operand format), zero outside each element's window, so the
// band structure costs no branches; windows of the forward sweep start at the
// first dof of the n-tile's first element and A rows past the tile's dofs are
// clamped to the last one (finite data times a zero table entry).
#pragma once

#include "apply3d_f32.cuh"
#include "apply3d_f32r.cuh"
#include "igasf_internal.h"
#include "layout.h"

namespace igasf {

enum { TC_TF32 = 0, TC_BF16 = 1 };

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// two floats as one bfloat16x2 word: lo in the low half (the smaller k)
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int P, int S1, int S2, int S3, int MK>
struct TileTC {
  static constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1, E3 = S3 + P - 1;
  static constexpr int Q1 = S1 * P, Q2 = S2 * P, Q3 = S3 * P;
  static_assert(Q1 % 2 == 0, "pencil pairs need an even number of q1 points per tile");
  static constexpr int H1 = Q1 / 2;
  static constexpr int NPEN = Q1 * Q2;
  static constexpr int PL = (NPEN + 7) / 8 * 8;     // factor layout row (pencils)
  static constexpr int UNITS = PL / 2;              // pairs per layout row
  static constexpr int NPAIR = H1 * Q2;
  static constexpr int NMT = (NPAIR + 7) / 8;       // m-tiles of 16 pencils
  static constexpr int MPEN = 16 * NMT;
  // Y plane stride (floats): conflict-free A-fragment loads, rows t (TF32) or
  // 2t (BF16) apart for the four thread groups of a half warp
  static constexpr int YMOD = MK == TC_TF32 ? 8 : 4;
  static constexpr int YS = (MPEN + 31 - YMOD) / 32 * 32 + YMOD;
  static constexpr int YS2 = YS / 2;                // in float2
  static constexpr int NQT = (Q3 + 7) / 8;          // n-tiles of 8 quadrature points (dir 3)
  static constexpr int NQP = (NQT + 1) / 2;         // pairs of them (BF16 transposed step)
  static constexpr int JT = (E3 + 7) / 8;           // n-tiles of 8 dofs (dir 3)
  static constexpr int PP = P + (P & 1);
  // forward window of n-tile nt: dofs wlo .. whi (the elements of its points)
  __host__ __device__ static constexpr int wlo(int nt) { return (8 * nt) / P; }
  __host__ __device__ static constexpr int whi(int nt) { return cmin(8 * nt + 7, Q3 - 1) / P + P - 1; }
  __host__ __device__ static constexpr int kf_of(int nt) {
    return (whi(nt) - wlo(nt) + (MK == TC_TF32 ? 8 : 16)) / (MK == TC_TF32 ? 8 : 16);
  }
  __host__ __device__ static constexpr int kf_max() {
    int m = 1;
    for (int nt = 0; nt < NQT; ++nt) m = cmax(m, kf_of(nt));
    return m;
  }
  static constexpr int KF = kf_max();               // k-steps of the forward product
  // output dof tiles of the transposed step: n-tile nt (TF32) or pair i (BF16)
  __host__ __device__ static constexpr int qlo_t(int s) { return MK == TC_TF32 ? 8 * s : 16 * s; }
  __host__ __device__ static constexpr int qhi_t(int s) {
    return cmin((MK == TC_TF32 ? 8 * s + 7 : 16 * s + 15), Q3 - 1);
  }
  __host__ __device__ static constexpr int jt0(int s) { return (qlo_t(s) / P) / 8; }
  __host__ __device__ static constexpr int jt1(int s) { return cmin(qhi_t(s) / P + P - 1, E3 - 1) / 8; }
  static constexpr int NSTEP = MK == TC_TF32 ? NQT : NQP;   // transposed steps
  static constexpr int NJ = 3;                              // dof tiles per step, at most
  __host__ __device__ static constexpr bool nj_ok() {
    for (int s = 0; s < NSTEP; ++s)
      if (jt1(s) - jt0(s) + 1 > NJ) return false;
    return true;
  }
  static_assert(nj_ok(), "a transposed step touches more than NJ dof tiles");
  static constexpr int T2 = 4 * PP * Q2;            // dup tables of dir 2 (B, B'), floats
  static constexpr int T1 = 2 * P * Q1;             // dir-1 tables [j][q1] (B, B')
  static constexpr int X = E3 * E2 * Q1;            // floats per X array
  static constexpr int Y = E3 * YS;                 // floats per Y array
  static constexpr int VOL = E1 * E2 * E3;
  // fragment tables, in 32-bit words: [table][step][j][lane][2]
  static constexpr int FWW = NQT * KF * 64;         // forward, per table
  static constexpr int BWW = NSTEP * NJ * 64;       // transposed, per table
  static constexpr size_t smem_words(bool stiff) {
    return (size_t)(stiff ? 2 : 1) * (FWW + BWW) + T2 + T1 + (stiff ? 2 : 1) * X +
           (stiff ? 3 : 1) * Y + VOL;
  }
};

template <int P, int S1, int S2, int S3, int MK, bool STIFF, bool BF, int NW>
__device__ __forceinline__ void apply3d_tc_body(const ApplyParams &prm, const int tile) {
  using G = TileTC<P, S1, S2, S3, MK>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int H1 = G::H1, PP = G::PP, UNITS = G::UNITS, NMT = G::NMT, YS2 = G::YS2;
  constexpr int NQT = G::NQT, KF = G::KF, NJ = G::NJ, JT = G::JT, NSTEP = G::NSTEP;
  constexpr int NT = 32 * NW;
  constexpr int NTAB = STIFF ? 2 : 1;               // B3 (and B3')
  constexpr int NCH = STIFF ? 3 : 1;                // factor chunks of a pair per slab
  constexpr int NF = STIFF ? 3 : 1;                 // fields through phase C
  using Chunk = typename FactorChunk<STIFF, BF>::type;

  extern __shared__ __align__(16) unsigned char smem_tc[];
  uint32_t *fw = reinterpret_cast<uint32_t *>(smem_tc);       // [NTAB][NQT][KF][32][2]
  uint32_t *bw = fw + NTAB * G::FWW;                          // [NTAB][NSTEP][NJ][32][2]
  float *t2b = reinterpret_cast<float *>(bw + NTAB * G::BWW); // [q2][PP] float2 {b, b}
  float *t2d = t2b + 2 * PP * Q2;
  float *t1b = t2d + 2 * PP * Q2, *t1d = t1b + P * Q1;        // [j][q1]
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

  // ---- factor chunks of m-tile mtl, n-tile nt: its pairs at slabs 8 nt + 2t + s,
  // s = 0, 1 (zero beyond the patch or the layout row). The warp's first m-tile
  // requests its first n-tile now, so that the latency overlaps the staging and
  // phases A and B; later n-tiles are requested one step ahead, and the next
  // m-tile's first n-tile during the last step of the current one.
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const Chunk *Dc = reinterpret_cast<const Chunk *>(prm.D) + (size_t)tile * Q3 * NCH * UNITS;
  auto load_factors = [&](const int mtl, const int nt, Chunk (&fc)[2][NCH]) {
    const int un = 8 * mtl + g;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int q3 = 8 * nt + 2 * t + s;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        if (un < UNITS && q3 < nslab) fc[s][c] = ldg_stream(Dc + ((size_t)q3 * NCH + c) * UNITS + un);
        else fc[s][c] = Chunk{};
      }
    }
  };
  // the tile's first factor slabs into L2 (the stream from DRAM then runs
  // during staging and phases A and B): the whole tile where it is small, else
  // about 96 KB (every warp walks all slabs once per m-tile, so a rolling
  // window per warp would not fit the block's access order)
  {
    constexpr uint32_t SLAB_ROW = (uint32_t)(NCH * UNITS * sizeof(Chunk));
    prefetch_factor_slabs(Dc, SLAB_ROW, 0, min(l2_window_slabs((int)SLAB_ROW, Q3), nslab), tid, NT);
  }
  Chunk fc[2][2][NCH];
  if (warp < NMT) load_factors(warp, 0, fc[0]);

  // ---- stage: direction-1/2 tables and the u box (as the packed kernels) ...
  stage_tile_f32<P, S1, S2, S3, NT, STIFF, false>(prm, tid, e01, e02, e03, t1b, t1d, t2b, t2d,
                                                  nullptr, nullptr, us);
  // ... and the direction-3 tables as B fragments. tab3(x, q3, j3): value
  // (x = 0) or derivative (x = 1) of dof j3 of the tile at point q3, zero
  // outside the element's window and beyond the tile.
  {
    const float *gb3 = static_cast<const float *>(prm.tabB[2]);
    const float *gd3 = static_cast<const float *>(prm.tabD[2]);
    const int qoff = e03 * P, qpad = prm.Qpad[2];
    auto tab3 = [&](int x, int q3, int j3) -> float {
      const int j = j3 - q3 / P;
      if (q3 >= Q3 || j < 0 || j >= P) return 0.f;
      return __ldg((x ? gd3 : gb3) + j * qpad + qoff + q3);
    };
    for (int i = tid; i < NTAB * NQT * KF * 32; i += NT) {
      const int lane = i & 31, r = i >> 5;
      const int ks = r % KF, nt = (r / KF) % NQT, x = r / (KF * NQT);
      const int g = lane >> 2, t = lane & 3;
      const int q3 = 8 * nt + g, wl = G::wlo(nt);
      uint32_t w0, w1;
      if constexpr (MK == TC_TF32) {
        w0 = tf32_bits(tab3(x, q3, wl + 8 * ks + t));
        w1 = tf32_bits(tab3(x, q3, wl + 8 * ks + t + 4));
      } else {
        const int j = wl + 16 * ks + 2 * t;
        w0 = bf16x2_bits(tab3(x, q3, j), tab3(x, q3, j + 1));
        w1 = bf16x2_bits(tab3(x, q3, j + 8), tab3(x, q3, j + 9));
      }
      fw[2 * i] = w0;
      fw[2 * i + 1] = w1;
    }
    for (int i = tid; i < NTAB * NSTEP * NJ * 32; i += NT) {
      const int lane = i & 31, r = i >> 5;
      const int j = r % NJ, s = (r / NJ) % NSTEP, x = r / (NJ * NSTEP);
      const int g = lane >> 2, t = lane & 3;
      const int jt = G::jt0(s) + j, j3 = 8 * jt + g;
      uint32_t w0 = 0u, w1 = 0u;
      if (jt <= G::jt1(s)) {
        if constexpr (MK == TC_TF32) {
          w0 = tf32_bits(tab3(x, 8 * s + 2 * t, j3));      // k = t     <-> q3 = 8s + 2t
          w1 = tf32_bits(tab3(x, 8 * s + 2 * t + 1, j3));  // k = t + 4 <-> q3 = 8s + 2t + 1
        } else {
          const int q = 16 * s + 2 * t;
          w0 = bf16x2_bits(tab3(x, q, j3), tab3(x, q + 1, j3));
          w1 = bf16x2_bits(tab3(x, q + 8, j3), tab3(x, q + 9, j3));
        }
      }
      bw[2 * i] = w0;
      bw[2 * i + 1] = w1;
    }
  }
  // the padding pencils of the last m-tile enter the products: keep them zero
  if constexpr (G::MPEN > G::NPEN) {
    constexpr int PADP = (G::MPEN - G::NPEN) / 2;   // float2 per row
    for (int i = tid; i < NF * E3 * PADP; i += NT) {
      const int c = i % PADP, r = i / PADP;
      const int f = r / E3, n = r % E3;
      float2 *Yf = f == 0 ? Y0 : (f == 1 ? Y1 : Y2);
      Yf[n * YS2 + G::NPEN / 2 + c] = make_float2(0.f, 0.f);
    }
  }
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
      const int idx = n3 * YS2 + q2 * H1 + k;
      Y0[idx] = y00;
      if (STIFF) {
        Y1[idx] = y01;
        Y2[idx] = y10;
      }
    }
  }
  __syncthreads();

  // ---- C on the tensor cores: per m-tile, for every n-tile of quadrature points
  // the forward products d = Y B3^T (d3 u from Y00 with B3', d2 u from Y01 and
  // d1 u from Y10 with B3), the product g = D grad u with the factors of the
  // thread's pair at its two slabs, and the transposed products into the dof
  // accumulators W3 = B3'^T g3, W2 = B3^T g2, W1 = B3^T g1 (mass: u, w = D u, B3^T w).
  {
    const bool full = nslab == Q3;   // no ragged slabs: the next m-tile's loads may start early
    const float2 *Yf[3] = {Y0, STIFF ? Y1 : Y0, STIFF ? Y2 : Y0};
    const uint2 *fw2 = reinterpret_cast<const uint2 *>(fw);
    const uint2 *bw2 = reinterpret_cast<const uint2 *>(bw);
    for (int mt = warp; mt < NMT; mt += NW) {
      const int unit = 8 * mt + g;
      const bool more = mt + NW < NMT;
      if (mt != warp) {
        if (!full) {
          load_factors(mt, 0, fc[0]);
        } else if constexpr (MK == TC_TF32 && (NQT & 1)) {
          // requested into the buffer after the last n-tile's
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int c = 0; c < NCH; ++c) fc[0][s2][c] = fc[1][s2][c];
        }
      }
      float za[NF][JT][4];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int jt = 0; jt < JT; ++jt)
#pragma unroll
          for (int c = 0; c < 4; ++c) za[f][jt][c] = 0.f;
      // forward product of n-tile nt and product with the factors: gq[f][4]
      // holds g (stiffness: g1, g2, g3; mass: w) at the accumulator positions
      auto forward_product = [&](const int nt, const Chunk (&fc)[2][NCH], float (&gq)[NF][4]) {
        float dv[NF][4];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int c = 0; c < 4; ++c) dv[f][c] = 0.f;
        const int wl = G::wlo(nt);
#pragma unroll
        for (int ks = 0; ks < KF; ++ks) {
          uint2 bb = fw2[((0 * NQT + nt) * KF + ks) * 32 + lane];
          uint2 bd = STIFF ? fw2[((1 * NQT + nt) * KF + ks) * 32 + lane] : bb;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            // fields: f = 0 -> d1 u from Y10 (Y2), f = 1 -> d2 u from Y01 (Y1),
            // f = 2 -> d3 u from Y00 (Y0) with the derivative table; mass: Y0
            const float2 *Ys = STIFF ? Yf[2 - f] : Yf[0];
            const uint2 bt = (STIFF && f == 2) ? bd : bb;
            if constexpr (MK == TC_TF32) {
              const int ja = min(wl + 8 * ks + t, E3 - 1), jb = min(wl + 8 * ks + t + 4, E3 - 1);
              const float2 ya = Ys[ja * YS2 + unit];
              const float2 yb = Ys[jb * YS2 + unit];
              mma_tf32(dv[f], tf32_bits(ya.x), tf32_bits(ya.y), tf32_bits(yb.x), tf32_bits(yb.y), bt.x, bt.y);
            } else {
              const int j = wl + 16 * ks + 2 * t;
              const float2 r0 = Ys[min(j, E3 - 1) * YS2 + unit];
              const float2 r1 = Ys[min(j + 1, E3 - 1) * YS2 + unit];
              const float2 r2 = Ys[min(j + 8, E3 - 1) * YS2 + unit];
              const float2 r3 = Ys[min(j + 9, E3 - 1) * YS2 + unit];
              mma_bf16(dv[f], bf16x2_bits(r0.x, r1.x), bf16x2_bits(r0.y, r1.y), bf16x2_bits(r2.x, r3.x),
                       bf16x2_bits(r2.y, r3.y), bt.x, bt.y);
            }
          }
        }
        // accumulator positions: [0] pencil 0 slab 0, [1] pencil 0 slab 1,
        // [2] pencil 1 slab 0, [3] pencil 1 slab 1
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if constexpr (STIFF) {
            const float4 c0 = widen(fc[s][0]), c1 = widen(fc[s][1]), c2 = widen(fc[s][2]);
            const float2 D11 = make_float2(c0.x, c0.y), D12 = make_float2(c0.z, c0.w);
            const float2 D13 = make_float2(c1.x, c1.y), D22 = make_float2(c1.z, c1.w);
            const float2 D23 = make_float2(c2.x, c2.y), D33 = make_float2(c2.z, c2.w);
            const float2 d1 = make_float2(dv[0][s], dv[0][2 + s]);
            const float2 d2 = make_float2(dv[1][s], dv[1][2 + s]);
            const float2 d3 = make_float2(dv[2][s], dv[2][2 + s]);
            const float2 g1 = ffma2(D13, d3, ffma2(D12, d2, fmul2(D11, d1)));
            const float2 g2 = ffma2(D23, d3, ffma2(D22, d2, fmul2(D12, d1)));
            const float2 g3 = ffma2(D33, d3, ffma2(D23, d2, fmul2(D13, d1)));
            gq[0][s] = g1.x; gq[0][2 + s] = g1.y;
            gq[1][s] = g2.x; gq[1][2 + s] = g2.y;
            gq[2][s] = g3.x; gq[2][2 + s] = g3.y;
          } else {
            const float2 dm = widen(fc[s][0]);
            gq[0][s] = dm.x * dv[0][s];
            gq[0][2 + s] = dm.y * dv[0][2 + s];
          }
        }
      };
      // transposed product of step s (TF32: n-tile s; BF16: n-tiles 2s, 2s + 1)
      // into the dof accumulators; ga, gb: g of the step's n-tile(s)
      auto transposed = [&](const int s, const float (&ga)[NF][4], const float (&gb)[NF][4]) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int jt = G::jt0(s) + j;
          if (jt <= G::jt1(s)) {
            const uint2 bb = bw2[((0 * NSTEP + s) * NJ + j) * 32 + lane];
            const uint2 bd = STIFF ? bw2[((1 * NSTEP + s) * NJ + j) * 32 + lane] : bb;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              // W1 = B3^T g1 (f = 0), W2 = B3^T g2 (f = 1), W3 = B3'^T g3 (f = 2)
              const uint2 bt = (STIFF && f == 2) ? bd : bb;
              if constexpr (MK == TC_TF32) {
                mma_tf32(za[f][jt], tf32_bits(ga[f][0]), tf32_bits(ga[f][2]), tf32_bits(ga[f][1]),
                         tf32_bits(ga[f][3]), bt.x, bt.y);
              } else {
                mma_bf16(za[f][jt], bf16x2_bits(ga[f][0], ga[f][1]), bf16x2_bits(ga[f][2], ga[f][3]),
                         bf16x2_bits(gb[f][0], gb[f][1]), bf16x2_bits(gb[f][2], gb[f][3]), bt.x, bt.y);
              }
            }
          }
        }
      };

#pragma unroll
      for (int s = 0; s < NSTEP; ++s) {
        if constexpr (MK == TC_TF32) {
          const int nt = s;
          if (8 * nt < nslab) {
            if (nt + 1 < NQT) load_factors(mt, nt + 1, fc[(nt + 1) & 1]);
            else if (full && more) load_factors(mt + NW, 0, fc[(nt + 1) & 1]);
            float gq[NF][4];
            forward_product(nt, fc[nt & 1], gq);
            transposed(s, gq, gq);
          }
        } else {
          const int na = 2 * s, nb = 2 * s + 1;
          if (8 * na < nslab) {
            float gqa[NF][4], gqb[NF][4];
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
              for (int c = 0; c < 4; ++c) gqb[f][c] = 0.f;
            if (nb < NQT) load_factors(mt, nb, fc[1]);
            forward_product(na, fc[0], gqa);
            // the next request into the freed buffer: n-tile nb + 1 of this
            // m-tile, or the next m-tile's first n-tile
            if (nb + 1 < NQT) load_factors(mt, nb + 1, fc[0]);
            else if (full && more) load_factors(mt + NW, 0, fc[0]);
            if (nb < NQT && 8 * nb < nslab) forward_product(nb, fc[1], gqb);
            transposed(s, gqa, gqb);
          }
        }
      }
      // dof accumulators back to shared memory, in place of this m-tile's Y:
      // [0] pencil 0 dof 2t, [1] pencil 0 dof 2t + 1, [2] pencil 1 dof 2t, [3] pencil 1 dof 2t + 1
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        float2 *Wf = STIFF ? (f == 0 ? Y2 : (f == 1 ? Y1 : Y0)) : Y0;
#pragma unroll
        for (int jt = 0; jt < JT; ++jt) {
          const int ja = 8 * jt + 2 * t;
          if (ja < E3) Wf[ja * YS2 + unit] = make_float2(za[f][jt][0], za[f][jt][2]);
          if (ja + 1 < E3) Wf[(ja + 1) * YS2 + unit] = make_float2(za[f][jt][1], za[f][jt][3]);
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
      const int idx = n3 * YS2 + q2 * H1 + k;
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

template <int P, int S1, int S2, int S3, int MK, bool STIFF, bool BF, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) apply3d_tc_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_tc_body<P, S1, S2, S3, MK, STIFF, BF, NW>(prm, blockIdx.x);
}

template <int P, int S1, int S2, int S3, int MK, bool STIFF, bool BF, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) apply3d_tc_batched(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  apply3d_tc_body<P, S1, S2, S3, MK, STIFF, BF, NW>(bp.params[patch], blockIdx.x - bp.first_block[patch]);
}

template <int P, int S1, int S2, int S3, int MK, bool STIFF, bool BF, int NW, int MINB>
cudaError_t launch_apply3d_tc(const ApplyParams &prm, cudaStream_t s) {
  using G = TileTC<P, S1, S2, S3, MK>;
  const size_t sh = G::smem_words(STIFF) * 4;
  apply3d_tc_kernel<P, S1, S2, S3, MK, STIFF, BF, NW, MINB><<<prm.ntiles, 32 * NW, sh, s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, int MK, bool STIFF, bool BF, int NW, int MINB>
cudaError_t launch_apply3d_tc_batched(const BatchParams &bp, int blocks, cudaStream_t s) {
  using G = TileTC<P, S1, S2, S3, MK>;
  const size_t sh = G::smem_words(STIFF) * 4;
  apply3d_tc_batched<P, S1, S2, S3, MK, STIFF, BF, NW, MINB><<<blocks, 32 * NW, sh, s>>>(bp);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, int MK, bool BF, int NW, int MINB>
cudaError_t prepare_apply3d_tc() {
  using G = TileTC<P, S1, S2, S3, MK>;
  const int sm = (int)(G::smem_words(false) * 4), sk = (int)(G::smem_words(true) * 4);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(apply3d_tc_kernel<P, S1, S2, S3, MK, false, BF, NW, MINB>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_tc_kernel<P, S1, S2, S3, MK, true, BF, NW, MINB>, a, sk);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_tc_batched<P, S1, S2, S3, MK, false, BF, NW, MINB>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_tc_batched<P, S1, S2, S3, MK, true, BF, NW, MINB>, a, sk);
  return e;
}

// MK = TC_TF32 with FP32-stored factors (IGASF_TF32), TC_BF16 with
// bfloat16-stored factors (IGASF_BF16_MMA). NW: warps per block. MINB: minimum
// resident blocks per SM asked of the register allocator.
template <int P, int S1, int S2, int S3, int MK, int NW = 8, int MINB = 1>
ApplyKernel make_apply3d_tc() {
  using G = TileTC<P, S1, S2, S3, MK>;
  constexpr bool BF = MK == TC_BF16;
  static_assert(32 * NW <= 1024, "block too large");
  static_assert(G::smem_words(true) * 4 <= 227 * 1024, "tile exceeds shared memory");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = S3;
  k.threads = 32 * NW;
  k.smem[IGASF_MASS] = G::smem_words(false) * 4;
  k.smem[IGASF_STIFFNESS] = G::smem_words(true) * 4;
  k.plane = G::PL;
  k.lanes = 2;
  k.variant = IGASF_KERNEL_MMA;
  k.launch[IGASF_MASS] = &launch_apply3d_tc<P, S1, S2, S3, MK, false, BF, NW, MINB>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d_tc<P, S1, S2, S3, MK, true, BF, NW, MINB>;
  k.launch_batched[IGASF_MASS] = &launch_apply3d_tc_batched<P, S1, S2, S3, MK, false, BF, NW, MINB>;
  k.launch_batched[IGASF_STIFFNESS] = &launch_apply3d_tc_batched<P, S1, S2, S3, MK, true, BF, NW, MINB>;
  k.prepare = &prepare_apply3d_tc<P, S1, S2, S3, MK, BF, NW, MINB>;
  return k;
}

}  // namespace igasf
