// FP32 tile kernel of the 3D apply with packed FP32x2 arithmetic (sm_100+
// FFMA2): each consumer thread owns a PAIR of neighbouring quadrature pencils
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
// The factors stream through a ring of R slab buffers in shared memory, filled
// by bulk copies (cp.async.bulk, the TMA engine) that one lane of a dedicated
// producer warp issues from kernel entry on, so the factor stream overlaps the
// staging and the first two sweeps, with up to R slabs per block in flight. A
// block may walk several tiles (the producer then runs ahead across tile
// boundaries); the launch uses one block per tile.
// Each slot has a "full" mbarrier (the copy's transaction count) and an
// "empty" mbarrier (one arrival per consumer warp once it has read the slot).
// Every wait is bounded in clock cycles; a wait that runs out sets the plan's
// device status word and the kernel carries on (its result is then invalid and
// the host sees IGASF_ERR_TIMEOUT from igasf_device_status).
// Tables of directions 2 and 3 are held as duplicated pairs {b, b} so that one
// 128-bit load feeds two FFMA2 table operands; the X and Y arrays have padded
// row strides so the register-blocked sweeps read shared memory without bank
// conflicts.
// BF (template flag): the factors are stored in bfloat16 (half the slab
// bytes) and widened to FP32 when read; everything else is unchanged.
#pragma once

#include "igasf_internal.h"
#include "layout.h"

namespace igasf {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Shared-memory load the compiler may not merge with an earlier load of the
// same address (keeps a value out of registers between two uses).
__device__ __forceinline__ float4 lds_volatile4(const float4 *p) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))));
  return r;
}

// ---- stored factor chunks of one pencil pair (layout.h: [chunk][unit][CE]) ----
// FP32: a float4 holds two fields of both pencils (stiffness, three chunks), a
// float2 the one mass field of both pencils. bfloat16: the same values in half
// the bytes (uint2, one 32-bit word); each 32-bit word is one field of the two
// pencils, and widening is exact (bfloat16 is the high half of an FP32 word).
template <bool STIFF, bool BF> struct FactorChunk;
template <> struct FactorChunk<true, false> { using type = float4; };
template <> struct FactorChunk<false, false> { using type = float2; };
template <> struct FactorChunk<true, true> { using type = uint2; };
template <> struct FactorChunk<false, true> { using type = uint32_t; };

__device__ __forceinline__ float2 bf16x2_to_float2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ float4 widen(float4 c) { return c; }
__device__ __forceinline__ float2 widen(float2 c) { return c; }
__device__ __forceinline__ float4 widen(uint2 c) {
  const float2 a = bf16x2_to_float2(c.x), b = bf16x2_to_float2(c.y);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float2 widen(uint32_t c) { return bf16x2_to_float2(c); }

// ---- staging of one tile: the tables of the three directions and the u box
// (the selection S_D u of eq. loc-basis-change). Every global load of a thread
// is issued through the read-only path before its first shared-memory store,
// so the block waits for one round of load latency instead of one per loop
// trip. Tables of directions 2 and 3 are stored as duplicated pairs {b, b},
// padded with zeros to PP entries per quadrature point. DIR3 = false skips the
// direction-3 tables (kernels that stage them in another form).
template <int P, int S1, int S2, int S3, int NT, bool STIFF, bool DIR3 = true>
__device__ __forceinline__ void stage_tile_f32(const ApplyParams &prm, const int tid, const int e01,
                                               const int e02, const int e03, float *t1b, float *t1d,
                                               float *t2b, float *t2d, float *t3b, float *t3d,
                                               float *us) {
  constexpr int E1 = S1 + P - 1, E2 = S2 + P - 1, E3 = S3 + P - 1;
  constexpr int Q1 = S1 * P, Q2 = S2 * P, Q3 = S3 * P, PP = P + (P & 1);
  constexpr int VOL = E1 * E2 * E3;
  constexpr int A1 = (P * Q1 + NT - 1) / NT, A2 = (PP * Q2 + NT - 1) / NT;
  constexpr int A3 = DIR3 ? (PP * Q3 + NT - 1) / NT : 0, AU = (VOL + NT - 1) / NT;
  const float *gb1 = static_cast<const float *>(prm.tabB[0]), *gd1 = static_cast<const float *>(prm.tabD[0]);
  const float *gb2 = static_cast<const float *>(prm.tabB[1]), *gd2 = static_cast<const float *>(prm.tabD[1]);
  const float *gb3 = static_cast<const float *>(prm.tabB[2]), *gd3 = static_cast<const float *>(prm.tabD[2]);
  const float *u = static_cast<const float *>(prm.u);
  float b1[A1], d1[A1], b2[A2], d2[A2], b3[A3 > 0 ? A3 : 1], d3[A3 > 0 ? A3 : 1], uv[AU];
#pragma unroll
  for (int k = 0; k < A1; ++k) {
    const int i = tid + k * NT;
    b1[k] = 0.f;
    d1[k] = 0.f;
    if (i < P * Q1) {
      const int j = i / Q1, q = i - j * Q1;
      const int g = j * prm.Qpad[0] + e01 * P + q;
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
  for (int k = 0; k < A3; ++k) {
    const int i = tid + k * NT;
    const int q = i / PP, j = i - q * PP;
    b3[k] = 0.f;
    d3[k] = 0.f;
    if (i < PP * Q3 && j < P) {
      const int g = j * prm.Qpad[2] + e03 * P + q;
      b3[k] = __ldg(gb3 + g);
      if (STIFF) d3[k] = __ldg(gd3 + g);
    }
  }
  const int N1 = prm.N[0], N2 = prm.N[1], N3 = prm.N[2];
#pragma unroll
  for (int k = 0; k < AU; ++k) {
    const int i = tid + k * NT;
    const int n1 = i % E1, r = i / E1;
    const int n2 = r % E2, n3 = r / E2;
    const int g1 = e01 + n1, g2 = e02 + n2, g3 = e03 + n3;
    uv[k] = 0.f;
    if (i < VOL && g1 < N1 && g2 < N2 && g3 < N3) uv[k] = __ldg(u + ((int64_t)g3 * N2 + g2) * N1 + g1);
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
  for (int k = 0; k < A3; ++k) {
    const int i = tid + k * NT;
    if (i < PP * Q3) {
      reinterpret_cast<float2 *>(t3b)[i] = make_float2(b3[k], b3[k]);
      if (STIFF) reinterpret_cast<float2 *>(t3d)[i] = make_float2(d3[k], d3[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < AU; ++k) {
    const int i = tid + k * NT;
    if (i < VOL) us[i] = uv[k];
  }
}

// ---- mbarrier and bulk-copy helpers (shared-memory addresses as 32-bit) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity, at most `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// L2 policy for data read once: its lines are the first to be evicted, so a
// prefetched factor stream does not push out what the gather reads back.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Bulk prefetch of `bytes` contiguous bytes of global memory into L2 (the TMA
// engine; no registers, no completion to wait for), with an L2 policy.
// Address and size multiples of 16 bytes.
__device__ __forceinline__ void prefetch_l2_bulk(const void *src, uint32_t bytes, uint64_t pol) {
  asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(src), "r"(bytes),
               "l"(pol)
               : "memory");
}

// Factor slabs s0 .. s1 - 1 of one tile (slab_bytes each, contiguous from
// base) requested into L2 as evict-first lines, one slab per thread.
__device__ __forceinline__ void prefetch_factor_slabs(const void *base, uint32_t slab_bytes, int s0,
                                                      int s1, int tid, int nthreads) {
  if (s0 + tid >= s1) return;
  const uint64_t pol = l2_evict_first_policy();
  for (int s = s0 + tid; s < s1; s += nthreads)
    prefetch_l2_bulk(static_cast<const unsigned char *>(base) + (size_t)s * slab_bytes, slab_bytes, pol);
}

// Slabs a tile kernel requests into L2 at entry: about 96 KB (at most the
// tile's Q3 slabs), so that the resident blocks' requests stay within L2.
__host__ __device__ constexpr int l2_window_slabs(int slab_bytes, int q3) {
  return (98304 / slab_bytes) < 1 ? 1 : ((98304 / slab_bytes) > q3 ? q3 : (98304 / slab_bytes));
}

// Global -> shared bulk copy completing on an mbarrier (sizes and addresses
// multiples of 16 bytes).
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <int P, int S1, int S2, int S3>
struct TileF2 {
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
  static constexpr int NTC = (NPAIR + 31) / 32 * 32;  // consumer threads
  static constexpr int NT = NTC + 32;                 // + one producer warp
  static constexpr int PP = P + (P & 1);            // j padded to even for 128-bit loads
  static constexpr int XS = H1 | 1;                 // X row stride (float2), odd
  static constexpr int YS = (NPAIR + 15) / 16 * 16 + 8;  // Y plane stride (float2)
  static constexpr int T2 = 4 * PP * Q2;            // dup tables of dir 2 (B, B'), floats
  static constexpr int T3 = 4 * PP * Q3;
  static constexpr int T1 = 2 * P * Q1;             // dir-1 tables [j][q1] (B, B')
  static constexpr int VOL = E1 * E2 * E3;
  static constexpr int X = 2 * E3 * E2 * XS;        // floats per X array
  static constexpr int Y = 2 * E3 * YS;             // floats per Y array
  // factor slab bytes (bf: bfloat16 factors) and ring depth (about 48 KB of
  // slabs in flight per block)
  __host__ __device__ static constexpr uint32_t slab_bytes(bool stiff, bool bf) {
    return (stiff ? 3u * UNITS * 16u : UNITS * 8u) / (bf ? 2u : 1u);
  }
  __host__ __device__ static constexpr int ring(bool stiff, bool bf) {
    return (int)(49152u / slab_bytes(stiff, bf)) < 2 ? 2
           : ((int)(49152u / slab_bytes(stiff, bf)) > Q3 ? Q3 : (int)(49152u / slab_bytes(stiff, bf)));
  }
  __host__ __device__ static constexpr size_t ring_bytes(bool stiff, bool bf) {
    return (size_t)ring(stiff, bf) * slab_bytes(stiff, bf);
  }
  __host__ __device__ static constexpr size_t smem_bytes(bool stiff, bool bf) {
    return ring_bytes(stiff, bf) + 16 * (size_t)ring(stiff, bf) +
           4 * ((size_t)T2 + T3 + T1 + (stiff ? 2 : 1) * X + (stiff ? 3 : 1) * Y + VOL);
  }
};

template <int P, int S1, int S2, int S3, bool STIFF, bool BF, bool RL>
__device__ __forceinline__ void apply3d_f32_body(const ApplyParams &prm, const int first_tile,
                                                 const int tile_stride, const int tile_end) {
  using G = TileF2<P, S1, S2, S3>;
  constexpr int E1 = G::E1, E2 = G::E2, E3 = G::E3;
  constexpr int Q1 = G::Q1, Q2 = G::Q2, Q3 = G::Q3;
  constexpr int H1 = G::H1, PP = G::PP, NTC = G::NTC, NPAIR = G::NPAIR, UNITS = G::UNITS;
  constexpr int XS = G::XS, YS = G::YS;
  constexpr int R = G::ring(STIFF, BF);
  constexpr uint32_t SB = G::slab_bytes(STIFF, BF);
  constexpr int NCH = STIFF ? 3 : 1;   // chunks of a pencil pair per slab
  using Chunk = typename FactorChunk<STIFF, BF>::type;
  static_assert(SB == NCH * UNITS * sizeof(Chunk), "slab size");

  extern __shared__ __align__(128) unsigned char smem_f32[];
  unsigned char *ring = smem_f32;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_f32 + G::ring_bytes(STIFF, BF));
  uint64_t *empty = full + R;
  float *sm = reinterpret_cast<float *>(empty + R);
  float *t2b = sm, *t2d = t2b + 2 * PP * Q2;        // [q2][PP] float2 {b, b}
  float *t3b = t2d + 2 * PP * Q2, *t3d = t3b + 2 * PP * Q3;
  float *t1b = t3d + 2 * PP * Q3, *t1d = t1b + P * Q1; // [j][q1]
  float2 *X0 = reinterpret_cast<float2 *>(t1d + P * Q1);
  float2 *X1 = X0 + G::X / 2;
  float2 *Y0 = STIFF ? X1 + G::X / 2 : X0 + G::X / 2;
  float2 *Y1 = Y0 + G::Y / 2, *Y2 = Y1 + G::Y / 2;
  float *us = reinterpret_cast<float *>(STIFF ? Y2 + G::Y / 2 : Y0 + G::Y / 2);

  const int tid = threadIdx.x;

  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(smem_addr(&full[r]), 1);
      mbar_init(smem_addr(&empty[r]), NTC / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // ---- producer warp: one lane streams the factor slabs of all of this block's
  // tiles into the ring, in the order the consumers use them (slab counter g)
  if (tid >= NTC) {
    if (tid == NTC) {
      bool bad = false;
      bool stopped = false;   // the test hook withheld a fill: issue no further copies
      uint32_t g = 0, issued = 0;
      for (int tile = first_tile; tile < tile_end && !stopped; tile += tile_stride) {
        const int t3 = tile / (prm.T[0] * prm.T[1]);
        const int nslab = min(S3, prm.K[2] - t3 * S3) * P;
        const unsigned char *src = static_cast<const unsigned char *>(prm.D) + (size_t)tile * Q3 * SB;
        for (int s = 0; s < nslab; ++s, ++g) {
          const uint32_t slot = g % R;
          if (g >= (uint32_t)R &&
              !mbar_wait_bounded(smem_addr(&empty[slot]), ((g / R) - 1) & 1, prm.wait_limit))
            bad = true;
          if (tile == 0 && s == prm.skip_slab) {   // test hook: a fill that never comes
            stopped = true;
            break;
          }
          mbar_arrive_expect_tx(smem_addr(&full[slot]), SB);
          bulk_copy_g2s(smem_addr(ring + (size_t)slot * SB), src + (size_t)s * SB, SB,
                        smem_addr(&full[slot]));
          issued = g + 1;
        }
      }
      // leave no copy in flight: wait for the last fill of every slot used.
      // Every fill issued completes the phase it was issued for (fills stop at
      // the first withheld one), so these waits see the copies land.
      const uint32_t used = issued < (uint32_t)R ? issued : (uint32_t)R;
      for (uint32_t k = 0; k < used; ++k) {
        const uint32_t gi = issued - 1 - k;
        if (!mbar_wait_bounded(smem_addr(&full[gi % R]), (gi / R) & 1, prm.wait_limit)) bad = true;
      }
      if (bad) atomicOr(prm.status, 1u);
    }
    return;
  }

  uint32_t gbase = 0;   // slabs of earlier tiles of this block
  for (int tile = first_tile; tile < tile_end; tile += tile_stride) {
    const int t1 = tile % prm.T[0];
    const int t2 = (tile / prm.T[0]) % prm.T[1];
    const int t3 = tile / (prm.T[0] * prm.T[1]);
    const int e01 = t1 * S1, e02 = t2 * S2, e03 = t3 * S3;
    const int ke3 = min(S3, prm.K[2] - e03);
    const int nslab = ke3 * P;

    // ---- stage tables and the u tile
    stage_tile_f32<P, S1, S2, S3, NTC, STIFF>(prm, tid, e01, e02, e03, t1b, t1d, t2b, t2d, t3b, t3d, us);
    consumer_sync(NTC);

    // ---- A: direction 1, X0 = B1 u, X1 = B1' u, one pencil pair per item
    for (int i = tid; i < E3 * E2 * H1; i += NTC) {
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
      X0[r * XS + k] = a0;
      if (STIFF) X1[r * XS + k] = a1;
    }
    consumer_sync(NTC);

    // ---- B: direction 2, one (n3, element e2, pair) per item: p inputs -> p outputs
    for (int i = tid; i < E3 * S2 * H1; i += NTC) {
      const int k = i % H1, t = i / H1;
      const int e2 = t % S2, n3 = t / S2;
      float2 xa[P], xb[P];
  #pragma unroll
      for (int j = 0; j < P; ++j) {
        xa[j] = X0[(n3 * E2 + e2 + j) * XS + k];
        if (STIFF) xb[j] = X1[(n3 * E2 + e2 + j) * XS + k];
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
        const int idx = n3 * YS + q2 * H1 + k;
        Y0[idx] = y00;
        if (STIFF) {
          Y1[idx] = y01;
          Y2[idx] = y10;
        }
      }
    }
    consumer_sync(NTC);

    // ---- C: pencil pairs: direction-3 sweep, product with D, transposed sweep
    {
      const bool has_pair = tid < NPAIR;
      const int lane = tid & 31;
      bool bad = false;
      float2 y0[E3], y1[E3], y2[E3], z0[E3], z1[E3], z2[E3];
  #pragma unroll
      for (int n = 0; n < E3; ++n) {
        const float2 zero = make_float2(0.f, 0.f);
        y0[n] = has_pair ? Y0[n * YS + tid] : zero;
        z0[n] = zero;
        if (STIFF) {
          y1[n] = has_pair ? Y1[n * YS + tid] : zero;
          y2[n] = has_pair ? Y2[n * YS + tid] : zero;
          z1[n] = zero;
          z2[n] = zero;
        }
      }
  #pragma unroll
      for (int e3 = 0; e3 < S3; ++e3) {
        if (e3 < ke3) {
  #pragma unroll
          for (int qq = 0; qq < P; ++qq) {
            const int q3 = e3 * P + qq;
            const uint32_t g = gbase + q3, slot = g % R, parity = (g / R) & 1;
            if (!mbar_wait_bounded(smem_addr(&full[slot]), parity, prm.wait_limit)) bad = true;
            float4 dc[NCH] = {};
            float2 dm = make_float2(0.f, 0.f);
            if (has_pair) {
              const Chunk *rs = reinterpret_cast<const Chunk *>(ring + (size_t)slot * SB);
              if constexpr (STIFF) {
  #pragma unroll
                for (int c = 0; c < NCH; ++c) dc[c] = widen(rs[c * UNITS + tid]);
              } else {
                dm = widen(rs[tid]);
              }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[slot]));
            if (!has_pair) continue;
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
              if constexpr (RL) {
                // read the tables again rather than keep them live (see the
                // register-prefetch kernel)
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
      }
      if (has_pair) {
  #pragma unroll
        for (int n = 0; n < E3; ++n) {
          Y0[n * YS + tid] = z0[n];
          if (STIFF) {
            Y1[n * YS + tid] = z1[n];
            Y2[n * YS + tid] = z2[n];
          }
        }
      }
      if (bad) atomicOr(prm.status, 1u);
    }
    consumer_sync(NTC);

    // ---- D: transposed direction 2, register-blocked over all q2 of the tile
    for (int i = tid; i < E3 * H1; i += NTC) {
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
        const int idx = n3 * YS + q2 * H1 + k;
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
        X0[(n3 * E2 + n) * XS + k] = ya[n];
        if (STIFF) X1[(n3 * E2 + n) * XS + k] = yb[n];
      }
    }
    consumer_sync(NTC);

    // ---- E: transposed direction 1, one (n3, n2) row per item, all q1 in registers
    float *vp = static_cast<float *>(prm.vpart) + (size_t)tile * G::VOL;
    for (int r = tid; r < E3 * E2; r += NTC) {
      float2 acc[E1];
  #pragma unroll
      for (int n = 0; n < E1; ++n) acc[n] = make_float2(0.f, 0.f);
  #pragma unroll
      for (int k = 0; k < H1; ++k) {
        const int qa = 2 * k, ea = qa / P, eb = (qa + 1) / P;
        const float2 ya = X0[r * XS + k];
        const float2 yb = STIFF ? X1[r * XS + k] : make_float2(0.f, 0.f);
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
    gbase += nslab;
    consumer_sync(NTC);   // the next tile's staging overwrites what phase E reads
  }
}

template <int P, int S1, int S2, int S3, bool STIFF, bool BF, bool RL>
__global__ void __launch_bounds__(TileF2<P, S1, S2, S3>::NT)
apply3d_f32_kernel(const ApplyParams prm) {
  pdl_allow_dependents();
  apply3d_f32_body<P, S1, S2, S3, STIFF, BF, RL>(prm, blockIdx.x, gridDim.x, prm.ntiles);
}

// Many patches in one launch: block b works on tile b - first_block[patch] of
// patch = block_patch[b], with that patch's parameters.
template <int P, int S1, int S2, int S3, bool STIFF, bool BF, bool RL>
__global__ void __launch_bounds__(TileF2<P, S1, S2, S3>::NT)
apply3d_f32_batched(const BatchParams bp) {
  const int patch = bp.block_patch[blockIdx.x];
  const int tile = blockIdx.x - bp.first_block[patch];
  apply3d_f32_body<P, S1, S2, S3, STIFF, BF, RL>(bp.params[patch], tile, 1, tile + 1);
}

// One block per tile (a persistent grid that walks tiles with a stride was
// measured slower on this workload; the body supports both).
template <int P, int S1, int S2, int S3, bool STIFF, bool BF, bool RL>
cudaError_t launch_apply3d_f32(const ApplyParams &prm, cudaStream_t s) {
  using G = TileF2<P, S1, S2, S3>;
  apply3d_f32_kernel<P, S1, S2, S3, STIFF, BF, RL><<<prm.ntiles, G::NT, G::smem_bytes(STIFF, BF), s>>>(prm);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool STIFF, bool BF, bool RL>
cudaError_t launch_apply3d_f32_batched(const BatchParams &bp, int blocks, cudaStream_t s) {
  using G = TileF2<P, S1, S2, S3>;
  apply3d_f32_batched<P, S1, S2, S3, STIFF, BF, RL><<<blocks, G::NT, G::smem_bytes(STIFF, BF), s>>>(bp);
  return cudaGetLastError();
}

template <int P, int S1, int S2, int S3, bool BF, bool RL>
cudaError_t prepare_apply3d_f32() {
  using G = TileF2<P, S1, S2, S3>;
  const int sm = (int)G::smem_bytes(false, BF), sk = (int)G::smem_bytes(true, BF);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(apply3d_f32_kernel<P, S1, S2, S3, false, BF, RL>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32_kernel<P, S1, S2, S3, true, BF, RL>, a, sk);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32_batched<P, S1, S2, S3, false, BF, RL>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(apply3d_f32_batched<P, S1, S2, S3, true, BF, RL>, a, sk);
  return e;
}

// BF = true: the same kernel reading bfloat16-stored factors. RL: phase C reads
// the direction-3 tables again for the transposed sweep.
template <int P, int S1, int S2, int S3, bool BF = false, bool RL = false>
ApplyKernel make_apply3d_f32() {
  using G = TileF2<P, S1, S2, S3>;
  static_assert(G::NT <= 1024, "tile too large for one block");
  static_assert(G::smem_bytes(true, BF) <= 227 * 1024, "tile exceeds shared memory");
  static_assert(G::slab_bytes(false, BF) % 16 == 0, "bulk copies move multiples of 16 bytes");
  ApplyKernel k;
  k.S[0] = S1;
  k.S[1] = S2;
  k.S[2] = S3;
  k.threads = G::NT;
  k.smem[IGASF_MASS] = G::smem_bytes(false, BF);
  k.smem[IGASF_STIFFNESS] = G::smem_bytes(true, BF);
  k.plane = G::PL;
  k.lanes = 2;
  k.variant = IGASF_KERNEL_RING;
  k.launch[IGASF_MASS] = &launch_apply3d_f32<P, S1, S2, S3, false, BF, RL>;
  k.launch[IGASF_STIFFNESS] = &launch_apply3d_f32<P, S1, S2, S3, true, BF, RL>;
  k.launch_batched[IGASF_MASS] = &launch_apply3d_f32_batched<P, S1, S2, S3, false, BF, RL>;
  k.launch_batched[IGASF_STIFFNESS] = &launch_apply3d_f32_batched<P, S1, S2, S3, true, BF, RL>;
  k.prepare = &prepare_apply3d_f32<P, S1, S2, S3, BF, RL>;
  return k;
}

}  // namespace igasf
