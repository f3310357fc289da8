// Setup-time device kernels: univariate tables (Sec. 6.1), geometry factors
// (Sec. 6.2, Example 1), table padding, factor export, and the gather that
// accumulates per-tile partial results (eq. loc-basis-change).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "igasf_internal.h"
#include "layout.h"

namespace igasf {

// ---------------------------------------------------------------------------
// Univariate tables. One thread per quadrature point q = e p + g of one
// direction: the g-th Gauss-Legendre node of the element's span (Newton's
// method on the Legendre polynomial of degree p), its weight, and the p
// non-zero B-splines there with their derivatives, by de Boor's triangular
// scheme (values of orders 1..p on the span, derivative from the order p-1
// values). Output layout [j][Q]: entry j is function (first active) + j. An
// empty span (a repeated knot) is an element of zero measure: its points sit
// at the knot with weight 0, and its table entries are 0.
// ---------------------------------------------------------------------------
__global__ void tables_kernel(int p, int K, const double *__restrict__ knots,
                              const int *__restrict__ span, double *nodes, double *weights,
                              double *tabB, double *tabD) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int Q = K * p;
  if (q >= Q) return;
  const int e = q / p, g = q - e * p;

  // Gauss node: roots of P_p, largest first for i = 0; we want ascending g.
  const int i = p - 1 - g;
  double z = cos(M_PI * (i + 0.75) / (p + 0.5));
  double pc = z, pm = 1.0;  // P_p(z), P_{p-1}(z)
  for (int it = 0; it < 64; ++it) {
    pm = 1.0;
    pc = z;
    for (int k = 2; k <= p; ++k) {
      const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
      pm = pc;
      pc = pn;
    }
    const double step = pc / (p * (z * pc - pm) / (z * z - 1.0));
    z -= step;
    if (fabs(step) <= 1e-16) break;
  }
  pm = 1.0;
  pc = z;
  for (int k = 2; k <= p; ++k) {
    const double pn = ((2 * k - 1) * z * pc - (k - 1) * pm) / k;
    pm = pc;
    pc = pn;
  }
  const double dpn = p * (z * pc - pm) / (z * z - 1.0);
  const double wg = 2.0 / ((1.0 - z * z) * dpn * dpn);

  const int k = span[e];
  const double lo = knots[k], hi = knots[k + 1];
  const double x = lo + 0.5 * (z + 1.0) * (hi - lo);
  nodes[q] = x;
  weights[q] = 0.5 * wg * (hi - lo);
  if (!(hi > lo)) {
    for (int s = 0; s < p; ++s) {
      tabB[s * Q + q] = 0.0;
      tabD[s * Q + q] = 0.0;
    }
    return;
  }

  double Nv[IGASF_MAX_ORDER], Nm1[IGASF_MAX_ORDER], left[IGASF_MAX_ORDER], right[IGASF_MAX_ORDER];
  Nv[0] = 1.0;
  Nm1[0] = 1.0;
  for (int r = 1; r < p; ++r) {
    left[r] = x - knots[k + 1 - r];
    right[r] = knots[k + r] - x;
    double saved = 0.0;
    for (int s = 0; s < r; ++s) {
      const double tmp = Nv[s] / (right[s + 1] + left[r - s]);
      Nv[s] = saved + right[s + 1] * tmp;
      saved = left[r - s] * tmp;
    }
    Nv[r] = saved;
    if (r == p - 2)
      for (int s = 0; s <= r; ++s) Nm1[s] = Nv[s];
  }
  for (int s = 0; s < p; ++s) {
    double der = 0.0;
    if (p > 1) {
      const int fi = k - p + 1 + s;  // global function index
      // order p-1 functions on this span are fi' = k-p+2 .. k, stored at Nm1[fi' - (k-p+2)]
      if (s >= 1) der += Nm1[s - 1] / (knots[fi + p - 1] - knots[fi]);
      if (s <= p - 2) der -= Nm1[s] / (knots[fi + p] - knots[fi + 1]);
      der *= (p - 1);
    }
    tabB[s * Q + q] = Nv[s];
    tabD[s * Q + q] = der;
  }
}

cudaError_t launch_tables(int p, int K, const double *knots, const int *span, double *nodes,
                          double *weights, double *tabB, double *tabD, cudaStream_t s) {
  const int Q = K * p;
  tables_kernel<<<(Q + 127) / 128, 128, 0, s>>>(p, K, knots, span, nodes, weights, tabB, tabD);
  return cudaGetLastError();
}

// Padded copy [j][Q] -> [j][Qpad] in the apply precision, zeros beyond Q.
template <typename T>
__global__ void pad_tables_kernel(int p, int Q, int Qpad, const double *src, T *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p * Qpad) return;
  const int j = i / Qpad, q = i - j * Qpad;
  dst[i] = q < Q ? (T)src[j * Q + q] : T(0);
}

cudaError_t launch_pad_tables(int p, int K, int Qpad, const double *src, void *dst, int to_float,
                              cudaStream_t s) {
  const int n = p * Qpad;
  if (to_float)
    pad_tables_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(p, K * p, Qpad, src, (float *)dst);
  else
    pad_tables_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(p, K * p, Qpad, src, (double *)dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Factor layout addressing (shared by the geometry writer and the exporter).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t layout_index(const FactorLayout &L, int nf, int f,
                                                const int *qg) {
  return layout_index_q(L.d, L.p, L.S, L.T, L.plane, L.lanes, L.elem_bytes, nf, f, qg);
}

// One factor, rounded once from FP64 to the stored type (to nearest even).
__device__ __forceinline__ void store_factor(const FactorLayout &L, void *base, int64_t idx, double v) {
  if (L.elem_bytes == 8) static_cast<double *>(base)[idx] = v;
  else if (L.elem_bytes == 4) static_cast<float *>(base)[idx] = __double2float_rn(v);
  else static_cast<__nv_bfloat16 *>(base)[idx] = __double2bfloat16(v);
}

__device__ void write_factors(const GeometryParams &g, const int *qg, double dm, const double *dk,
                              int nfk) {
  for (int o = 0; o < g.nout; ++o) {
    const FactorLayout &L = g.out[o];
    store_factor(L, L.DM, layout_index(L, 1, 0, qg), dm);
    for (int f = 0; f < nfk; ++f) store_factor(L, L.DK, layout_index(L, nfk, f, qg), dk[f]);
  }
}

__device__ __forceinline__ double coefficient(const GeometryParams &g, const double *x,
                                              int64_t qlin) {
  if (g.coef_kind == IGASF_COEF_EXP_SIN_COS) {
    const double c = g.d > 1 ? cos(2.0 * M_PI * x[1]) : 1.0;
    return exp(g.coef_alpha * sin(2.0 * M_PI * x[0]) * c);
  }
  if (g.coef_kind == IGASF_COEF_VALUES) return g.coef_values[qlin];
  return g.coef_const;
}

// ---------------------------------------------------------------------------
// 3D geometry factors by sum-factorized evaluation (Alg. 3 applied to each
// component of G and to its derivatives, Sec. 6.2), on blocks of Gs x Gs x 1
// elements:  C = B1 c -> B2 -> B3 with the derivative table in the one
// direction being differentiated. Then, per quadrature point,
//   J_ij = dG_i/dxi_j, adj = det(J) J^-1,
//   D_M = w |det J|,  D_K = w a(G) |det J| J^-1 J^-T = w a(G) adj adj^T / |det J|.
// ---------------------------------------------------------------------------
__global__ void geometry3d_kernel(const GeometryParams g, int Gs, int nb1, int nb2) {
  extern __shared__ double gsm[];
  const int P = g.p;
  const int Eg = Gs + P - 1, Qg = Gs * P;
  double *cs = gsm;                              // [c][n3][n2][n1]
  double *A0 = cs + 3 * P * Eg * Eg;             // [c][n3][n2][q1]
  double *A1 = A0 + 3 * P * Eg * Qg;
  double *C00 = A1 + 3 * P * Eg * Qg;            // [c][n3][q2][q1]
  double *C01 = C00 + 3 * P * Qg * Qg;
  double *C10 = C01 + 3 * P * Qg * Qg;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int b = blockIdx.x;
  const int b1 = b % nb1, b2 = (b / nb1) % nb2, e3 = b / (nb1 * nb2);
  const int e01 = b1 * Gs, e02 = b2 * Gs;
  const int N1 = g.N[0], N2 = g.N[1];
  const int Qt1 = g.K[0] * P, Qt2 = g.K[1] * P, Qt3 = g.K[2] * P;

  for (int i = tid; i < 3 * P * Eg * Eg; i += nt) {
    const int n1 = i % Eg, n2 = (i / Eg) % Eg, n3 = (i / (Eg * Eg)) % P, c = i / (Eg * Eg * P);
    const int g1 = e01 + n1, g2 = e02 + n2, g3 = e3 + n3;
    cs[i] = (g1 < N1 && g2 < N2) ? g.ctrl[(((int64_t)g3 * N2 + g2) * N1 + g1) * 3 + c] : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < 3 * P * Eg * Qg; i += nt) {
    const int q1 = i % Qg, r = i / Qg;
    const int e1 = q1 / P, q1g = e01 * P + q1;
    double a0 = 0.0, a1 = 0.0;
    if (q1g < Qt1) {
      for (int j = 0; j < P; ++j) {
        const double c = cs[r * Eg + e1 + j];
        a0 += g.tabB[0][j * Qt1 + q1g] * c;
        a1 += g.tabD[0][j * Qt1 + q1g] * c;
      }
    }
    A0[i] = a0;
    A1[i] = a1;
  }
  __syncthreads();
  for (int i = tid; i < 3 * P * Qg * Qg; i += nt) {
    const int q1 = i % Qg, q2 = (i / Qg) % Qg, r = i / (Qg * Qg);
    const int e2 = q2 / P, q2g = e02 * P + q2;
    double c00 = 0.0, c01 = 0.0, c10 = 0.0;
    if (q2g < Qt2) {
      for (int j = 0; j < P; ++j) {
        const int ia = (r * Eg + e2 + j) * Qg + q1;
        const double bb = g.tabB[1][j * Qt2 + q2g], db = g.tabD[1][j * Qt2 + q2g];
        c00 += bb * A0[ia];
        c01 += db * A0[ia];
        c10 += bb * A1[ia];
      }
    }
    C00[i] = c00;
    C01[i] = c01;
    C10[i] = c10;
  }
  __syncthreads();
  for (int pen = tid; pen < Qg * Qg; pen += nt) {
    const int q1 = pen % Qg, q2 = pen / Qg;
    const int q1g = e01 * P + q1, q2g = e02 * P + q2;
    if (q1g >= Qt1 || q2g >= Qt2) continue;
    for (int qq = 0; qq < P; ++qq) {
      const int q3g = e3 * P + qq;
      double J[3][3], X[3];
      for (int c = 0; c < 3; ++c) {
        double gv = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
        for (int j = 0; j < P; ++j) {
          const int ic = ((c * P + j) * Qg + q2) * Qg + q1;
          const double bb = g.tabB[2][j * Qt3 + q3g], db = g.tabD[2][j * Qt3 + q3g];
          gv += bb * C00[ic];
          d3 += db * C00[ic];
          d2 += bb * C01[ic];
          d1 += bb * C10[ic];
        }
        X[c] = gv;
        J[c][0] = d1;
        J[c][1] = d2;
        J[c][2] = d3;
      }
      double adj[3][3];
      adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
      const double w = g.wq[0][q1g] * g.wq[1][q2g] * g.wq[2][q3g];
      if (w > 0.0 && !(det > 0.0)) atomicOr(g.bad_det, 1u);   // w = 0: an empty span
      const double adet = fabs(det);
      const int64_t qlin = ((int64_t)q3g * Qt2 + q2g) * Qt1 + q1g;
      const double a = coefficient(g, X, qlin);
      const double s = adet > 0.0 ? w * a / adet : 0.0;
      double dk[6];
      const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
      for (int f = 0; f < 6; ++f) {
        const int r = ii[f], c = jj[f];
        dk[f] = s * (adj[r][0] * adj[c][0] + adj[r][1] * adj[c][1] + adj[r][2] * adj[c][2]);
      }
      const int qg[3] = {q1g, q2g, q3g};
      write_factors(g, qg, w * adet, dk, 6);
      if (g.xq_out)
        for (int c = 0; c < 3; ++c) g.xq_out[qlin * 3 + c] = X[c];
    }
  }
}

// 2D geometry factors: one thread per quadrature point, G and J by the direct
// sum over the p^2 active functions (cheap in two dimensions).
__global__ void geometry2d_kernel(const GeometryParams g) {
  const int P = g.p;
  const int Qt1 = g.K[0] * P, Qt2 = g.K[1] * P;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)Qt1 * Qt2) return;
  const int q1g = (int)(q % Qt1), q2g = (int)(q / Qt1);
  const int f1 = q1g / P, f2 = q2g / P;  // first active function = element (span index - p + 1)
  double X[2] = {0.0, 0.0}, J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int j2 = 0; j2 < P; ++j2) {
    const double b2 = g.tabB[1][j2 * Qt2 + q2g], d2 = g.tabD[1][j2 * Qt2 + q2g];
    for (int j1 = 0; j1 < P; ++j1) {
      const double b1 = g.tabB[0][j1 * Qt1 + q1g], d1 = g.tabD[0][j1 * Qt1 + q1g];
      const int64_t n = (int64_t)(f2 + j2) * g.N[0] + (f1 + j1);
      for (int c = 0; c < 2; ++c) {
        const double cc = g.ctrl[n * 2 + c];
        X[c] += b1 * b2 * cc;
        J[c][0] += d1 * b2 * cc;
        J[c][1] += b1 * d2 * cc;
      }
    }
  }
  const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double w = g.wq[0][q1g] * g.wq[1][q2g];
  if (w > 0.0 && !(det > 0.0)) atomicOr(g.bad_det, 1u);   // w = 0: an empty span
  const double adet = fabs(det);
  // adj = det J^-1 = [[J11, -J01], [-J10, J00]]
  const double adj[2][2] = {{J[1][1], -J[0][1]}, {-J[1][0], J[0][0]}};
  const double a = coefficient(g, X, q);
  const double s = adet > 0.0 ? w * a / adet : 0.0;
  double dk[3];
  dk[0] = s * (adj[0][0] * adj[0][0] + adj[0][1] * adj[0][1]);
  dk[1] = s * (adj[0][0] * adj[1][0] + adj[0][1] * adj[1][1]);
  dk[2] = s * (adj[1][0] * adj[1][0] + adj[1][1] * adj[1][1]);
  const int qg[2] = {q1g, q2g};
  write_factors(g, qg, w * adet, dk, 3);
  if (g.xq_out) {
    g.xq_out[q * 2] = X[0];
    g.xq_out[q * 2 + 1] = X[1];
  }
}

int geometry_block_elems(int p) {
  // elements per block in directions 1 and 2 for the 3D geometry kernel
  if (p <= 2) return 8;
  if (p <= 4) return 4;
  if (p <= 7) return 2;
  return 1;
}

size_t geometry3d_smem(int p, int Gs) {
  const size_t Eg = Gs + p - 1, Qg = (size_t)Gs * p;
  return sizeof(double) * (3 * p * Eg * Eg + 6 * p * Eg * Qg + 9 * p * Qg * Qg);
}

cudaError_t launch_geometry(const GeometryParams &g, cudaStream_t s) {
  if (g.d == 3) {
    const int Gs = geometry_block_elems(g.p);
    const int nb1 = (g.K[0] + Gs - 1) / Gs, nb2 = (g.K[1] + Gs - 1) / Gs;
    const size_t smem = geometry3d_smem(g.p, Gs);
    cudaError_t e = cudaFuncSetAttribute(geometry3d_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int threads = Gs * g.p * Gs * g.p;
    threads = ((threads + 31) / 32) * 32;
    if (threads > 512) threads = 512;
    const int64_t blocks = (int64_t)nb1 * nb2 * g.K[2];
    geometry3d_kernel<<<(unsigned)blocks, threads, smem, s>>>(g, Gs, nb1, nb2);
  } else {
    const int64_t Q = (int64_t)g.K[0] * g.p * g.K[1] * g.p;
    geometry2d_kernel<<<(unsigned)((Q + 127) / 128), 128, 0, s>>>(g);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Export of stored factors to FP64 in lexicographic quadrature order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename T>
__global__ void export_kernel(const FactorLayout L, int nf, const void *src, int64_t Qtot,
                              int Q0, int Q1, int Q2, double *out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Qtot) return;
  int qg[3];
  qg[0] = (int)(q % Q0);
  qg[1] = (int)((q / Q0) % Q1);
  qg[2] = (int)(q / ((int64_t)Q0 * Q1));
  (void)Q2;
  for (int f = 0; f < nf; ++f) out[q * nf + f] = to_double(static_cast<const T *>(src)[layout_index(L, nf, f, qg)]);
}

cudaError_t launch_export_factors(const FactorLayout &L, int op, int64_t Qtot, const int *Q,
                                  double *out, cudaStream_t s) {
  const int nf = num_fields(L.d, op);
  const void *src = op == IGASF_MASS ? L.DM : L.DK;
  const unsigned blocks = (unsigned)((Qtot + 255) / 256);
  const int Q2 = L.d > 2 ? Q[2] : 1, Q1 = L.d > 1 ? Q[1] : 1;
  if (L.elem_bytes == 4) export_kernel<float><<<blocks, 256, 0, s>>>(L, nf, src, Qtot, Q[0], Q1, Q2, out);
  else if (L.elem_bytes == 2)
    export_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(L, nf, src, Qtot, Q[0], Q1, Q2, out);
  else export_kernel<double><<<blocks, 256, 0, s>>>(L, nf, src, Qtot, Q[0], Q1, Q2, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gather: v_n = sum over the tiles D containing dof n of (v_D)_{local(n)}
// (the accumulation S_D^T v_D of eq. loc-basis-change), in a fixed tile order
// so that the result is bitwise reproducible.
// ---------------------------------------------------------------------------
// The tiles containing dof index i of one direction are t*S <= i <= t*S + E - 1,
// 0 <= t < T; per direction a table gives, for every i, the first such tile
// (.x) and (number of tiles << 16) | (i's local index in the first tile) (.y),
// built on the host at setup (gather_table), so the kernel does no per-tile
// division. The tables are constant, so they are read before the wait for the
// tile kernel's results.
//
// TWO (at most two tiles per direction contain a dof): a thread owns one
// (i0, i1) of the flattened first two directions (one division by N0), so no
// thread idles on short rows; its <= 8 loads are predicated, not looped.
// Otherwise a block covers 128 consecutive i0 of one row (i1, i2 from the
// grid), so the threads of a warp share the per-row tile counts of their loops.
template <typename T, bool TWO>
__global__ void gather_kernel(const T *__restrict__ vpart, T *__restrict__ v, const int2 *__restrict__ g0,
                              const int2 *__restrict__ g1, const int2 *__restrict__ g2, int N0, int N1,
                              int N2, int T0, int T1, int S0, int S1, int S2, int E0, int E1, int vol) {
  const int N01 = N0 * N1;
  int i0, i1;
  bool active;
  if (TWO) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    active = n < N01;
    i1 = active ? n / N0 : 0;
    i0 = n - i1 * N0;
  } else {
    i0 = blockIdx.x * blockDim.x + threadIdx.x;
    i1 = blockIdx.y;
    active = i0 < N0;
  }
  const int z0 = TWO ? blockIdx.y : blockIdx.z, zstep = TWO ? gridDim.y : gridDim.z;
  int2 a0 = make_int2(0, 0), a1 = make_int2(0, 0), a2z = make_int2(0, 0);
  if (active) {
    a0 = g0[i0];
    if (i1 < N1) a1 = g1[i1];
    if (z0 < N2) a2z = g2[z0];
  }
  pdl_wait_primary();
  if (!active) return;
  const int c0 = a0.y >> 16, l0 = a0.y & 0xffff;
  for (; i1 < N1; i1 += TWO ? N1 : gridDim.y) {
    if (!TWO && i1 != (int)blockIdx.y) a1 = g1[i1];
    const int c1 = a1.y >> 16, l1 = a1.y & 0xffff;
    for (int i2 = z0; i2 < N2; i2 += zstep) {
      const int2 a2 = i2 == z0 ? a2z : g2[i2];
      const int c2 = a2.y >> 16, l2 = a2.y & 0xffff;
      T acc = T(0);
      if (TWO) {
        // all loads first, then the sums in tile order (t2, t1, t0 ascending)
        T x[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int k2 = c >> 2, k1 = (c >> 1) & 1, k0 = c & 1;
          x[c] = T(0);
          if (k2 < c2 && k1 < c1 && k0 < c0) {
            const int64_t tile = ((int64_t)(a2.x + k2) * T1 + (a1.x + k1)) * T0 + (a0.x + k0);
            const int loc = ((l2 - k2 * S2) * E1 + (l1 - k1 * S1)) * E0 + (l0 - k0 * S0);
            x[c] = vpart[tile * vol + loc];
          }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc += x[c];
      } else {
        for (int k2 = 0; k2 < c2; ++k2)
          for (int k1 = 0; k1 < c1; ++k1)
            for (int k0 = 0; k0 < c0; ++k0) {
              const int64_t tile = ((int64_t)(a2.x + k2) * T1 + (a1.x + k1)) * T0 + (a0.x + k0);
              const int loc = ((l2 - k2 * S2) * E1 + (l1 - k1 * S1)) * E0 + (l0 - k0 * S0);
              acc += vpart[tile * vol + loc];
            }
      }
      v[(int64_t)i2 * N01 + (int64_t)i1 * N0 + i0] = acc;
    }
  }
}

void gather_table(int N, int S, int E, int T, std::vector<int2> &out) {
  out.resize(N > 0 ? N : 1);
  if (N <= 0) {
    out[0] = make_int2(0, 1 << 16);
    return;
  }
  for (int i = 0; i < N; ++i) {
    const int lo = i - E + 1 > 0 ? (i - E + S) / S : 0;
    const int hi = std::min(T - 1, i / S);
    out[i] = make_int2(lo, ((hi - lo + 1) << 16) | (i - lo * S));
  }
}

cudaError_t launch_gather(int d, int float_vectors, const void *vpart, void *v, const int *N,
                          const int *T, const int *S, int p, int2 *const *gtab, cudaStream_t s) {
  const int N1 = d > 1 ? N[1] : 1, N2 = d > 2 ? N[2] : 1;
  const int T1 = d > 1 ? T[1] : 1;
  const int S1 = d > 1 ? S[1] : 1, S2 = d > 2 ? S[2] : 1;
  const int E0 = S[0] + p - 1, E1 = d > 1 ? S1 + p - 1 : 1, E2 = d > 2 ? S2 + p - 1 : 1;
  const int vol = E0 * E1 * E2;
  const bool two = E0 <= 2 * S[0] && E1 <= 2 * S1 && E2 <= 2 * S2;
  // launched with a programmatic dependency on the tile kernel before it
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if (two)
    cfg.gridDim = dim3((N[0] * N1 - 1) / 128 + 1, std::min(N2, 65535), 1);
  else
    cfg.gridDim = dim3((N[0] + 127) / 128, std::min(N1, 65535), std::min(N2, 65535));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define IGASF_GATHER(TT, TWO_)                                                                      \
  cudaLaunchKernelEx(&cfg, gather_kernel<TT, TWO_>, (const TT *)vpart, (TT *)v, (const int2 *)gtab[0], \
                     (const int2 *)gtab[1], (const int2 *)gtab[2], N[0], N1, N2, T[0], T1, S[0], S1, S2, \
                     E0, E1, vol)
  cudaError_t e;
  if (float_vectors)
    e = two ? IGASF_GATHER(float, true) : IGASF_GATHER(float, false);
  else
    e = two ? IGASF_GATHER(double, true) : IGASF_GATHER(double, false);
#undef IGASF_GATHER
  return e;
}

}  // namespace igasf
