// igasf_assemble_csr: FP64 CSR assembly of the quadrature operator on the
// device by sum factorization over the whole patch (Sec. 3.1, Alg. 1, with
// eq. recursive-step1 applied to one direction after the other).
//
// Notation: direction a has N_a functions, K_a elements (knot spans, empty
// ones of repeated knots included) and Q_a = K_a p Gauss points; function m of
// a direction is non-zero on the elements m - p + 1..m, so a pair (m, n) of
// one direction can interact only for |m - n| <= p - 1. Columns of a row are
// addressed by offsets o = n - m + p - 1 in [0, W), W = 2p - 1, per direction.
// The pattern holds the pairs that share a non-empty element in every
// direction (Sec. 3, Cor. 3 and its nnz count); per direction and row m these
// are the n of an interval [lo_a(m), lo_a(m) + cnt_a(m) - 1], since the shared
// elements of (m, n) shrink as |m - n| grows. Empty elements have zero
// tables, so pairs outside the pattern would only have received zeros. Term t of the bilinear form pairs the test function
// psi_m, differentiated (or not) per direction, with the trial function phi_n
// and one stored factor F_t = w F_ij (weights folded in). Mass: one term, no
// derivatives, F = w |det J|. Stiffness: the d^2 terms (i, j), derivative of
// psi_m along i, of phi_n along j, factor w F_ij.
//
// Level 1, direction 1, for every later quadrature point (x_2[, x_3]):
//   L1_t(x_2, x_3; m1, o1) = sum_{x_1} psi^t_{m1}(x_1) phi^t_{n1}(x_1) F_t(x_1, x_2, x_3)
// Level 2 (d = 3), direction 2, for every x_3:
//   L2_g(x_3; m2, o2, m1, o1) = sum_{t in g} sum_{x_2} psi^t_{m2} phi^t_{n2} L1_t(x_2, x_3; m1, o1)
// Last level, direction d:
//   A(m, n) = sum_g sum_{x_d} psi^g_{md} phi^g_{nd} L_{d-1, g}(x_d; ...)
// Terms are grouped (g) by the tables they use in the last direction, as soon
// as every earlier direction has been summed: 4 groups for the stiffness, 1
// for the mass. Every sum over one direction's quadrature points runs only
// over the elements shared by the two functions.
//
// The last direction is processed in chunks of element layers, so that the
// intermediate levels of one chunk stay within a workspace limit; each chunk
// adds its part to the CSR values (rows next to a chunk boundary receive the
// parts of both chunks, in chunk order), so the result is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "igasf.h"
#include "igasf_internal.h"
#include "layout.h"
#include "plan.h"

namespace igasf {

int set_error(int code, const char *msg);

namespace {

struct AsmDims {
  int d, p, W;
  int N[3], K[3], Q[3];       // unused directions: 1
  const double *tabB[3], *tabD[3];  // FP64 [j][Q_a]
  int stiff;                  // 0: mass, 1: stiffness
  int nterms, ngroups, nf;
  // products of the two univariate tables over the shared elements of every pair:
  // PT[a][choice][m][o][i][k] = tm(m - e, q) tn(n - e, q), e = first shared
  // element + i, q = e p + k; choice = 2 (psi differentiated) + (phi differentiated)
  const double *PT[3];
};

// term t of the stiffness form: (i, j) = (t / d, t % d)
__device__ __forceinline__ int term_i(const AsmDims &g, int t) { return g.stiff ? t / g.d : -1; }
__device__ __forceinline__ int term_j(const AsmDims &g, int t) { return g.stiff ? t % g.d : -1; }

// stored field of F_ij: 3D (11 12 13 22 23 33), 2D (11 12 22)
__device__ __forceinline__ int term_field(const AsmDims &g, int t) {
  if (!g.stiff) return 0;
  int i = term_i(g, t), j = term_j(g, t);
  if (i > j) {
    const int s = i;
    i = j;
    j = s;
  }
  if (g.d == 3) return i == 0 ? j : (i == 1 ? 2 + j : 5);
  return i + j;
}

// group of a term: which tables it uses in the last direction (bit 1: psi
// differentiated, bit 0: phi differentiated)
__device__ __forceinline__ int term_group(const AsmDims &g, int t) {
  if (!g.stiff) return 0;
  return 2 * (term_i(g, t) == g.d - 1) + (term_j(g, t) == g.d - 1);
}

// elements shared by functions m and n of direction a, clipped to [elo, ehi]
__device__ __forceinline__ void common_elements(const AsmDims &g, int a, int m, int n, int elo,
                                                int ehi, int &lo, int &hi) {
  lo = max(max(m, n) - (g.p - 1), max(elo, 0));
  hi = min(min(m, n), min(ehi, g.K[a] - 1));
}

// sum over the shared quadrature points of direction a, elements lo..hi (a
// sub-range of the pair's shared elements), of psi_m phi_n x(q), with the
// products psi_m phi_n read from the pair-product table (one FMA per point);
// x read at x + (q - q0) * x_stride
__device__ __forceinline__ double contract(const AsmDims &g, int a, bool dm, bool dn, int m, int o,
                                           int lo, int hi, const double *x, int64_t x_stride,
                                           int q0) {
  const int p = g.p, n = m + o - (p - 1);
  const int first = max(max(m, n) - (p - 1), 0);
  const int choice = 2 * dm + dn;
  const double *pt = g.PT[a] + ((((int64_t)choice * g.N[a] + m) * g.W + o) * p) * p;
  double s = 0.0;
  for (int e = lo; e <= hi; ++e) {
    const double *pe = pt + (e - first) * p;
    const double *xe = x + (int64_t)(e * p - q0) * x_stride;
    for (int k = 0; k < p; ++k) s = fma(pe[k], xe[k * x_stride], s);
  }
  return s;
}

// pair-product tables of one direction: one thread per (choice, m, o, i, k)
__global__ void pair_table_kernel(const AsmDims g, int a, double *PT) {
  const int p = g.p, W = g.W, N = g.N[a];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)4 * N * W * p * p) return;
  const int k = (int)(idx % p);
  int64_t r = idx / p;
  const int i = (int)(r % p);
  r /= p;
  const int o = (int)(r % W);
  r /= W;
  const int m = (int)(r % N);
  const int choice = (int)(r / N);
  const int n = m + o - (p - 1);
  double v = 0.0;
  if (n >= 0 && n < N) {
    const int first = max(max(m, n) - (p - 1), 0);
    const int last = min(min(m, n), g.K[a] - 1);
    const int e = first + i;
    if (e <= last) {
      const int Q = g.Q[a], q = e * p + k;
      const double *tm = (choice & 2) ? g.tabD[a] : g.tabB[a];
      const double *tn = (choice & 1) ? g.tabD[a] : g.tabB[a];
      v = tm[(int64_t)(m - e) * Q + q] * tn[(int64_t)(n - e) * Q + q];
    }
  }
  PT[idx] = v;
}

// ---- chunk factors, lexicographic: Fc[f][qc][qmid][q1] ------------------------
__global__ void chunk_factors_kernel(const AsmDims g, FactorLayout L, const double *D, int qL0,
                                     int QC, int Qmid, double *Fc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)Qmid * g.Q[0];
  if (idx >= QC * plane) return;
  const int q1 = (int)(idx % g.Q[0]);
  const int qmid = (int)((idx / g.Q[0]) % Qmid);
  const int qc = (int)(idx / plane);
  int qg[3] = {q1, 0, 0};
  if (g.d == 3) {
    qg[1] = qmid;
    qg[2] = qL0 + qc;
  } else {
    qg[1] = qL0 + qc;
  }
  for (int f = 0; f < g.nf; ++f)
    Fc[(int64_t)f * QC * plane + idx] = D[layout_index_q(L.d, L.p, L.S, L.T, L.plane, L.lanes, 8, g.nf, f, qg)];
}

// ---- level 1: L1[t][qc][qmid][m1][o1] ------------------------------------------
__global__ void level1_kernel(const AsmDims g, const double *Fc, int QC, int Qmid, double *L1) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int W = g.W, N1 = g.N[0];
  const int64_t per_t = (int64_t)QC * Qmid * N1 * W;
  if (idx >= g.nterms * per_t) return;
  const int o1 = (int)(idx % W);
  int64_t r = idx / W;
  const int m1 = (int)(r % N1);
  r /= N1;
  const int qmid = (int)(r % Qmid);
  r /= Qmid;
  const int qc = (int)(r % QC);
  const int t = (int)(r / QC);
  const int n1 = m1 + o1 - (g.p - 1);
  double s = 0.0;
  if (n1 >= 0 && n1 < N1) {
    int lo, hi;
    common_elements(g, 0, m1, n1, 0, g.K[0] - 1, lo, hi);
    const double *x = Fc + (((int64_t)term_field(g, t) * QC + qc) * Qmid + qmid) * g.Q[0];
    s = contract(g, 0, term_i(g, t) == 0, term_j(g, t) == 0, m1, o1, lo, hi, x, 1, 0);
  }
  L1[idx] = s;
}

// ---- level 2 (d = 3): L2[g][qc][m2][o2][m1][o1] --------------------------------
__global__ void level2_kernel(const AsmDims g, const double *L1, int QC, double *L2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int W = g.W, N1 = g.N[0], N2 = g.N[1], Q2 = g.Q[1];
  const int64_t inner1 = (int64_t)N1 * W;                 // (m1, o1)
  const int64_t inner = (int64_t)N2 * W * inner1;         // (m2, o2, m1, o1)
  if (idx >= QC * inner) return;
  const int64_t e1 = idx % inner1;
  int64_t r = idx / inner1;
  const int o2 = (int)(r % W);
  r /= W;
  const int m2 = (int)(r % N2);
  const int qc = (int)(r / N2);
  const int n2 = m2 + o2 - (g.p - 1);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (n2 >= 0 && n2 < N2) {
    int lo, hi;
    common_elements(g, 1, m2, n2, 0, g.K[1] - 1, lo, hi);
    for (int t = 0; t < g.nterms; ++t) {
      const double *x = L1 + ((int64_t)t * QC + qc) * Q2 * inner1 + e1;
      acc[term_group(g, t)] +=
          contract(g, 1, term_i(g, t) == 1, term_j(g, t) == 1, m2, o2, lo, hi, x, inner1, 0);
    }
  }
  const int64_t off = (int64_t)qc * inner + ((int64_t)m2 * W + o2) * inner1 + e1;
  for (int gg = 0; gg < g.ngroups; ++gg) L2[(int64_t)gg * QC * inner + off] = acc[gg];
}

// ---- CSR addressing -------------------------------------------------------------
struct CsrDims {
  const int64_t *pre[3];   // prefix sums of the per-direction column counts, N_a + 1 each
  const int *lo[3];        // first column of each row, per direction
};

__device__ __forceinline__ int count_1d(const CsrDims &c, int a, int m) {
  return (int)(c.pre[a][m + 1] - c.pre[a][m]);
}

// is column n of direction a in the pattern of row m
__device__ __forceinline__ bool in_pattern_1d(const CsrDims &c, int a, int m, int n) {
  const int lo = c.lo[a][m];
  return n >= lo && n < lo + count_1d(c, a, m);
}

__device__ __forceinline__ int64_t row_start(const AsmDims &g, const CsrDims &c, const int *m) {
  const int64_t T1 = c.pre[0][g.N[0]];
  if (g.d == 2) return c.pre[1][m[1]] * T1 + (int64_t)count_1d(c, 1, m[1]) * c.pre[0][m[0]];
  const int64_t T2 = c.pre[1][g.N[1]];
  return c.pre[2][m[2]] * T2 * T1 +
         (int64_t)count_1d(c, 2, m[2]) *
             (c.pre[1][m[1]] * T1 + (int64_t)count_1d(c, 1, m[1]) * c.pre[0][m[0]]);
}

// position of column offset o within row m (columns ascending = last direction slowest)
__device__ __forceinline__ int64_t rank_in_row(const AsmDims &g, const CsrDims &c, const int *m,
                                               const int *o) {
  int64_t r = 0;
  for (int a = g.d - 1; a >= 0; --a) {
    const int olo = c.lo[a][m[a]] - m[a] + g.p - 1;
    r = r * count_1d(c, a, m[a]) + (o[a] - olo);
  }
  return r;
}

__global__ void csr_structure_kernel(const AsmDims g, const CsrDims c, int64_t *rowptr,
                                     int64_t *colind) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t Wd = 1, Ntot = 1;
  for (int a = 0; a < g.d; ++a) {
    Wd *= g.W;
    Ntot *= g.N[a];
  }
  if (idx >= Ntot * Wd) return;
  int o[3] = {0, 0, 0}, m[3] = {0, 0, 0};
  int64_t r = idx;
  for (int a = 0; a < g.d; ++a) {
    o[a] = (int)(r % g.W);
    r /= g.W;
  }
  for (int a = 0; a < g.d; ++a) {
    m[a] = (int)(r % g.N[a]);
    r /= g.N[a];
  }
  int64_t col = 0, stride = 1;
  for (int a = 0; a < g.d; ++a) {
    const int n = m[a] + o[a] - (g.p - 1);
    if (!in_pattern_1d(c, a, m[a], n)) return;
    col += n * stride;
    stride *= g.N[a];
  }
  const int64_t start = row_start(g, c, m);
  colind[start + rank_in_row(g, c, m, o)] = col;
  bool first = true;
  for (int a = 0; a < g.d; ++a) first = first && m[a] + o[a] - (g.p - 1) == c.lo[a][m[a]];
  if (first) {
    rowptr[idx / Wd] = start;
    if (idx / Wd == Ntot - 1) {
      int64_t cnt = 1;
      for (int a = 0; a < g.d; ++a) cnt *= count_1d(c, a, m[a]);
      rowptr[Ntot] = start + cnt;
    }
  }
}

// ---- last level: values += contribution of the chunk's elements ----------------
// Lprev[g][qc][inner], inner = (m2, o2, m1, o1) for d = 3 or (m1, o1) for d = 2.
__global__ void last_level_kernel(const AsmDims g, const CsrDims c, const double *Lprev, int QC,
                                  int e0, int e1, int mL0, int nrows, double *values) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int W = g.W, a = g.d - 1, p = g.p;
  int64_t inner = 1;
  for (int b = 0; b < a; ++b) inner *= (int64_t)g.N[b] * W;
  if (idx >= (int64_t)nrows * W * inner) return;
  const int64_t e_in = idx % inner;
  const int64_t r = idx / inner;
  int m[3], o[3];
  o[a] = (int)(r % W);
  m[a] = mL0 + (int)(r / W);
  int64_t t = e_in;
  for (int b = 0; b < a; ++b) {
    o[b] = (int)(t % W);
    t /= W;
    m[b] = (int)(t % g.N[b]);
    t /= g.N[b];
  }
  for (int b = 0; b < g.d; ++b)
    if (!in_pattern_1d(c, b, m[b], m[b] + o[b] - (p - 1))) return;
  const int nL = m[a] + o[a] - (p - 1);
  int lo, hi;
  common_elements(g, a, m[a], nL, e0, e1 - 1, lo, hi);
  if (lo > hi) return;
  double s = 0.0;
  for (int gg = 0; gg < g.ngroups; ++gg) {
    const double *x = Lprev + (int64_t)gg * QC * inner + e_in;
    s += contract(g, a, (gg & 2) != 0 && g.stiff, (gg & 1) != 0 && g.stiff, m[a], o[a], lo, hi, x,
                  inner, e0 * p);
  }
  values[row_start(g, c, m) + rank_in_row(g, c, m, o)] += s;
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Columns of every row of direction a: lo[m] and the count; returns their sum.
// Column n belongs to row m when an element e in [max(m, n) - p + 1, min(m, n)]
// is non-empty.
int64_t pattern_1d(const igasf_plan *h, int a, std::vector<int> &lo, std::vector<int> &cnt) {
  const int p = h->p, N = h->N[a], K = h->K[a];
  const std::vector<unsigned char> &ne = h->nonempty[a];
  auto shares = [&](int m, int n) {
    for (int e = std::max(std::max(m, n) - p + 1, 0); e <= std::min(std::min(m, n), K - 1); ++e)
      if (ne[e]) return true;
    return false;
  };
  lo.assign(N, 0);
  cnt.assign(N, 0);
  int64_t total = 0;
  for (int m = 0; m < N; ++m) {
    int a0 = m, b0 = m;
    while (a0 - 1 >= std::max(m - p + 1, 0) && shares(m, a0 - 1)) --a0;
    while (b0 + 1 <= std::min(m + p - 1, N - 1) && shares(m, b0 + 1)) ++b0;
    lo[m] = a0;
    cnt[m] = b0 - a0 + 1;
    total += cnt[m];
  }
  return total;
}

}  // namespace
}  // namespace igasf

extern "C" int64_t igasf_assembled_nnz(igasf_handle h) try {
  using namespace igasf;
  if (!h) return set_error(IGASF_ERR_INVALID_ARG, "handle is NULL");
  int64_t nnz = 1;
  std::vector<int> lo, cnt;
  for (int a = 0; a < h->d; ++a) nnz *= pattern_1d(h, a, lo, cnt);
  return nnz;
} IGASF_CATCH_HOST

extern "C" int igasf_assemble_csr(igasf_handle h, int op, int64_t *rowptr, int64_t *colind,
                                  double *values, size_t workspace_limit_bytes, void *stream) try {
  using namespace igasf;
  if (!h || !rowptr || !colind || !values)
    return set_error(IGASF_ERR_INVALID_ARG, "handle, rowptr, colind and values must be non-NULL");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return set_error(IGASF_ERR_INVALID_ARG, "bad op");
  if (((uintptr_t)rowptr | (uintptr_t)colind | (uintptr_t)values) % 8)
    return set_error(IGASF_ERR_INVALID_ARG, "rowptr, colind and values must be 8-byte aligned");
  const Variant &v64 = h->var[IGASF_FP64];
  if (!v64.present) return set_error(IGASF_ERR_UNSUPPORTED, "assembly reads the FP64 factors: store FP64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t limit = workspace_limit_bytes ? workspace_limit_bytes : ((size_t)2 << 30);

  AsmDims g;
  memset(&g, 0, sizeof(g));
  g.d = h->d;
  g.p = h->p;
  g.W = 2 * h->p - 1;
  for (int a = 0; a < 3; ++a) {
    g.N[a] = a < h->d ? h->N[a] : 1;
    g.K[a] = a < h->d ? h->K[a] : 1;
    g.Q[a] = a < h->d ? h->Q[a] : 1;
    g.tabB[a] = a < h->d ? h->tabB[a] : nullptr;
    g.tabD[a] = a < h->d ? h->tabD[a] : nullptr;
  }
  g.stiff = op == IGASF_STIFFNESS;
  g.nterms = g.stiff ? h->d * h->d : 1;
  g.ngroups = g.stiff ? 4 : 1;
  g.nf = num_fields(h->d, op);
  const int d = h->d, p = h->p, W = g.W, L = d - 1;
  const int Qmid = d == 3 ? g.Q[1] : 1;

  // per-direction first columns and prefix sums of the column counts (host, then device)
  std::vector<int64_t> pre_h;
  std::vector<int> lo_h;
  size_t pre_off[3] = {0, 0, 0}, lo_off[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    std::vector<int> lo, cnt;
    pattern_1d(h, a, lo, cnt);
    pre_off[a] = pre_h.size();
    lo_off[a] = lo_h.size();
    int64_t acc = 0;
    pre_h.push_back(0);
    for (int m = 0; m < g.N[a]; ++m) {
      acc += cnt[m];
      pre_h.push_back(acc);
    }
    lo_h.insert(lo_h.end(), lo.begin(), lo.end());
  }
  // chunk size: element layers of the last direction whose levels fit the limit
  const int64_t inner1 = (int64_t)g.N[0] * W;
  const int64_t inner = d == 3 ? (int64_t)g.N[1] * W * inner1 : inner1;
  const int64_t per_q = (int64_t)g.nf * Qmid * g.Q[0] + (int64_t)g.nterms * Qmid * inner1 +
                        (d == 3 ? (int64_t)g.ngroups * inner : 0);   // doubles per last-dir point
  const int64_t per_layer_bytes = per_q * p * 8;
  int layers = (int)std::max<int64_t>(1, std::min<int64_t>(g.K[L], (int64_t)(limit / per_layer_bytes)));
  const int64_t QCmax = (int64_t)layers * p;

  int64_t *pre_d = nullptr;
  int *lo_d = nullptr;
  double *Fc = nullptr, *L1 = nullptr, *L2 = nullptr, *PT = nullptr;
  size_t pt_off[3] = {0, 0, 0}, pt_total = 0;
  for (int a = 0; a < d; ++a) {
    pt_off[a] = pt_total;
    pt_total += (size_t)4 * g.N[a] * W * p * p;
  }
  cudaError_t e = cudaMalloc((void **)&pre_d, sizeof(int64_t) * pre_h.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&lo_d, sizeof(int) * lo_h.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&PT, sizeof(double) * pt_total);
  if (e == cudaSuccess) e = cudaMalloc((void **)&Fc, sizeof(double) * g.nf * QCmax * Qmid * g.Q[0]);
  if (e == cudaSuccess) e = cudaMalloc((void **)&L1, sizeof(double) * g.nterms * QCmax * Qmid * inner1);
  if (e == cudaSuccess && d == 3) e = cudaMalloc((void **)&L2, sizeof(double) * g.ngroups * QCmax * inner);
  auto release = [&]() {
    cudaFree(PT);
    cudaFree(pre_d);
    cudaFree(lo_d);
    cudaFree(Fc);
    cudaFree(L1);
    cudaFree(L2);
  };
  if (e != cudaSuccess) {
    release();
    return set_error(e == cudaErrorMemoryAllocation ? IGASF_ERR_OOM : IGASF_ERR_CUDA,
                     (std::string("assembly workspace: ") + cudaGetErrorString(e)).c_str());
  }
  e = cudaMemcpyAsync(pre_d, pre_h.data(), sizeof(int64_t) * pre_h.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lo_d, lo_h.data(), sizeof(int) * lo_h.size(), cudaMemcpyHostToDevice, s);
  CsrDims c;
  for (int a = 0; a < 3; ++a) {
    c.pre[a] = a < d ? pre_d + pre_off[a] : nullptr;
    c.lo[a] = a < d ? lo_d + lo_off[a] : nullptr;
  }
  int64_t Ntot = 1, Wd = 1;
  for (int a = 0; a < d; ++a) {
    Ntot *= g.N[a];
    Wd *= W;
  }
  const int64_t nnz = igasf_assembled_nnz(h);
  const int T = 256;
  for (int a = 0; a < d && e == cudaSuccess; ++a) {
    g.PT[a] = PT + pt_off[a];
    pair_table_kernel<<<blocks_for((int64_t)4 * g.N[a] * W * p * p, T), T, 0, s>>>(g, a, PT + pt_off[a]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(values, 0, sizeof(double) * nnz, s);
  if (e == cudaSuccess) {
    csr_structure_kernel<<<blocks_for(Ntot * Wd, T), T, 0, s>>>(g, c, rowptr, colind);
    e = cudaGetLastError();
  }
  const double *D = static_cast<const double *>(op == IGASF_MASS ? v64.L.DM : v64.L.DK);
  for (int e0 = 0; e0 < g.K[L] && e == cudaSuccess; e0 += layers) {
    const int e1 = std::min(g.K[L], e0 + layers);
    const int QC = (e1 - e0) * p;
    chunk_factors_kernel<<<blocks_for((int64_t)QC * Qmid * g.Q[0], T), T, 0, s>>>(g, v64.L, D, e0 * p, QC,
                                                                                 Qmid, Fc);
    level1_kernel<<<blocks_for((int64_t)g.nterms * QC * Qmid * inner1, T), T, 0, s>>>(g, Fc, QC, Qmid, L1);
    const double *Lprev = L1;
    if (d == 3) {
      level2_kernel<<<blocks_for((int64_t)QC * inner, T), T, 0, s>>>(g, L1, QC, L2);
      Lprev = L2;
    }
    // rows of the last direction touched by elements e0..e1-1
    const int mL0 = e0, mL1 = std::min(e1 - 1 + p - 1, g.N[L] - 1);
    const int nrows = mL1 - mL0 + 1;
    last_level_kernel<<<blocks_for((int64_t)nrows * W * inner, T), T, 0, s>>>(g, c, Lprev, QC, e0, e1, mL0,
                                                                              nrows, values);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess)
    return set_error(IGASF_ERR_CUDA, (std::string("assembly: ") + cudaGetErrorString(e)).c_str());
  return IGASF_OK;
} IGASF_CATCH_HOST
