// igasf_cg_solve: Jacobi-preconditioned CG for the stiffness operator with
// homogeneous Dirichlet conditions, all-FP64 or with FP32 inner solves inside
// FP64 iterative refinement. The operator is only ever applied matrix-free
// (v = K u through the tile kernels); vectors, dot products and the Jacobi
// diagonal are computed by the kernels below. Reductions are two-pass with a
// fixed grid and a fixed summation order, so a solve is bitwise reproducible.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "igasf.h"
#include "igasf_internal.h"
#include "layout.h"
#include "plan.h"

namespace igasf {

int set_error(int code, const char *msg);

namespace {

constexpr int kRedBlocks = 1024;  // first reduction pass: fixed grid
constexpr int kRedThreads = 256;

// Interior dof: index 1..N_a - 2 in every direction.
__device__ __forceinline__ bool interior(int64_t n, int N0, int N1, int N2) {
  const int i0 = (int)(n % N0);
  const int64_t r = n / N0;
  const int i1 = (int)(r % N1), i2 = (int)(r / N1);
  return i0 > 0 && i0 < N0 - 1 && i1 > 0 && i1 < N1 - 1 && i2 > 0 && i2 < N2 - 1;
}

// ---------------------------------------------------------------------------
// Jacobi diagonal of K, FP64: diag_m = sum over the elements of supp(phi_m),
// their quadrature points and (i, j) of d_i phi_m D_ij d_j phi_m, one thread
// per dof, read from the FP64 stiffness factors (w folded in). Deterministic.
// ---------------------------------------------------------------------------
struct DiagParams {
  int p;
  int N[3], K[3], S[3], T[3];
  int plane, lanes;
  const double *DK;
  const double *tabB[3], *tabD[3];   // FP64 [j][K p]
  double *dinv64;
  float *dinv32;
};

__device__ double factor_k(const DiagParams &g, int f, const int *qg) {
  return g.DK[layout_index_q(3, g.p, g.S, g.T, g.plane, g.lanes, 8, 6, f, qg)];
}

__global__ void diag_kernel(const DiagParams g) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t Ntot = (int64_t)g.N[0] * g.N[1] * g.N[2];
  if (n >= Ntot) return;
  int m[3];
  m[0] = (int)(n % g.N[0]);
  m[1] = (int)((n / g.N[0]) % g.N[1]);
  m[2] = (int)(n / ((int64_t)g.N[0] * g.N[1]));
  if (!(m[0] > 0 && m[0] < g.N[0] - 1 && m[1] > 0 && m[1] < g.N[1] - 1 && m[2] > 0 &&
        m[2] < g.N[2] - 1)) {
    g.dinv64[n] = 0.0;   // boundary dofs stay zero
    g.dinv32[n] = 0.f;
    return;
  }
  const int p = g.p;
  const int fi[6] = {0, 0, 0, 1, 1, 2}, fj[6] = {0, 1, 2, 1, 2, 2};
  double diag = 0.0;
  // elements e with m - p + 1 <= e <= m, inside the patch (every knot span is an
  // element; the empty spans of repeated knots have zero factors)
  for (int e2 = max(0, m[2] - p + 1); e2 <= min(g.K[2] - 1, m[2]); ++e2)
    for (int e1 = max(0, m[1] - p + 1); e1 <= min(g.K[1] - 1, m[1]); ++e1)
      for (int e0 = max(0, m[0] - p + 1); e0 <= min(g.K[0] - 1, m[0]); ++e0) {
        const int j[3] = {m[0] - e0, m[1] - e1, m[2] - e2};
        const int e[3] = {e0, e1, e2};
        for (int c = 0; c < p; ++c)
          for (int b = 0; b < p; ++b)
            for (int a = 0; a < p; ++a) {
              const int qg[3] = {e[0] * p + a, e[1] * p + b, e[2] * p + c};
              double val[3], der[3];
              for (int d = 0; d < 3; ++d) {
                const int Qd = g.K[d] * p;
                val[d] = g.tabB[d][j[d] * Qd + qg[d]];
                der[d] = g.tabD[d][j[d] * Qd + qg[d]];
              }
              const double grad[3] = {der[0] * val[1] * val[2], val[0] * der[1] * val[2],
                                      val[0] * val[1] * der[2]};
              for (int f = 0; f < 6; ++f) {
                const double t = grad[fi[f]] * grad[fj[f]] * factor_k(g, f, qg);
                diag += fi[f] == fj[f] ? t : 2.0 * t;
              }
            }
      }
  g.dinv64[n] = diag > 0.0 ? 1.0 / diag : 0.0;
  g.dinv32[n] = (float)g.dinv64[n];
}

// ---------------------------------------------------------------------------
// Vector kernels. Every reduction runs on a fixed grid of kRedBlocks blocks
// with grid-stride loops, accumulates in FP64, and writes one partial per
// block; final_kernel adds the partials in a fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  __syncthreads();
  return t;   // valid in thread 0
}

// partial[k * kRedBlocks + b] -> out[k] for k < nout
__global__ void final_kernel(const double *partial, double *out, int nout) {
  __shared__ double sh[32];
  for (int k = 0; k < nout; ++k) {
    double v = 0.0;
    for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) v += partial[k * kRedBlocks + i];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) out[k] = t;
  }
}

// r = mask(b - Kx); partial of r.r
__global__ void residual_kernel(const double *b, const double *kx, double *r, int64_t n, int N0,
                                int N1, int N2, double *partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = interior(i, N0, N1, N2) ? b[i] - kx[i] : 0.0;
    r[i] = v;
    acc += v * v;
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// start of a PCG: x = 0, r = rhs (masked, converted), z = Dinv r, p = z;
// partials of r.z and r.r
template <typename T, typename TR>
__global__ void pcg_start_kernel(const TR *rhs, T *x, T *r, T *z, T *pv, const T *dinv, int64_t n,
                                 int N0, int N1, int N2, double *partial) {
  __shared__ double sh[32];
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = interior(i, N0, N1, N2) ? (T)rhs[i] : T(0);
    const T zi = dinv[i] * ri;
    x[i] = T(0);
    r[i] = ri;
    z[i] = zi;
    pv[i] = zi;
    rz += (double)ri * (double)zi;
    rr += (double)ri * (double)ri;
  }
  double t = block_sum(rz, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
  t = block_sum(rr, sh);
  if (threadIdx.x == 0) partial[kRedBlocks + blockIdx.x] = t;
}

// partial of p.q (p is zero on the boundary, so this is the interior sum)
template <typename T>
__global__ void dot_kernel(const T *a, const T *b, int64_t n, double *partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// x += alpha p; r = mask(r - alpha q); z = Dinv r; partials of r.z and r.r
template <typename T>
__global__ void pcg_update_kernel(T *x, T *r, T *z, const T *pv, const T *q, const T *dinv,
                                  double alpha, int64_t n, int N0, int N1, int N2,
                                  double *partial) {
  __shared__ double sh[32];
  const T a = (T)alpha;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * pv[i];
    const T ri = interior(i, N0, N1, N2) ? r[i] - a * q[i] : T(0);
    const T zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    rz += (double)ri * (double)zi;
    rr += (double)ri * (double)ri;
  }
  double t = block_sum(rz, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
  t = block_sum(rr, sh);
  if (threadIdx.x == 0) partial[kRedBlocks + blockIdx.x] = t;
}

// p = z + beta p
template <typename T>
__global__ void direction_kernel(T *pv, const T *z, double beta, int64_t n) {
  const T bt = (T)beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    pv[i] = z[i] + bt * pv[i];
}

// x64 += d32 (the refinement step)
__global__ void refine_kernel(double *x, const float *d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

}  // namespace
}  // namespace igasf

namespace {

using igasf::kRedBlocks;
using igasf::kRedThreads;

// Device scratch of one solve: FP64 vectors, FP32 vectors (refined solve only),
// reduction partials and scalars.
struct Work {
  double *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr, *kx = nullptr;
  float *d32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  double *partial = nullptr, *scal = nullptr;
  void release() {
    void *ptrs[] = {r, z, pv, q, kx, d32, r32, z32, p32, q32, partial, scal};
    for (void *p : ptrs) cudaFree(p);
  }
};

struct Ctx {
  igasf_plan *h;
  cudaStream_t s;
  int64_t n;
  int N0, N1, N2;
  Work w;
  cudaError_t err = cudaSuccess;
  int rc = IGASF_OK;
  // sum the first `k` partial rows and copy them to the host
  bool fetch(int k, double *out) {
    igasf::final_kernel<<<1, kRedThreads, 0, s>>>(w.partial, w.scal, k);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(out, w.scal, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    return err == cudaSuccess;
  }
  bool apply(int prec, const void *u, void *v) {
    rc = igasf_apply_prec(h, IGASF_STIFFNESS, prec, u, v, s);
    return rc == IGASF_OK;
  }
};

// PCG on K y = rhs (masked), y from zero, in precision T; stops when the
// residual norm drops to rel * ||rhs|| or after max_it iterations.
template <typename T, typename TR>
bool pcg(Ctx &c, int prec, const TR *rhs, T *y, T *r, T *z, T *pv, T *q, const T *dinv, double rel,
         int max_it, int *iters, double *rnorm0) {
  igasf::pcg_start_kernel<T, TR><<<kRedBlocks, kRedThreads, 0, c.s>>>(rhs, y, r, z, pv, dinv, c.n, c.N0,
                                                                     c.N1, c.N2, c.w.partial);
  double sc[2];
  if (!c.fetch(2, sc)) return false;
  double rz = sc[0];
  const double r0 = std::sqrt(sc[1]);
  if (rnorm0) *rnorm0 = r0;
  if (r0 == 0.0) return true;
  for (int it = 0; it < max_it; ++it) {
    if (!c.apply(prec, pv, q)) return false;
    igasf::dot_kernel<T><<<kRedBlocks, kRedThreads, 0, c.s>>>(pv, q, c.n, c.w.partial);
    double pq;
    if (!c.fetch(1, &pq)) return false;
    if (!(pq > 0.0)) break;   // breakdown (or an exact solve)
    const double alpha = rz / pq;
    igasf::pcg_update_kernel<T><<<kRedBlocks, kRedThreads, 0, c.s>>>(y, r, z, pv, q, dinv, alpha, c.n,
                                                                    c.N0, c.N1, c.N2, c.w.partial);
    if (!c.fetch(2, sc)) return false;
    ++*iters;
    if (std::sqrt(sc[1]) <= rel * r0) break;
    const double beta = sc[0] / rz;
    rz = sc[0];
    igasf::direction_kernel<T><<<kRedBlocks, kRedThreads, 0, c.s>>>(pv, z, beta, c.n);
  }
  return true;
}

// r = mask(b - K x) in FP64; returns ||r||
bool residual(Ctx &c, const double *b, const double *x, double *rn) {
  if (!c.apply(IGASF_FP64, x, c.w.kx)) return false;
  igasf::residual_kernel<<<kRedBlocks, kRedThreads, 0, c.s>>>(b, c.w.kx, c.w.r, c.n, c.N0, c.N1, c.N2,
                                                              c.w.partial);
  double rr;
  if (!c.fetch(1, &rr)) return false;
  *rn = std::sqrt(rr);
  return true;
}

}  // namespace

extern "C" int igasf_cg_solve(igasf_handle h, int inner_prec, const double *b, double *x,
                              double rtol, double inner_rtol, int max_iterations,
                              igasf_cg_report *report, void *stream) try {
  using namespace igasf;
  if (!h || !b || !x) return set_error(IGASF_ERR_INVALID_ARG, "handle, b and x must be non-NULL");
  if (h->d != 3) return set_error(IGASF_ERR_UNSUPPORTED, "the solver handles d = 3 plans");
  if (inner_prec < 0 || inner_prec >= kNumPrec)
    return set_error(IGASF_ERR_INVALID_ARG, "inner_prec must be one of the igasf_prec values");
  if (!h->var[IGASF_FP64].present || !h->var[inner_prec].present)
    return set_error(IGASF_ERR_UNSUPPORTED, "the solve needs FP64 (and the inner precision) stored");
  if (!(rtol > 0.0) || !(inner_rtol > 0.0 && inner_rtol < 1.0) || max_iterations < 1)
    return set_error(IGASF_ERR_INVALID_ARG, "need rtol > 0, 0 < inner_rtol < 1, max_iterations >= 1");
  if (((uintptr_t)b % 8) || ((uintptr_t)x % 8)) return set_error(IGASF_ERR_INVALID_ARG, "b and x must be 8-byte aligned");
  Ctx c;
  c.h = h;
  c.s = static_cast<cudaStream_t>(stream);
  c.n = h->Ntot;
  c.N0 = h->N[0];
  c.N1 = h->N[1];
  c.N2 = h->N[2];
  const size_t n = (size_t)c.n;
  auto fail_cuda = [&](cudaError_t e, const char *what) {
    c.w.release();
    return set_error(e == cudaErrorMemoryAllocation ? IGASF_ERR_OOM : IGASF_ERR_CUDA,
                     (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
  };
  cudaError_t e = cudaSuccess;
  // Jacobi diagonal, once per plan
  if (!h->dinv64) {
    e = cudaMalloc((void **)&h->dinv64, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dinv32, sizeof(float) * n);
    if (e != cudaSuccess) {
      cudaFree(h->dinv64);
      cudaFree(h->dinv32);
      h->dinv64 = nullptr;
      h->dinv32 = nullptr;
      return fail_cuda(e, "Jacobi diagonal");
    }
    const Variant &v = h->var[IGASF_FP64];
    DiagParams g;
    memset(&g, 0, sizeof(g));
    g.p = h->p;
    for (int a = 0; a < 3; ++a) {
      g.N[a] = h->N[a];
      g.K[a] = h->K[a];
      g.S[a] = v.k.S[a];
      g.T[a] = v.T[a];
      g.tabB[a] = h->tabB[a];
      g.tabD[a] = h->tabD[a];
    }
    g.plane = v.L.plane;
    g.lanes = v.L.lanes;
    g.DK = static_cast<const double *>(v.L.DK);
    g.dinv64 = h->dinv64;
    g.dinv32 = h->dinv32;
    diag_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c.s>>>(g);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
    if (e != cudaSuccess) {
      cudaFree(h->dinv64);
      cudaFree(h->dinv32);
      h->dinv64 = nullptr;
      h->dinv32 = nullptr;
      return fail_cuda(e, "Jacobi diagonal kernel");
    }
  }
  // workspace
  Work &w = c.w;
  double **d64[] = {&w.r, &w.z, &w.pv, &w.q, &w.kx};
  for (double **pp : d64)
    if (e == cudaSuccess) e = cudaMalloc((void **)pp, sizeof(double) * n);
  if (inner_prec != IGASF_FP64) {
    float **f32[] = {&w.d32, &w.r32, &w.z32, &w.p32, &w.q32};
    for (float **pp : f32)
      if (e == cudaSuccess) e = cudaMalloc((void **)pp, sizeof(float) * n);
  }
  if (e == cudaSuccess) e = cudaMalloc((void **)&w.partial, sizeof(double) * 2 * kRedBlocks);
  if (e == cudaSuccess) e = cudaMalloc((void **)&w.scal, sizeof(double) * 2);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return fail_cuda(e, "solver workspace");

  const auto t0 = std::chrono::steady_clock::now();
  igasf_cg_report rep;
  memset(&rep, 0, sizeof(rep));
  bool ok = true;
  double bnorm = 0.0, rn = 0.0;
  if (inner_prec == IGASF_FP64) {
    double r0 = 0.0;
    ok = pcg<double, double>(c, IGASF_FP64, b, x, w.r, w.z, w.pv, w.q, h->dinv64, rtol,
                             max_iterations, &rep.inner_iterations, &r0);
    bnorm = r0;
    if (ok) ok = residual(c, b, x, &rn);
    rep.outer_iterations = 1;
  } else {
    e = cudaMemsetAsync(x, 0, sizeof(double) * n, c.s);
    ok = e == cudaSuccess && residual(c, b, x, &rn);   // r = b (masked), x = 0
    bnorm = rn;
    while (ok && rn > rtol * bnorm && rep.inner_iterations < max_iterations) {
      int it_before = rep.inner_iterations;
      ok = pcg<float, double>(c, inner_prec, w.r, w.d32, w.r32, w.z32, w.p32, w.q32, h->dinv32,
                              inner_rtol, max_iterations - rep.inner_iterations,
                              &rep.inner_iterations, nullptr);
      if (!ok) break;
      refine_kernel<<<kRedBlocks, kRedThreads, 0, c.s>>>(x, w.d32, c.n);
      ok = residual(c, b, x, &rn);
      ++rep.outer_iterations;
      if (rep.inner_iterations == it_before) break;   // no progress possible
    }
  }
  if (!ok) {
    const int rc = c.rc != IGASF_OK ? c.rc : -1;
    if (c.rc != IGASF_OK) {
      w.release();
      return rc;
    }
    return fail_cuda(c.err != cudaSuccess ? c.err : cudaErrorUnknown, "solver");
  }
  rep.final_relres = bnorm > 0.0 ? rn / bnorm : 0.0;
  rep.converged = rep.final_relres <= rtol;
  rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  w.release();
  if (report) *report = rep;
  return IGASF_OK;
} IGASF_CATCH_HOST
