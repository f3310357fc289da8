// C ABI of libigasf: argument validation, plan lifetime, dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "igasf.h"
#include "igasf_internal.h"
#include "plan.h"

using namespace igasf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(IGASF_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(IGASF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void destroy_events(igasf_plan *h) {
  for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
  h->prof_events.clear();
  h->prof_next = 0;
}

void free_plan(igasf_plan *h) {
  if (!h) return;
  destroy_events(h);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  cudaFree(h->status);
  cudaFree(h->ctrl64);
  cudaFree(h->dinv64);
  cudaFree(h->dinv32);
  for (int a = 0; a < kMaxDim; ++a) {
    cudaFree(h->knots[a]);
    cudaFree(h->span[a]);
    cudaFree(h->nodes[a]);
    cudaFree(h->weights[a]);
    cudaFree(h->tabB[a]);
    cudaFree(h->tabD[a]);
  }
  for (auto &v : h->var) {
    cudaFree(v.L.DM);
    cudaFree(v.L.DK);
    for (int a = 0; a < kMaxDim; ++a) {
      cudaFree(v.tabB[a]);
      cudaFree(v.tabD[a]);
      cudaFree(v.wq32[a]);
      cudaFree(v.gtab[a]);
    }
    cudaFree(v.ctrl32);
    cudaFree(v.vpart);
    cudaFree(v.u_stage);
    cudaFree(v.u_stage2);
    cudaFree(v.v_stage);
  }
  delete h;
}

size_t prec_size(int prec) { return vector_bytes(prec); }

// Position in the plan's full quadrature grid (all spans) of the API's
// quadrature point q = (q_3 Qe_2 + q_2) Qe_1 + q_1 (non-empty spans only).
int64_t full_qp_index(const igasf_plan *h, int64_t q) {
  int64_t full = 0, stride = 1;
  for (int a = 0; a < h->d; ++a) {
    const int64_t Qe = (int64_t)h->Ke[a] * h->p;
    const int qa = (int)(q % Qe);
    q /= Qe;
    full += ((int64_t)h->elem[a][qa / h->p] * h->p + qa % h->p) * stride;
    stride *= h->Q[a];
  }
  return full;
}

// Per-point data with nc components: the API's points out of the full grid,
// and back (the points of empty spans get zeros).
void compact_qp(const igasf_plan *h, const double *full, double *api, int nc) {
  for (int64_t q = 0; q < h->Qapi; ++q) {
    const int64_t f = full_qp_index(h, q);
    for (int c = 0; c < nc; ++c) api[q * nc + c] = full[f * nc + c];
  }
}

void expand_qp(const igasf_plan *h, const double *api, double *full, int nc) {
  std::fill(full, full + h->Qtot * nc, 0.0);
  for (int64_t q = 0; q < h->Qapi; ++q) {
    const int64_t f = full_qp_index(h, q);
    for (int c = 0; c < nc; ++c) full[f * nc + c] = api[q * nc + c];
  }
}

// Validate one open knot vector (interior multiplicity at most p - 1); count
// its elements, the knot spans k = p-1 .. nk-p-1 with empty ones included.
// Returns IGASF_OK or an error.
int check_knots(int dir, int p, int nk, const double *t, int *K_out) {
  if (!t) return fail(IGASF_ERR_INVALID_ARG, "knots[%d] is NULL", dir);
  if (nk < 2 * p) return fail(IGASF_ERR_KNOTS, "knot vector %d has %d entries, needs >= %d", dir, nk, 2 * p);
  for (int i = 0; i < nk; ++i)
    if (!(t[i] == t[i]) || t[i] - t[i] != 0.0)
      return fail(IGASF_ERR_KNOTS, "knot vector %d has a non-finite entry", dir);
  for (int i = 0; i + 1 < nk; ++i)
    if (t[i + 1] < t[i]) return fail(IGASF_ERR_KNOTS, "knot vector %d decreases at %d", dir, i);
  for (int i = 1; i < p; ++i)
    if (t[i] != t[0] || t[nk - 1 - i] != t[nk - 1])
      return fail(IGASF_ERR_KNOTS, "knot vector %d is not open (ends need multiplicity %d)", dir, p);
  if (t[p] == t[0]) return fail(IGASF_ERR_KNOTS, "knot vector %d: first knot repeated more than p times", dir);
  if (t[nk - 1 - p] == t[nk - 1]) return fail(IGASF_ERR_KNOTS, "knot vector %d: last knot repeated more than p times", dir);
  if (!(t[nk - 1] > t[0])) return fail(IGASF_ERR_KNOTS, "knot vector %d spans an empty interval", dir);
  int K = 0;
  for (int i = p; i < nk - p;) {
    int m = 1;
    while (i + m < nk - p && t[i + m] == t[i]) ++m;
    if (m >= p) return fail(IGASF_ERR_KNOTS, "knot vector %d: interior multiplicity %d >= order %d", dir, m, p);
    i += m;
  }
  K = nk - 2 * p + 1;
  *K_out = K;
  return IGASF_OK;
}

int alloc(void **p, size_t bytes, const char *what) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  return IGASF_OK;
}

#define TRY(x)                  \
  do {                          \
    int rc_ = (x);              \
    if (rc_ != IGASF_OK) {      \
      free_plan(h);             \
      return rc_;               \
    }                           \
  } while (0)

#define TRY_CUDA(x, what)                   \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) {                \
      int rc_ = cuda_fail(e_, what);        \
      free_plan(h);                         \
      return rc_;                           \
    }                                       \
  } while (0)

}  // namespace

namespace igasf {

// Used by igasf_apply_noalloc (noalloc.cu): the apply with a caller-given
// scratch buffer in place of the plan's workspace.
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

void make_apply_params(const igasf_plan *h, const Variant &var, int op, const void *u, void *vpart,
                       ApplyParams *prm) {
  memset(prm, 0, sizeof(*prm));
  prm->u = u;
  prm->vpart = vpart;
  prm->D = op == IGASF_MASS ? var.L.DM : var.L.DK;
  for (int a = 0; a < kMaxDim; ++a) {
    prm->tabB[a] = var.tabB[a];
    prm->tabD[a] = var.tabD[a];
    prm->N[a] = h->N[a];
    prm->K[a] = h->K[a];
    prm->T[a] = var.T[a];
    prm->Qpad[a] = var.Qpad[a];
    prm->wq[a] = var.wq32[a];
  }
  prm->ntiles = var.ntiles;
  prm->status = h->status;
  prm->wait_limit = h->wait_limit;
  prm->skip_slab = h->skip_slab;
  prm->ctrl = var.ctrl32;
  prm->coef_kind = h->coef_kind;
  prm->coef_a = (float)(h->coef_kind == IGASF_COEF_EXP_SIN_COS ? h->coef_alpha : h->coef_constant);
}

int apply_with_workspace(igasf_plan *h, int op, int prec, const void *u, void *v, void *ws,
                         size_t ws_bytes, void *stream) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return fail(IGASF_ERR_INVALID_ARG, "op = %d", op);
  if (prec < 0 || prec >= kNumPrec) return fail(IGASF_ERR_INVALID_ARG, "prec = %d", prec);
  Variant &var = h->var[prec];
  if (!var.present) return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  if (!u || !v) return fail(IGASF_ERR_INVALID_ARG, "u and v must be non-NULL");
  if (var.vpart_bytes > ws_bytes)
    return fail(IGASF_ERR_UNSUPPORTED,
                "this plan needs %zu bytes of scratch; the static scratch holds %zu bytes",
                var.vpart_bytes, ws_bytes);
  const size_t es = prec_size(prec);
  if (((uintptr_t)u % es) || ((uintptr_t)v % es))
    return fail(IGASF_ERR_INVALID_ARG, "u and v must be aligned to %zu bytes", es);
  const uintptr_t ub = (uintptr_t)u, vb = (uintptr_t)v, len = (uintptr_t)h->Ntot * es;
  if (ub < vb + len && vb < ub + len) return fail(IGASF_ERR_INVALID_ARG, "u and v overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ApplyParams prm;
  make_apply_params(h, var, op, u, ws, &prm);
  cudaError_t e = var.k.launch[op](prm, s);
  if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
  e = launch_gather(h->d, vectors_are_float(prec), ws, v, h->N, var.T, var.k.S, h->p, var.gtab, s);
  if (e != cudaSuccess) return cuda_fail(e, "gather kernel launch");
  return IGASF_OK;
}

}  // namespace igasf

extern "C" {

int igasf_version(void) { return IGASF_VERSION; }

const char *igasf_last_error_message(void) { return g_last_error.c_str(); }

int igasf_list_kernels(int d, int p, int prec, int geometry, int *tiles, int *variants, int max_out) {
  g_last_error.clear();
  if (d != 2 && d != 3) return fail(IGASF_ERR_INVALID_ARG, "d = %d (2 or 3)", d);
  if (p < 2 || p > IGASF_MAX_ORDER) return fail(IGASF_ERR_INVALID_ARG, "p = %d (2..%d)", p, IGASF_MAX_ORDER);
  if (prec < 0 || prec >= kNumPrec) return fail(IGASF_ERR_INVALID_ARG, "prec = %d", prec);
  if (geometry != IGASF_GEOMETRY_STORED && geometry != IGASF_GEOMETRY_ON_THE_FLY)
    return fail(IGASF_ERR_INVALID_ARG, "geometry = %d", geometry);
  if (max_out < 0) return fail(IGASF_ERR_INVALID_ARG, "max_out < 0");
  ApplyKernel cand[kMaxCandidates];
  int n = 0;
  if (geometry == IGASF_GEOMETRY_STORED)
    n = list_apply_kernels(d, p, prec, cand, kMaxCandidates);
  else if (d == 3 && prec == IGASF_FP32)
    n = list_geometry_kernels(p, cand, kMaxCandidates);
  for (int i = 0; i < n && i < max_out; ++i) {
    for (int a = 0; a < 3; ++a)
      if (tiles) tiles[3 * i + a] = a < d ? cand[i].S[a] : 1;
    if (variants) variants[i] = cand[i].variant;
  }
  return n;
}

// The body of igasf_setup. *created receives the plan as soon as it exists; the
// error paths free it themselves (after recording their message, the last step
// that can throw), and igasf_setup frees it if a host exception interrupts the
// setup.
static int setup_impl(int d, const int *orders, const int *knot_lengths, const double *const *knots,
                      const double *ctrl, const igasf_coef *coef, const igasf_options *opt,
                      igasf_handle *out, igasf_plan **created) {
  g_last_error.clear();
  if (!out) return fail(IGASF_ERR_INVALID_ARG, "out is NULL");
  if (d != 2 && d != 3) return fail(IGASF_ERR_UNSUPPORTED, "d = %d; supported: 2, 3", d);
  if (!orders || !knot_lengths || !knots || !ctrl)
    return fail(IGASF_ERR_INVALID_ARG, "orders, knot_lengths, knots and ctrl must be non-NULL");
  const int p = orders[0];
  for (int a = 0; a < d; ++a) {
    if (orders[a] < 1) return fail(IGASF_ERR_INVALID_ARG, "order %d in direction %d", orders[a], a);
    if (orders[a] != p) return fail(IGASF_ERR_UNSUPPORTED, "orders differ between directions");
  }
  if (p < 2 || p > IGASF_MAX_ORDER)
    return fail(IGASF_ERR_UNSUPPORTED, "order p = %d; kernels are built for 2..%d", p, IGASF_MAX_ORDER);
  igasf_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  for (int r : o.reserved)
    if (r != 0) return fail(IGASF_ERR_INVALID_ARG, "options.reserved must be zero");
  if (o.kernel_variant < 0 || o.kernel_variant == IGASF_KERNEL_ON_THE_FLY ||
      o.kernel_variant > IGASF_KERNEL_MMA)
    return fail(IGASF_ERR_INVALID_ARG, "options.kernel_variant = %d", o.kernel_variant);
  if (o.default_prec < 0 || o.default_prec >= kNumPrec)
    return fail(IGASF_ERR_INVALID_ARG, "options.default_prec = %d", o.default_prec);
  unsigned precs = o.precisions ? o.precisions : IGASF_PREC_BIT(o.default_prec);
  if (precs & ~((1u << kNumPrec) - 1u))
    return fail(IGASF_ERR_INVALID_ARG, "options.precisions has unknown bits 0x%x", precs);
  if (!(precs & IGASF_PREC_BIT(o.default_prec)))
    return fail(IGASF_ERR_INVALID_ARG, "options.precisions must include default_prec");
  if (o.geometry != IGASF_GEOMETRY_STORED && o.geometry != IGASF_GEOMETRY_ON_THE_FLY)
    return fail(IGASF_ERR_INVALID_ARG, "options.geometry = %d", o.geometry);
  if (o.deterministic != 0 && o.deterministic != 1)
    return fail(IGASF_ERR_INVALID_ARG, "options.deterministic = %d (0 or 1)", o.deterministic);
  const bool geo = o.geometry == IGASF_GEOMETRY_ON_THE_FLY;
  if (geo && !(precs & IGASF_PREC_BIT(IGASF_FP32)))
    return fail(IGASF_ERR_INVALID_ARG, "factors on the fly are an FP32 mode: store FP32");
  igasf_coef c;
  c.kind = IGASF_COEF_CONSTANT;
  c.constant = 1.0;
  c.alpha = 0.0;
  c.values = nullptr;
  if (coef) c = *coef;
  if (c.kind < IGASF_COEF_CONSTANT || c.kind > IGASF_COEF_VALUES)
    return fail(IGASF_ERR_INVALID_ARG, "coef.kind = %d", c.kind);
  if (c.kind == IGASF_COEF_VALUES && !c.values)
    return fail(IGASF_ERR_INVALID_ARG, "coef.values is NULL");
  int K[kMaxDim] = {1, 1, 1};
  double ntot = 1.0, qtot = 1.0;
  for (int a = 0; a < d; ++a) {
    int rc = check_knots(a, p, knot_lengths[a], knots[a], &K[a]);
    if (rc != IGASF_OK) return rc;
    ntot *= knot_lengths[a] - p;
    qtot *= (double)K[a] * p;
  }
  if (ntot >= 2147483647.0 || qtot >= 9.0e15)
    return fail(IGASF_ERR_UNSUPPORTED, "patch too large: %.0f dofs (limit 2^31 - 1)", ntot);
  if (geo && d != 3) return fail(IGASF_ERR_UNSUPPORTED, "factors on the fly are built for d = 3");
  if (geo && c.kind == IGASF_COEF_VALUES)
    return fail(IGASF_ERR_UNSUPPORTED, "factors on the fly need a constant or exp-sin-cos coefficient");
  // which kernels
  ApplyKernel kern[kNumPrec];
  for (int prec = 0; prec < kNumPrec; ++prec) {
    if (!(precs & IGASF_PREC_BIT(prec))) continue;
    if (geo && prec == IGASF_FP32) {
      if (!find_geometry_kernel(p, o.tile, &kern[prec]))
        return fail(IGASF_ERR_UNSUPPORTED, "tile (%d, %d, %d) is not built for factors on the fly at p=%d",
                    o.tile[0], o.tile[1], o.tile[2], p);
      continue;
    }
    if (!find_apply_kernel(d, p, prec, nullptr, 0, &kern[prec]))
      return fail(IGASF_ERR_UNSUPPORTED, "no kernel for d=%d p=%d prec=%d", d, p, prec);
    if (!find_apply_kernel(d, p, prec, o.tile, o.kernel_variant, &kern[prec]))
      return fail(IGASF_ERR_UNSUPPORTED,
                  "tile (%d, %d, %d) with kernel variant %d is not built for d=%d p=%d prec=%d",
                  o.tile[0], o.tile[1], o.tile[2], o.kernel_variant, d, p, prec);
  }
  // host-side validation done: now the device
  igasf_plan *h = new (std::nothrow) igasf_plan();
  if (!h) return fail(IGASF_ERR_OOM, "host allocation");
  *created = h;
  h->d = d;
  h->p = p;
  h->default_prec = o.default_prec;
  h->coef_kind = c.kind;
  h->coef_constant = c.constant;
  h->coef_alpha = c.alpha;
  TRY_CUDA(cudaGetDevice(&h->device), "cudaGetDevice");
  TRY_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
  for (int i = 0; i < 2; ++i) {
    TRY_CUDA(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming), "events");
    TRY_CUDA(cudaEventCreateWithFlags(&h->ev_free[i], cudaEventDisableTiming), "events");
  }
  TRY(alloc((void **)&h->status, sizeof(unsigned int), "status word"));
  TRY_CUDA(cudaMemset(h->status, 0, sizeof(unsigned int)), "status word");
  h->Ntot = 1;
  h->Qtot = 1;
  for (int a = 0; a < d; ++a) {
    h->K[a] = K[a];
    h->N[a] = knot_lengths[a] - p;
    h->Q[a] = K[a] * p;
    h->Ntot *= h->N[a];
    h->Qtot *= h->Q[a];
  }
  h->Qapi = 1;
  for (int a = 0; a < d; ++a) {
    const double *t = knots[a];
    h->nonempty[a].assign(K[a], 0);
    for (int e = 0; e < K[a]; ++e)
      if (t[p + e] > t[p - 1 + e]) {
        h->nonempty[a][e] = 1;
        h->elem[a].push_back(e);
      }
    h->Ke[a] = (int)h->elem[a].size();
    h->Qapi *= (int64_t)h->Ke[a] * p;
    if (h->Ke[a] != K[a]) h->empty_spans = true;
  }
  cudaStream_t s = nullptr;
  // knots, spans, tables
  for (int a = 0; a < d; ++a) {
    const int nk = knot_lengths[a], Qa = h->Q[a];
    std::vector<int> span(K[a]);
    for (int e = 0; e < K[a]; ++e) span[e] = p - 1 + e;
    TRY(alloc((void **)&h->knots[a], sizeof(double) * nk, "knots"));
    TRY(alloc((void **)&h->span[a], sizeof(int) * K[a], "spans"));
    TRY(alloc((void **)&h->nodes[a], sizeof(double) * Qa, "nodes"));
    TRY(alloc((void **)&h->weights[a], sizeof(double) * Qa, "weights"));
    TRY(alloc((void **)&h->tabB[a], sizeof(double) * Qa * p, "tables"));
    TRY(alloc((void **)&h->tabD[a], sizeof(double) * Qa * p, "tables"));
    TRY_CUDA(cudaMemcpy(h->knots[a], knots[a], sizeof(double) * nk, cudaMemcpyHostToDevice), "copy knots");
    TRY_CUDA(cudaMemcpy(h->span[a], span.data(), sizeof(int) * K[a], cudaMemcpyHostToDevice), "copy spans");
    TRY_CUDA(launch_tables(p, K[a], h->knots[a], h->span[a], h->nodes[a], h->weights[a], h->tabB[a],
                           h->tabD[a], s),
             "tables kernel");
  }
  // per-precision layouts, tables, workspace
  GeometryParams g;
  memset(&g, 0, sizeof(g));
  for (int prec = 0; prec < kNumPrec; ++prec) {
    if (!(precs & IGASF_PREC_BIT(prec))) continue;
    Variant &v = h->var[prec];
    v.present = true;
    v.k = kern[prec];
    const size_t es = prec_size(prec);
    v.ntiles = 1;
    int64_t vol = 1;
    for (int a = 0; a < kMaxDim; ++a) v.T[a] = 1;
    for (int a = 0; a < d; ++a) {
      v.T[a] = (K[a] + v.k.S[a] - 1) / v.k.S[a];
      v.Qpad[a] = v.T[a] * v.k.S[a] * p;
      v.ntiles *= v.T[a];
      vol *= v.k.S[a] + p - 1;
    }
    v.L.d = d;
    v.L.p = p;
    for (int a = 0; a < kMaxDim; ++a) {
      v.L.S[a] = a < d ? v.k.S[a] : 1;
      v.L.T[a] = v.T[a];
    }
    v.L.plane = v.k.plane;
    v.L.lanes = v.k.lanes;
    v.L.elem_bytes = factor_bytes(prec);
    v.on_the_fly = geo && prec == IGASF_FP32;
    const int64_t Qlast = (int64_t)v.k.S[d - 1] * p;
    const int64_t rows = (int64_t)v.ntiles * Qlast;
    if (!v.on_the_fly) {
      v.bytesM = (size_t)rows * 1 * v.L.plane * v.L.elem_bytes;
      v.bytesK = (size_t)rows * num_fields(d, IGASF_STIFFNESS) * v.L.plane * v.L.elem_bytes;
      TRY(alloc(&v.L.DM, v.bytesM, "mass factors"));
      TRY(alloc(&v.L.DK, v.bytesK, "stiffness factors"));
      TRY_CUDA(cudaMemsetAsync(v.L.DM, 0, v.bytesM, s), "memset");
      TRY_CUDA(cudaMemsetAsync(v.L.DK, 0, v.bytesK, s), "memset");
    } else {
      // control points (FP32, one array per component) and padded FP32 weights
      std::vector<float> cs((size_t)3 * h->Ntot);
      for (int64_t n = 0; n < h->Ntot; ++n)
        for (int i = 0; i < 3; ++i) cs[(size_t)i * h->Ntot + n] = (float)ctrl[n * 3 + i];
      TRY(alloc((void **)&v.ctrl32, sizeof(float) * cs.size(), "control points"));
      TRY_CUDA(cudaMemcpy(v.ctrl32, cs.data(), sizeof(float) * cs.size(), cudaMemcpyHostToDevice), "copy");
      for (int a = 0; a < d; ++a) {
        std::vector<double> wd(h->Q[a]);
        std::vector<float> wf(v.Qpad[a], 0.f);
        TRY_CUDA(cudaMemcpy(wd.data(), h->weights[a], sizeof(double) * h->Q[a], cudaMemcpyDeviceToHost),
                 "weights");
        for (int q = 0; q < h->Q[a]; ++q) wf[q] = (float)wd[q];
        TRY(alloc((void **)&v.wq32[a], sizeof(float) * v.Qpad[a], "weights"));
        TRY_CUDA(cudaMemcpy(v.wq32[a], wf.data(), sizeof(float) * v.Qpad[a], cudaMemcpyHostToDevice), "copy");
      }
    }
    for (int a = 0; a < d; ++a) {
      TRY(alloc(&v.tabB[a], es * p * v.Qpad[a], "tables"));
      TRY(alloc(&v.tabD[a], es * p * v.Qpad[a], "tables"));
      TRY_CUDA(launch_pad_tables(p, K[a], v.Qpad[a], h->tabB[a], v.tabB[a], vectors_are_float(prec), s),
               "pad tables");
      TRY_CUDA(launch_pad_tables(p, K[a], v.Qpad[a], h->tabD[a], v.tabD[a], vectors_are_float(prec), s),
               "pad tables");
    }
    for (int a = 0; a < kMaxDim; ++a) {
      std::vector<int2> gt;
      if (a < d) gather_table(h->N[a], v.k.S[a], v.k.S[a] + p - 1, v.T[a], gt);
      else gather_table(0, 1, 1, 1, gt);
      TRY(alloc((void **)&v.gtab[a], sizeof(int2) * gt.size(), "gather tables"));
      TRY_CUDA(cudaMemcpy(v.gtab[a], gt.data(), sizeof(int2) * gt.size(), cudaMemcpyHostToDevice),
               "gather tables");
    }
    v.vpart_bytes = (size_t)v.ntiles * vol * es;
    TRY(alloc(&v.vpart, v.vpart_bytes, "workspace"));
    TRY(alloc(&v.u_stage, (size_t)h->Ntot * es, "staging"));
    TRY(alloc(&v.u_stage2, (size_t)h->Ntot * es, "staging"));
    TRY(alloc(&v.v_stage, (size_t)h->Ntot * es, "staging"));
    TRY_CUDA(v.k.prepare(), "kernel attributes");
    if (!v.on_the_fly) g.out[g.nout++] = v.L;
  }
  // geometry factors (the FP64 control points stay on the device for igasf_quad_points)
  double *coef_d = nullptr;
  unsigned int *bad_d = nullptr;
  TRY(alloc((void **)&h->ctrl64, sizeof(double) * h->Ntot * d, "control points"));
  double *ctrl_d = h->ctrl64;
  auto cleanup_tmp = [&]() {
    cudaFree(coef_d);
    cudaFree(bad_d);
  };
  cudaError_t ce = cudaMemcpy(ctrl_d, ctrl, sizeof(double) * h->Ntot * d, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess && c.kind == IGASF_COEF_VALUES) {
    // the caller's values belong to the non-empty spans' points
    std::vector<double> full;
    const double *src = c.values;
    if (h->empty_spans) {
      full.resize((size_t)h->Qtot);
      expand_qp(h, c.values, full.data(), 1);
      src = full.data();
    }
    ce = cudaMalloc((void **)&coef_d, sizeof(double) * h->Qtot);
    if (ce == cudaSuccess) ce = cudaMemcpy(coef_d, src, sizeof(double) * h->Qtot, cudaMemcpyHostToDevice);
  }
  if (ce == cudaSuccess) ce = cudaMalloc((void **)&bad_d, sizeof(unsigned int));
  if (ce == cudaSuccess) ce = cudaMemset(bad_d, 0, sizeof(unsigned int));
  if (ce != cudaSuccess) {
    cleanup_tmp();
    int rc = cuda_fail(ce, "geometry inputs");
    free_plan(h);
    return rc;
  }
  g.d = d;
  g.p = p;
  for (int a = 0; a < kMaxDim; ++a) {
    g.N[a] = h->N[a];
    g.K[a] = h->K[a];
    g.tabB[a] = h->tabB[a];
    g.tabD[a] = h->tabD[a];
    g.wq[a] = h->weights[a];
  }
  g.ctrl = ctrl_d;
  g.coef_kind = c.kind;
  g.coef_const = c.constant;
  g.coef_alpha = c.alpha;
  g.coef_values = coef_d;
  g.bad_det = bad_d;
  ce = launch_geometry(g, s);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  unsigned int bad = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(&bad, bad_d, sizeof(bad), cudaMemcpyDeviceToHost);
  cleanup_tmp();
  if (ce != cudaSuccess) {
    int rc = cuda_fail(ce, "geometry kernel");
    free_plan(h);
    return rc;
  }
  if (bad) {
    const int rc = fail(IGASF_ERR_GEOMETRY, "det J <= 0 at some quadrature point: G is not orientation preserving");
    free_plan(h);
    return rc;
  }
  // locate the static scratch of igasf_apply_noalloc on this device now, so
  // that its first call allocates nothing (noalloc.cu)
  noalloc_prepare(h->device);
  *out = h;
  return IGASF_OK;
}

int igasf_setup(int d, const int *orders, const int *knot_lengths, const double *const *knots,
                const double *ctrl, const igasf_coef *coef, const igasf_options *opt,
                igasf_handle *out) {
  igasf_plan *created = nullptr;
  try {
    return setup_impl(d, orders, knot_lengths, knots, ctrl, coef, opt, out, &created);
  } catch (const std::bad_alloc &) {
    if (created) free_plan(created);
    return fail(IGASF_ERR_OOM, "host allocation failed during setup");
  } catch (...) {
    if (created) free_plan(created);
    return fail(IGASF_ERR_INVALID_ARG, "unexpected host exception during setup");
  }
}

int igasf_apply_prec(igasf_handle h, int op, int prec, const void *u, void *v, void *stream) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return fail(IGASF_ERR_INVALID_ARG, "op = %d", op);
  if (prec < 0 || prec >= kNumPrec) return fail(IGASF_ERR_INVALID_ARG, "prec = %d", prec);
  Variant &var = h->var[prec];
  if (!var.present) return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  if (!u || !v) return fail(IGASF_ERR_INVALID_ARG, "u and v must be non-NULL");
  const size_t es = prec_size(prec);
  if (((uintptr_t)u % es) || ((uintptr_t)v % es))
    return fail(IGASF_ERR_INVALID_ARG, "u and v must be aligned to %zu bytes", es);
  const uintptr_t ub = (uintptr_t)u, vb = (uintptr_t)v, len = (uintptr_t)h->Ntot * es;
  if (ub < vb + len && vb < ub + len) return fail(IGASF_ERR_INVALID_ARG, "u and v overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ApplyParams prm;
  make_apply_params(h, var, op, u, var.vpart, &prm);
  cudaEvent_t *ev = nullptr;
  if ((size_t)(h->prof_next + 1) * 3 <= h->prof_events.size()) {
    ev = &h->prof_events[(size_t)h->prof_next * 3];
    ++h->prof_next;
    cudaEventRecord(ev[0], s);
  }
  cudaError_t e = var.k.launch[op](prm, s);
  if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
  if (ev) cudaEventRecord(ev[1], s);
  e = launch_gather(h->d, vectors_are_float(prec), var.vpart, v, h->N, var.T, var.k.S, h->p, var.gtab, s);
  if (e != cudaSuccess) return cuda_fail(e, "gather kernel launch");
  if (ev) cudaEventRecord(ev[2], s);
  return IGASF_OK;
}

int igasf_apply(igasf_handle h, int op, const void *u, void *v, void *stream) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  return igasf_apply_prec(h, op, h->default_prec, u, v, stream);
}

int igasf_apply_host(igasf_handle h, int op, int prec, const void *u_host, void *v_host,
                     void *stream) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (prec < 0 || prec >= kNumPrec || !h->var[prec].present)
    return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  if (!u_host || !v_host) return fail(IGASF_ERR_INVALID_ARG, "u and v must be non-NULL");
  Variant &var = h->var[prec];
  const size_t bytes = (size_t)h->Ntot * prec_size(prec);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(var.u_stage, u_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy u to the device");
  // A page-locked v (cudaHostAlloc / cudaHostRegister) is written by the
  // gather directly through its device mapping: no staging copy back.
  cudaPointerAttributes at;
  void *v_dev = nullptr;
  if (cudaPointerGetAttributes(&at, v_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr && ((uintptr_t)at.devicePointer % prec_size(prec)) == 0)
    v_dev = at.devicePointer;
  cudaGetLastError();   // a pageable pointer may leave an error from the attribute query
  int rc = igasf_apply_prec(h, op, prec, var.u_stage, v_dev ? v_dev : var.v_stage, stream);
  if (rc != IGASF_OK) return rc;
  if (!v_dev) {
    e = cudaMemcpyAsync(v_host, var.v_stage, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy v to the host");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return IGASF_OK;
}

int igasf_apply_host_async(igasf_handle h, int op, int prec, const void *u_host, void *v_host,
                           void *stream) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (prec < 0 || prec >= kNumPrec || !h->var[prec].present)
    return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  if (!u_host || !v_host) return fail(IGASF_ERR_INVALID_ARG, "u and v must be non-NULL");
  Variant &var = h->var[prec];
  const size_t bytes = (size_t)h->Ntot * prec_size(prec);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int b = h->stage_next;
  void *ub = b ? var.u_stage2 : var.u_stage;
  // the copy into buffer b waits for the apply that last read it (two calls ago),
  // runs on the copy stream (overlapping the previous call's apply), and the apply
  // waits for the copy
  cudaError_t e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ub, u_host, bytes, cudaMemcpyHostToDevice, h->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[b], h->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_copied[b], 0);
  if (e != cudaSuccess) return cuda_fail(e, "copy u to the device");
  cudaPointerAttributes at;
  void *v_dev = nullptr;
  if (cudaPointerGetAttributes(&at, v_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr && ((uintptr_t)at.devicePointer % prec_size(prec)) == 0)
    v_dev = at.devicePointer;
  cudaGetLastError();   // a pageable pointer may leave an error from the attribute query
  int rc = igasf_apply_prec(h, op, prec, ub, v_dev ? v_dev : var.v_stage, stream);
  if (rc != IGASF_OK) return rc;
  e = cudaEventRecord(h->ev_free[b], s);
  if (e == cudaSuccess && !v_dev) e = cudaMemcpyAsync(v_host, var.v_stage, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "order the host-buffer apply");
  h->stage_next = b ^ 1;
  return IGASF_OK;
}

int igasf_destroy(igasf_handle h) {
  if (!h) return IGASF_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(h);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize before destroy");
  return IGASF_OK;
}

int igasf_profile_begin(igasf_handle h, int max_applies) {
  if (!h || max_applies < 1) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL or max_applies < 1");
  destroy_events(h);
  try {
    h->prof_events.reserve((size_t)max_applies * 3);
  } catch (...) {
    return fail(IGASF_ERR_OOM, "host allocation");
  }
  for (int i = 0; i < max_applies * 3; ++i) {
    cudaEvent_t e;
    cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) {
      destroy_events(h);
      return cuda_fail(ce, "cudaEventCreate");
    }
    h->prof_events.push_back(e);
  }
  return IGASF_OK;
}

int igasf_profile_end(igasf_handle h, double *ms, int *applies) {
  if (!h || !ms) return fail(IGASF_ERR_INVALID_ARG, "handle or ms is NULL");
  double sum[2] = {0.0, 0.0};
  const int n = h->prof_next;
  for (int i = 0; i < n; ++i) {
    cudaEvent_t *ev = &h->prof_events[(size_t)i * 3];
    cudaError_t ce = cudaEventSynchronize(ev[2]);
    float a = 0.f, b = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&b, ev[1], ev[2]);
    if (ce != cudaSuccess) {
      destroy_events(h);
      return cuda_fail(ce, "profile events");
    }
    sum[0] += a;
    sum[1] += b;
  }
  ms[0] = sum[0];
  ms[1] = sum[1];
  if (applies) *applies = n;
  destroy_events(h);
  return IGASF_OK;
}

int igasf_device_status(igasf_handle h, int clear) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  unsigned int st = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear && st) e = cudaMemset(h->status, 0, sizeof(st));
  if (e != cudaSuccess) return cuda_fail(e, "read the device status word");
  if (st) return fail(IGASF_ERR_TIMEOUT, "a bounded device wait ran out: results since the last clear are invalid");
  return IGASF_OK;
}

int igasf_set_test_fault(igasf_handle h, int skip_slab, long long wait_limit_cycles) {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (wait_limit_cycles < 1000) return fail(IGASF_ERR_INVALID_ARG, "wait limit below 1000 cycles");
  h->skip_slab = skip_slab;
  h->wait_limit = wait_limit_cycles;
  return IGASF_OK;
}

int64_t igasf_num_dofs(igasf_handle h) { return h ? h->Ntot : -1; }

int64_t igasf_num_quad_points(igasf_handle h) { return h ? h->Qapi : -1; }

int igasf_describe(igasf_handle h, int prec, igasf_plan_desc *out) {
  if (!h || !out) return fail(IGASF_ERR_INVALID_ARG, "handle or out is NULL");
  if (prec < 0 || prec >= kNumPrec || !h->var[prec].present)
    return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  const Variant &v = h->var[prec];
  memset(out, 0, sizeof(*out));
  out->d = h->d;
  out->order = h->p;
  for (int a = 0; a < kMaxDim; ++a) {
    out->tile[a] = a < h->d ? v.k.S[a] : 1;
    out->tiles[a] = v.T[a];
  }
  out->threads_per_block = v.k.threads;
  out->kernel_variant = v.k.variant;
  out->num_dofs = h->Ntot;
  out->num_quad_points = h->Qapi;
  out->factor_bytes[IGASF_MASS] = (int64_t)v.bytesM;
  out->factor_bytes[IGASF_STIFFNESS] = (int64_t)v.bytesK;
  out->workspace_bytes = (int64_t)v.vpart_bytes;
  out->smem_bytes[0] = v.k.smem[0];
  out->smem_bytes[1] = v.k.smem[1];
  return IGASF_OK;
}

int igasf_get_tables(igasf_handle h, int dir, double *nodes, double *weights, double *B,
                     double *dB) try {
  if (!h) return fail(IGASF_ERR_INVALID_ARG, "handle is NULL");
  if (dir < 0 || dir >= h->d) return fail(IGASF_ERR_INVALID_ARG, "dir = %d", dir);
  // output: the non-empty spans' points, i.e. full point elem[i] p + g for API point i p + g
  const int Q = h->Q[dir], p = h->p, Qe = h->Ke[dir] * p;
  auto full_q = [&](int q) { return h->elem[dir][q / p] * p + q % p; };
  cudaError_t e = cudaSuccess;
  std::vector<double> tmp((size_t)Q * p);
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    double *dst = which ? weights : nodes;
    if (!dst) continue;
    e = cudaMemcpy(tmp.data(), which ? h->weights[dir] : h->nodes[dir], sizeof(double) * Q,
                   cudaMemcpyDeviceToHost);
    for (int q = 0; q < Qe && e == cudaSuccess; ++q) dst[q] = tmp[full_q(q)];
  }
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    double *dst = which ? dB : B;
    if (!dst) continue;
    e = cudaMemcpy(tmp.data(), which ? h->tabD[dir] : h->tabB[dir], sizeof(double) * Q * p,
                   cudaMemcpyDeviceToHost);
    for (int q = 0; q < Qe && e == cudaSuccess; ++q)
      for (int j = 0; j < p; ++j) dst[(size_t)q * p + j] = tmp[(size_t)j * Q + full_q(q)];
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy tables");
  return IGASF_OK;
} IGASF_CATCH_HOST

int igasf_quad_points(igasf_handle h, double *xyz_host) try {
  if (!h || !xyz_host) return fail(IGASF_ERR_INVALID_ARG, "handle or xyz_host is NULL");
  GeometryParams g;
  memset(&g, 0, sizeof(g));
  g.d = h->d;
  g.p = h->p;
  for (int a = 0; a < kMaxDim; ++a) {
    g.N[a] = h->N[a];
    g.K[a] = h->K[a];
    g.tabB[a] = h->tabB[a];
    g.tabD[a] = h->tabD[a];
    g.wq[a] = h->weights[a];
  }
  g.ctrl = h->ctrl64;
  g.coef_kind = IGASF_COEF_CONSTANT;   // points only: no factor is written (nout = 0)
  g.coef_const = 1.0;
  g.nout = 0;
  const size_t bytes = sizeof(double) * (size_t)h->Qtot * h->d;
  // host buffer first: nothing on the device is left behind if it cannot be had
  std::vector<double> full(h->empty_spans ? (size_t)h->Qtot * h->d : 0);
  double *tmp = nullptr;
  unsigned int *bad = nullptr;
  cudaError_t e = cudaMalloc((void **)&tmp, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&bad, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(unsigned int));
  if (e == cudaSuccess) {
    g.bad_det = bad;
    g.xq_out = tmp;
    e = launch_geometry(g, nullptr);
  }
  if (e == cudaSuccess) {
    if (h->empty_spans) {
      e = cudaMemcpy(full.data(), tmp, bytes, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) compact_qp(h, full.data(), xyz_host, h->d);
    } else {
      e = cudaMemcpy(xyz_host, tmp, bytes, cudaMemcpyDeviceToHost);
    }
  }
  cudaFree(tmp);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "quadrature points");
  return IGASF_OK;
} IGASF_CATCH_HOST

int igasf_get_factors(igasf_handle h, int op, int prec, double *out) try {
  if (!h || !out) return fail(IGASF_ERR_INVALID_ARG, "handle or out is NULL");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return fail(IGASF_ERR_INVALID_ARG, "op = %d", op);
  if (prec < 0 || prec >= kNumPrec || !h->var[prec].present)
    return fail(IGASF_ERR_UNSUPPORTED, "precision %d was not stored at setup", prec);
  if (h->var[prec].on_the_fly)
    return fail(IGASF_ERR_UNSUPPORTED, "precision %d evaluates its factors on the fly: none are stored", prec);
  const int nf = num_fields(h->d, op);
  const size_t bytes = sizeof(double) * (size_t)h->Qtot * nf;
  std::vector<double> full(h->empty_spans ? (size_t)h->Qtot * nf : 0);   // host buffer first
  double *tmp = nullptr;
  cudaError_t e = cudaMalloc((void **)&tmp, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "export buffer");
  e = launch_export_factors(h->var[prec].L, op, h->Qtot, h->Q, tmp, nullptr);
  if (e == cudaSuccess) {
    if (h->empty_spans) {
      e = cudaMemcpy(full.data(), tmp, bytes, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) compact_qp(h, full.data(), out, nf);
    } else {
      e = cudaMemcpy(out, tmp, bytes, cudaMemcpyDeviceToHost);
    }
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "export factors");
  return IGASF_OK;
} IGASF_CATCH_HOST

}  // extern "C"
