// Many independent patches applied as one CUDA graph, and the tile autotuner.
//
// A batch groups its patches by tile kernel (order, tile shape, factor-stream
// variant). Each group is one launch of that kernel's batched wrapper, whose
// blocks map to (patch, tile) through device tables; one batched gather then
// sums the per-tile partial results of every patch. The launches are captured
// once into a CUDA graph, so one batch apply is one graph launch. Per-tile
// results and the gather's summation order are those of the single-patch
// apply, so a batch apply equals the patches' individual applies bit for bit.
//
// The autotuner sets a patch up with every compiled (tile, variant) candidate
// for its order and precision, times a few applies of each with CUDA events,
// and returns the fastest (the paper's macro-element shape study, Sec. 7, made
// empirical per order and patch shape).
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "igasf.h"
#include "igasf_internal.h"
#include "plan.h"

namespace igasf {

int set_error(int code, const char *msg);

namespace {

struct GatherParams {
  const void *vpart;
  void *v;
  int N0, N1, Ntot;
  int T0, T1, T2, S0, S1, S2, E0, E1, E2, vol;
  int two;                    // at most two tiles per direction contain a dof
  const int2 *g[3];           // the plan's per-direction gather tables
};

// Same arithmetic and summation order as the single-patch gather.
template <typename T>
__global__ void batched_gather_kernel(const GatherParams *gp, const int *block_patch,
                                      const int *first_block) {
  const int patch = block_patch[blockIdx.x];
  const GatherParams g = gp[patch];
  const int n = (blockIdx.x - first_block[patch]) * blockDim.x + threadIdx.x;
  if (n >= g.Ntot) return;
  const T *vpart = static_cast<const T *>(g.vpart);
  const int i0 = n % g.N0, r = n / g.N0;
  const int i1 = r % g.N1, i2 = r / g.N1;
  const int2 a0 = g.g[0][i0], a1 = g.g[1][i1], a2 = g.g[2][i2];
  const int c0 = a0.y >> 16, l0 = a0.y & 0xffff;
  const int c1 = a1.y >> 16, l1 = a1.y & 0xffff;
  const int c2 = a2.y >> 16, l2 = a2.y & 0xffff;
  T acc = T(0);
  if (g.two) {
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k2 = c >> 2, k1 = (c >> 1) & 1, k0 = c & 1;
      x[c] = T(0);
      if (k2 < c2 && k1 < c1 && k0 < c0) {
        const int64_t tile = ((int64_t)(a2.x + k2) * g.T1 + (a1.x + k1)) * g.T0 + (a0.x + k0);
        const int loc = ((l2 - k2 * g.S2) * g.E1 + (l1 - k1 * g.S1)) * g.E0 + (l0 - k0 * g.S0);
        x[c] = vpart[tile * g.vol + loc];
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += x[c];
  } else {
    for (int k2 = 0; k2 < c2; ++k2)
      for (int k1 = 0; k1 < c1; ++k1)
        for (int k0 = 0; k0 < c0; ++k0) {
          const int64_t tile = ((int64_t)(a2.x + k2) * g.T1 + (a1.x + k1)) * g.T0 + (a0.x + k0);
          const int loc = ((l2 - k2 * g.S2) * g.E1 + (l1 - k1 * g.S1)) * g.E0 + (l0 - k0 * g.S0);
          acc += vpart[tile * g.vol + loc];
        }
  }
  static_cast<T *>(g.v)[n] = acc;
}

constexpr int kGatherThreads = 256;

}  // namespace
}  // namespace igasf

struct igasf_batch_s {
  int n = 0, op = 0, prec = 0;
  std::vector<igasf_plan *> plans;
  std::vector<int64_t> offset;             // first dof of each patch in packed u, v
  int64_t total_dofs = 0, total_qp = 0, factor_bytes = 0;
  struct Group {
    igasf::ApplyKernel k{};
    std::vector<int> patches;
    int blocks = 0;
    std::vector<igasf::ApplyParams> h_params;
    igasf::ApplyParams *d_params = nullptr;
    int *d_block_patch = nullptr, *d_first_block = nullptr;
  };
  std::vector<Group> groups;
  std::vector<igasf::GatherParams> h_gp;
  igasf::GatherParams *d_gp = nullptr;
  int *d_gblock_patch = nullptr, *d_gfirst = nullptr;
  int gblocks = 0;
  // schedule IGASF_BATCH_PERSISTENT: one launch over a (patch, tile) work list
  bool persistent = false;
  std::vector<igasf::ApplyParams> p_params;  // per patch
  igasf::ApplyParams *d_pparams = nullptr;
  int *d_porder = nullptr;
  int2 *d_items = nullptr;
  int nitems = 0, pgrid = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void *last_u = nullptr;
  void *last_v = nullptr;
};

namespace {

void free_batch(igasf_batch b) {
  if (!b) return;
  for (auto &g : b->groups) {
    cudaFree(g.d_params);
    cudaFree(g.d_block_patch);
    cudaFree(g.d_first_block);
  }
  cudaFree(b->d_pparams);
  cudaFree(b->d_porder);
  cudaFree(b->d_items);
  cudaFree(b->d_gp);
  cudaFree(b->d_gblock_patch);
  cudaFree(b->d_gfirst);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

template <typename V>
cudaError_t upload(V **dst, const std::vector<V> &src) {
  cudaError_t e = cudaMalloc((void **)dst, sizeof(V) * (src.empty() ? 1 : src.size()));
  if (e == cudaSuccess && !src.empty())
    e = cudaMemcpy(*dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice);
  return e;
}

// Point the per-patch parameters at packed u and v and upload them.
cudaError_t bind_vectors(igasf_batch b, const void *u, void *v) {
  const size_t es = b->prec == IGASF_FP64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  for (auto &g : b->groups) {
    for (size_t i = 0; i < g.patches.size(); ++i)
      g.h_params[i].u = static_cast<const char *>(u) + es * b->offset[g.patches[i]];
    if (e == cudaSuccess)
      e = cudaMemcpy(g.d_params, g.h_params.data(), sizeof(igasf::ApplyParams) * g.h_params.size(),
                     cudaMemcpyHostToDevice);
  }
  if (b->persistent) {
    for (int i = 0; i < b->n; ++i) b->p_params[i].u = static_cast<const char *>(u) + es * b->offset[i];
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_pparams, b->p_params.data(), sizeof(igasf::ApplyParams) * b->n,
                     cudaMemcpyHostToDevice);
  }
  for (int i = 0; i < b->n; ++i) b->h_gp[i].v = static_cast<char *>(v) + es * b->offset[i];
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_gp, b->h_gp.data(), sizeof(igasf::GatherParams) * b->h_gp.size(),
                   cudaMemcpyHostToDevice);
  b->last_u = u;
  b->last_v = v;
  return e;
}

}  // namespace

extern "C" {

int igasf_batch_create(int nplans, const igasf_handle *plans, int op, int prec, igasf_batch *out) {
  return igasf_batch_create_ex(nplans, plans, op, prec, IGASF_BATCH_GRAPH, out);
}

// The body of igasf_batch_create_ex; *created receives the batch as soon as it
// exists (its error paths free it themselves).
static int batch_create_impl(int nplans, const igasf_handle *plans, int op, int prec, int schedule,
                             igasf_batch *out, igasf_batch *created) {
  using namespace igasf;
  if (!out || !plans || nplans < 1) return set_error(IGASF_ERR_INVALID_ARG, "need nplans >= 1, plans and out");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return set_error(IGASF_ERR_INVALID_ARG, "bad op");
  if (prec < 0 || prec >= kNumPrec) return set_error(IGASF_ERR_INVALID_ARG, "bad prec");
  if (schedule != IGASF_BATCH_GRAPH && schedule != IGASF_BATCH_PERSISTENT)
    return set_error(IGASF_ERR_INVALID_ARG, "bad schedule");
  const bool pers = schedule == IGASF_BATCH_PERSISTENT;
  for (int i = 0; i < nplans; ++i) {
    const igasf_plan *h = plans[i];
    if (!h) return set_error(IGASF_ERR_INVALID_ARG, "a plan is NULL");
    if (!h->var[prec].present) return set_error(IGASF_ERR_UNSUPPORTED, "a plan lacks the batch precision");
    if (!h->var[prec].k.launch_batched[op])
      return set_error(IGASF_ERR_UNSUPPORTED, "a plan's kernel has no batched form (2D plans)");
    if (pers) {
      int S[3];
      const ApplyKernel &k = h->var[prec].k;
      if (h->d != 3 || h->var[prec].on_the_fly || !persistent_tile(h->p, prec, S) || k.S[0] != S[0] ||
          k.S[1] != S[1] || k.S[2] != S[2])
        return set_error(IGASF_ERR_UNSUPPORTED,
                         "the persistent schedule needs FP32 or BF16 3D plans of order 2..6 set up with "
                         "the persistent tile of their order (igasf_batch_persistent_tile)");
    }
  }
  igasf_batch b = new (std::nothrow) igasf_batch_s();
  if (!b) return set_error(IGASF_ERR_OOM, "host allocation");
  *created = b;
  b->persistent = pers;
  b->n = nplans;
  b->op = op;
  b->prec = prec;
  b->plans.assign(plans, plans + nplans);
  b->offset.resize(nplans);
  b->h_gp.resize(nplans);
  int64_t off = 0;
  for (int i = 0; i < nplans; ++i) {
    igasf_plan *h = b->plans[i];
    const Variant &v = h->var[prec];
    b->offset[i] = off;
    off += h->Ntot;
    b->total_qp += h->Qapi;
    b->factor_bytes += op == IGASF_MASS ? v.bytesM : v.bytesK;
    // group by kernel
    int gi = -1;
    for (size_t g = 0; g < b->groups.size(); ++g)
      if (b->groups[g].k.launch_batched[op] == v.k.launch_batched[op]) gi = (int)g;
    if (gi < 0) {
      b->groups.emplace_back();
      gi = (int)b->groups.size() - 1;
      b->groups[gi].k = v.k;
    }
    auto &G = b->groups[gi];
    G.patches.push_back(i);
    ApplyParams prm;
    make_apply_params(h, v, op, nullptr, v.vpart, &prm);
    prm.skip_slab = -1;
    G.h_params.push_back(prm);
    if (pers) b->p_params.push_back(prm);
    GatherParams &gp = b->h_gp[i];
    gp.vpart = v.vpart;
    gp.N0 = h->N[0];
    gp.N1 = h->N[1];
    gp.Ntot = (int)h->Ntot;
    gp.T0 = v.T[0];
    gp.T1 = v.T[1];
    gp.T2 = v.T[2];
    gp.S0 = v.k.S[0];
    gp.S1 = v.k.S[1];
    gp.S2 = v.k.S[2];
    gp.E0 = gp.S0 + h->p - 1;
    gp.E1 = gp.S1 + h->p - 1;
    gp.E2 = gp.S2 + h->p - 1;
    gp.vol = gp.E0 * gp.E1 * gp.E2;
    gp.two = gp.E0 <= 2 * gp.S0 && gp.E1 <= 2 * gp.S1 && gp.E2 <= 2 * gp.S2;
    for (int a = 0; a < 3; ++a) gp.g[a] = v.gtab[a];
  }
  b->total_dofs = off;
  // device tables
  cudaError_t e = cudaSuccess;
  for (auto &G : b->groups) {
    std::vector<int> bp;
    std::vector<int> local_first(G.patches.size());
    for (size_t j = 0; j < G.patches.size(); ++j) {
      local_first[j] = (int)bp.size();
      for (int t = 0; t < G.h_params[j].ntiles; ++t) bp.push_back((int)j);
    }
    G.blocks = (int)bp.size();
    if (e == cudaSuccess) e = upload(&G.d_block_patch, bp);
    if (e == cudaSuccess) e = upload(&G.d_first_block, local_first);
    if (e == cudaSuccess) e = upload(&G.d_params, G.h_params);
  }
  {
    std::vector<int> bp, first(b->n);
    for (int i = 0; i < b->n; ++i) {
      first[i] = (int)bp.size();
      const int nb = (b->h_gp[i].Ntot + kGatherThreads - 1) / kGatherThreads;
      for (int k = 0; k < nb; ++k) bp.push_back(i);
    }
    b->gblocks = (int)bp.size();
    if (e == cudaSuccess) e = upload(&b->d_gblock_patch, bp);
    if (e == cudaSuccess) e = upload(&b->d_gfirst, first);
    if (e == cudaSuccess) e = upload(&b->d_gp, b->h_gp);
  }
  // the persistent schedule's work list: (patch, tile), highest order first
  if (e == cudaSuccess && pers) {
    std::vector<int> order(b->n);
    std::vector<int2> items;
    for (int i = 0; i < b->n; ++i) order[i] = b->plans[i]->p;
    for (int p = 9; p >= 1; --p)
      for (int i = 0; i < b->n; ++i)
        if (order[i] == p)
          for (int t = 0; t < b->p_params[i].ntiles; ++t) items.push_back(make_int2(i, t));
    b->nitems = (int)items.size();
    e = prepare_persistent(op, prec, &b->pgrid);
    if (e == cudaSuccess) e = upload(&b->d_pparams, b->p_params);
    if (e == cudaSuccess) e = upload(&b->d_porder, order);
    if (e == cudaSuccess) e = upload(&b->d_items, items);
  }
  // capture the launches into a graph
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (pers) {
      const cudaError_t le = launch_persistent(op, prec, b->d_pparams, b->d_porder, b->d_items,
                                               b->nitems, b->pgrid, b->cap);
      if (le != cudaSuccess && e == cudaSuccess) e = le;
    } else {
      for (auto &G : b->groups) {
        BatchParams bp;
        bp.params = G.d_params;
        bp.block_patch = G.d_block_patch;
        bp.first_block = G.d_first_block;
        const cudaError_t le = G.k.launch_batched[op](bp, G.blocks, b->cap);
        if (le != cudaSuccess && e == cudaSuccess) e = le;
      }
    }
    if (vectors_are_float(prec))
      batched_gather_kernel<float><<<b->gblocks, kGatherThreads, 0, b->cap>>>(b->d_gp, b->d_gblock_patch,
                                                                            b->d_gfirst);
    else
      batched_gather_kernel<double><<<b->gblocks, kGatherThreads, 0, b->cap>>>(b->d_gp, b->d_gblock_patch,
                                                                             b->d_gfirst);
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &b->graph);
    if (e == cudaSuccess) e = ce;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    // the message first (it can throw), then the batch
    const int rc = set_error(e == cudaErrorMemoryAllocation ? IGASF_ERR_OOM : IGASF_ERR_CUDA,
                             (std::string("batch set-up: ") + cudaGetErrorString(e)).c_str());
    free_batch(b);
    return rc;
  }
  *out = b;
  return IGASF_OK;
}

int igasf_batch_create_ex(int nplans, const igasf_handle *plans, int op, int prec, int schedule,
                          igasf_batch *out) {
  igasf_batch created = nullptr;
  try {
    return batch_create_impl(nplans, plans, op, prec, schedule, out, &created);
  } catch (const std::bad_alloc &) {
    if (created) free_batch(created);
    return igasf::set_error(IGASF_ERR_OOM, "host allocation failed while creating the batch");
  } catch (...) {
    if (created) free_batch(created);
    return igasf::set_error(IGASF_ERR_INVALID_ARG, "unexpected host exception while creating the batch");
  }
}

int igasf_batch_apply(igasf_batch b, const void *u, void *v, void *stream) try {
  using namespace igasf;
  if (!b || !u || !v) return set_error(IGASF_ERR_INVALID_ARG, "batch, u and v must be non-NULL");
  const size_t es = b->prec == IGASF_FP64 ? 8 : 4;
  if (((uintptr_t)u % es) || ((uintptr_t)v % es))
    return set_error(IGASF_ERR_INVALID_ARG, "u and v must be aligned to the element size");
  const uintptr_t ub = (uintptr_t)u, vb = (uintptr_t)v, len = (uintptr_t)b->total_dofs * es;
  if (ub < vb + len && vb < ub + len) return set_error(IGASF_ERR_INVALID_ARG, "u and v overlap");
  cudaError_t e = cudaSuccess;
  if (u != b->last_u || v != b->last_v) {
    e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));   // earlier launches read the old tables
    if (e == cudaSuccess) e = bind_vectors(b, u, v);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_error(IGASF_ERR_CUDA, (std::string("batch apply: ") + cudaGetErrorString(e)).c_str());
  return IGASF_OK;
} IGASF_CATCH_HOST

int igasf_batch_info(igasf_batch b, int64_t *total_dofs, int64_t *total_quad_points,
                     int64_t *factor_bytes, int *launch_groups) {
  if (!b) return igasf::set_error(IGASF_ERR_INVALID_ARG, "batch is NULL");
  if (total_dofs) *total_dofs = b->total_dofs;
  if (total_quad_points) *total_quad_points = b->total_qp;
  if (factor_bytes) *factor_bytes = b->factor_bytes;
  if (launch_groups) *launch_groups = b->persistent ? 1 : (int)b->groups.size();
  return IGASF_OK;
}

int igasf_batch_persistent_tile(int p, int prec, int *tile) {
  if (!tile) return igasf::set_error(IGASF_ERR_INVALID_ARG, "tile is NULL");
  if (!igasf::persistent_tile(p, prec, tile))
    return igasf::set_error(IGASF_ERR_UNSUPPORTED, "no persistent tile for this order and precision");
  return IGASF_OK;
}

int igasf_batch_destroy(igasf_batch b) {
  if (!b) return IGASF_OK;
  const cudaError_t e = cudaDeviceSynchronize();
  free_batch(b);
  if (e != cudaSuccess) return igasf::set_error(IGASF_ERR_CUDA, cudaGetErrorString(e));
  return IGASF_OK;
}

}  // extern "C"

extern "C" int igasf_autotune(int d, const int *orders, const int *knot_lengths,
                              const double *const *knots, const double *ctrl, const igasf_coef *coef,
                              int op, int prec, int repeats, int *tile, int *kernel_variant,
                              double *best_ms) try {
  using namespace igasf;
  if (!tile || !kernel_variant || !orders || repeats < 1)
    return set_error(IGASF_ERR_INVALID_ARG, "need orders, tile, kernel_variant and repeats >= 1");
  if (op != IGASF_MASS && op != IGASF_STIFFNESS) return set_error(IGASF_ERR_INVALID_ARG, "bad op");
  ApplyKernel cand[kMaxCandidates];
  const int nc = list_apply_kernels(d, orders[0], prec, cand, kMaxCandidates);
  if (nc < 1) return set_error(IGASF_ERR_UNSUPPORTED, "no kernel for this order and precision");
  double best = 1e300;
  int best_i = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  void *u = nullptr, *v = nullptr;
  int rc = IGASF_OK;
  for (int i = 0; i < nc && ce == cudaSuccess && rc == IGASF_OK; ++i) {
    igasf_options o;
    memset(&o, 0, sizeof(o));
    o.precisions = IGASF_PREC_BIT(prec);
    o.default_prec = prec;
    for (int a = 0; a < d; ++a) o.tile[a] = cand[i].S[a];
    o.kernel_variant = cand[i].variant;
    igasf_handle h = nullptr;
    rc = igasf_setup(d, orders, knot_lengths, knots, ctrl, coef, &o, &h);
    if (rc != IGASF_OK) break;
    const size_t bytes = (size_t)igasf_num_dofs(h) * (prec == IGASF_FP64 ? 8 : 4);
    if (!u) {
      ce = cudaMalloc(&u, bytes);
      if (ce == cudaSuccess) ce = cudaMalloc(&v, bytes);
      if (ce == cudaSuccess) ce = cudaMemset(u, 0, bytes);
    }
    for (int w = 0; w < 2 && ce == cudaSuccess && rc == IGASF_OK; ++w)
      rc = igasf_apply_prec(h, op, prec, u, v, s);   // warm-up
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
    for (int r = 0; r < repeats && ce == cudaSuccess && rc == IGASF_OK; ++r)
      rc = igasf_apply_prec(h, op, prec, u, v, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    const int drc = igasf_destroy(h);
    if (rc == IGASF_OK) rc = drc;
    if (ce == cudaSuccess && rc == IGASF_OK && ms / repeats < best) {
      best = ms / repeats;
      best_i = i;
    }
  }
  cudaFree(u);
  cudaFree(v);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (rc != IGASF_OK) return rc;
  if (ce != cudaSuccess) return set_error(IGASF_ERR_CUDA, (std::string("autotune: ") + cudaGetErrorString(ce)).c_str());
  for (int a = 0; a < 3; ++a) tile[a] = a < d ? cand[best_i].S[a] : 1;
  *kernel_variant = cand[best_i].variant;
  if (best_ms) *best_ms = best;
  return IGASF_OK;
} IGASF_CATCH_HOST
