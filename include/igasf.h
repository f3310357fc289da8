/*
 * igasf: matrix-free, sum-factorized isogeometric mass and stiffness operators
 * on one GB300 (sm_103a).
 *
 * The operator is the quadrature approximation of the bilinear form
 * (Sec. 2, eq. quadrature:1):
 *
 *     A_mn = sum_{x in X} w(x) F(x) d^theta phi_n(x) d^eta phi_m(x)
 *
 * for tensor-product B-splines phi_n of order p (degree + 1) on open knot
 * vectors, Gauss quadrature with p points per element per direction
 * (Example gauss), and the pull-back coefficient of Example 1 (eq. cdr:1)
 * for a geometry map G = sum_n c_n phi_n (Sec. 6.2):
 *
 *     mass       (theta = eta = 0):  F = |det J|
 *     stiffness  (|theta|=|eta|=1):  F = a(G(x)) |det J| J^-1 J^-T,
 *                                    J_ij = dG_i / dxi_j.
 *
 * v = A u is applied without forming A, by the matrix-free sum factorization
 * of Alg. 2 and Alg. 3 (d directional sweeps dofs -> quadrature points, the
 * pointwise product with the precomputed factors w F, and d transposed sweeps
 * back), localized to macro-element tiles as in Sec. 4 (eq. loc-basis-change:
 * A = sum_D S_D^T A_D S_D).
 *
 * Conventions for every entry point:
 *   - Dofs are lexicographic with the first index fastest (Sec. 3.1, the
 *     ordering pi): n = n_1 + N_1 (n_2 + N_2 n_3). Quadrature points likewise.
 *   - Return value: IGASF_OK (0) or a negative igasf_status. On error
 *     igasf_last_error_message() describes it (per host thread).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Device pointers are plain CUDA device addresses on the device
 *     that was current when igasf_setup ran; that device must be current for
 *     every later call on the handle.
 *   - A handle may be used from one host thread / one stream at a time.
 */
#ifndef IGASF_H
#define IGASF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IGASF_VERSION 1
#define IGASF_MAX_DIM 3
/* Orders the CUDA kernels are built for: 2 <= p <= IGASF_MAX_ORDER. */
#define IGASF_MAX_ORDER 9

typedef enum {
  IGASF_OK = 0,
  IGASF_ERR_INVALID_ARG = -1, /* null/misaligned pointer, bad enum or size */
  IGASF_ERR_KNOTS = -2,       /* knot vector not open, decreasing, or too short */
  IGASF_ERR_GEOMETRY = -3,    /* det J <= 0 at some quadrature point */
  IGASF_ERR_UNSUPPORTED = -4, /* valid input the GPU path does not handle */
  IGASF_ERR_CUDA = -5,        /* a CUDA runtime call or kernel launch failed */
  IGASF_ERR_OOM = -6,         /* device or host allocation failed */
  IGASF_ERR_TIMEOUT = -7      /* a bounded device wait gave up */
} igasf_status;
/* Every call reports failures through these codes (and igasf_last_error_message);
 * no C++ exception leaves the library. */

typedef enum { IGASF_MASS = 0, IGASF_STIFFNESS = 1 } igasf_op;

/* Arithmetic of an apply. The factors w F are always computed in FP64 at
 * setup (Sec. 6.2); a precision says how they are stored and how the apply
 * computes.
 * FP64: FP64 factors, tables, vectors and arithmetic.
 * FP32: FP32 factors (each rounded once), tables, vectors and arithmetic.
 * BF16: factors stored in bfloat16 (each rounded once to nearest even, half
 *       the bytes of FP32); tables, vectors (u, v: float) and arithmetic FP32.
 *       The operator applied is the quadrature operator with those rounded
 *       factors: at most 2^-8 relative perturbation of every w F, meant for
 *       inner solves and preconditioners.
 * TF32: FP32 factors, tables and vectors; the direction-3 contractions (the
 *       last forward sweep and the first transposed sweep, which carry most of
 *       the multiply-adds at high order) run on the tensor cores with TF32
 *       operands (the direction-2 results, the products D grad u and the
 *       direction-3 tables rounded to 11 significant bits) and FP32
 *       accumulation; all other arithmetic FP32. 3D only.
 * BF16_MMA: factors stored in bfloat16 as for BF16; the direction-3
 *       contractions on the tensor cores with bfloat16 operands (8 significant
 *       bits) and FP32 accumulation; all other arithmetic FP32. 3D only.
 * The two tensor-core precisions keep their own factor copy (the tile shapes
 * of their kernels differ from the FP32/BF16 ones). */
typedef enum {
  IGASF_FP64 = 0,
  IGASF_FP32 = 1,
  IGASF_BF16 = 2,
  IGASF_TF32 = 3,
  IGASF_BF16_MMA = 4
} igasf_prec;
#define IGASF_PREC_BIT(prec) (1u << (unsigned)(prec))

/* Coefficient a of the stiffness operator (Example 1 with A = a I, evaluated
 * at the physical point G(x)); the mass operator ignores it. */
typedef enum {
  IGASF_COEF_CONSTANT = 0,    /* a = constant */
  IGASF_COEF_EXP_SIN_COS = 1, /* a = exp(alpha sin(2 pi x_1) cos(2 pi x_2)), cos term = 1 for d = 1 */
  IGASF_COEF_VALUES = 2       /* a given per quadrature point (host array, lexicographic) */
} igasf_coef_kind;

typedef struct {
  int kind;              /* igasf_coef_kind */
  double constant;       /* IGASF_COEF_CONSTANT */
  double alpha;          /* IGASF_COEF_EXP_SIN_COS */
  const double *values;  /* IGASF_COEF_VALUES: host, igasf_num_quad_points() values; copied */
} igasf_coef;

/* Zero-initialised = defaults. */
typedef struct {
  unsigned precisions;   /* bitmask of IGASF_PREC_BIT(prec) whose factors setup stores;
                            0 = only default_prec */
  int default_prec;      /* precision used by igasf_apply (default IGASF_FP64) */
  int tile[3];           /* elements per tile per direction, 0 = the library's choice;
                            honoured only where a kernel is built for that shape */
  int kernel_variant;    /* IGASF_KERNEL_*, 0 = the library's choice */
  int geometry;          /* IGASF_GEOMETRY_*, 0 = stored factors */
  int deterministic;     /* 0 (default) or 1: applies are bitwise reproducible from run to
                            run. This is the only mode built: the gather sums the <= 2^d tile
                            contributions of each dof in a fixed order and no kernel uses
                            floating-point atomics. Other values: IGASF_ERR_INVALID_ARG */
  int reserved[5];       /* must be zero */
} igasf_options;

/* Where the FP32 apply gets the factors w F.
 * STORED: computed once at setup (FP64, Sec. 6.2) and streamed from HBM.
 * ON_THE_FLY: the FP32 3D tile kernel evaluates them itself at every apply
 *   from the control points (Sec. 6.2: G and its derivatives by the same
 *   sum factorization as u, then det J, the cofactors of J and the
 *   coefficient at G(x)), in FP32; no FP32 factors are stored and the apply
 *   reads O(N) bytes instead of O(p^3 N). Requires d = 3, FP32 among the
 *   stored precisions and a constant or exp-sin-cos coefficient. FP64 and
 *   BF16 stay stored. */
enum { IGASF_GEOMETRY_STORED = 0, IGASF_GEOMETRY_ON_THE_FLY = 1 };

/* How the FP32 and BF16 3D tile kernels receive their factors (FP64 and 2D
 * kernels have one scheme: per-thread loads), and which family a kernel is. */
enum {
  IGASF_KERNEL_DEFAULT = 0,
  IGASF_KERNEL_REGISTERS = 1, /* each thread loads its factors into registers, slabs ahead */
  IGASF_KERNEL_RING = 2,      /* bulk copies into a shared-memory ring by a producer warp */
  IGASF_KERNEL_ON_THE_FLY = 3, /* reported by igasf_describe for IGASF_GEOMETRY_ON_THE_FLY */
  IGASF_KERNEL_MMA = 4        /* direction-3 sweeps on the tensor cores: the kernels of
                                 IGASF_TF32 and IGASF_BF16_MMA (per-thread factor loads) */
};

typedef struct igasf_plan *igasf_handle;

/* Static description of a plan for one precision. */
typedef struct {
  int d, order;
  int tile[3];              /* elements per tile per direction (1 in unused directions) */
  int tiles[3];             /* tiles per direction */
  int threads_per_block;
  int64_t num_dofs;
  int64_t num_quad_points;
  int64_t factor_bytes[2];  /* stored factor bytes for [IGASF_MASS], [IGASF_STIFFNESS],
                               including the zero padding of ragged tiles */
  int64_t workspace_bytes;  /* per-tile partial results of v */
  size_t smem_bytes[2];     /* dynamic shared memory per block, [op] */
  int kernel_variant;       /* IGASF_KERNEL_* of the tile kernel */
} igasf_plan_desc;

/*
 * Build a plan: univariate tables (Sec. 6.1), the geometry factors w F at all
 * quadrature points (Sec. 6.2; computed in FP64 on the device by sum-factorized
 * evaluation of G and its derivatives, Alg. 3), and the workspace. Blocks until
 * the factors are computed and checked.
 *
 *   d            dimension, 2 or 3.
 *   orders       host, d ints: order p per direction (all equal, 2..IGASF_MAX_ORDER).
 *   knot_lengths host, d ints: entries of each knot vector.
 *   knots        host, d pointers to non-decreasing open knot vectors (first and
 *                last knot repeated p times, interior knots at most p - 1 times:
 *                C^(p-1-m) continuity at a knot of multiplicity m, Sec. 2). The
 *                elements are the non-empty knot spans (Sec. 3); internally the
 *                empty spans of repeated knots are kept as elements of zero
 *                weight, so that the tile kernels see the simple-knot numbering.
 *   ctrl         host, N*d doubles: control point n at ctrl[n*d .. n*d+d-1].
 *   coef         host, may be NULL (= constant 1).
 *   opt          host, may be NULL (= defaults).
 *   out          receives the handle; untouched on error.
 * All host inputs are copied; the caller may free them on return.
 * Errors: INVALID_ARG, KNOTS, GEOMETRY (det J <= 0 somewhere), UNSUPPORTED,
 * CUDA, OOM. Nothing is leaked on error.
 */
int igasf_setup(int d, const int *orders, const int *knot_lengths, const double *const *knots,
                const double *ctrl, const igasf_coef *coef, const igasf_options *opt,
                igasf_handle *out);

/*
 * v = A u on `stream` in the handle's default precision (Alg. 2 after Alg. 3,
 * localized per Sec. 4). u and v: device arrays of num_dofs values of the
 * precision's type (double for FP64, float for FP32 and BF16), aligned to it,
 * not overlapping. v is overwritten. Asynchronous: returns after enqueueing; it
 * allocates nothing and does not synchronise, so it may be captured into a CUDA
 * graph (two kernel nodes: the tile kernel, then the gather with a programmatic
 * dependency). Errors: INVALID_ARG (null or
 * misaligned pointer, bad op), UNSUPPORTED (precision not stored at setup),
 * CUDA (launch failure).
 */
int igasf_apply(igasf_handle h, int op, const void *u, void *v, void *stream);

/* As igasf_apply, with the precision given explicitly. */
int igasf_apply_prec(igasf_handle h, int op, int prec, const void *u, void *v, void *stream);

/*
 * As igasf_apply_prec with HOST arrays u and v (pinned memory gives the
 * fastest copies): copies u to the plan's device staging buffer, applies, and
 * returns the result in v, then waits for `stream`. A page-locked v (from
 * cudaHostAlloc or cudaHostRegister) is written directly by the last kernel
 * through its device mapping; any other v receives a copy from a device
 * staging buffer. The staging buffers are allocated at setup. Synchronous.
 */
int igasf_apply_host(igasf_handle h, int op, int prec, const void *u_host, void *v_host,
                     void *stream);

/*
 * As igasf_apply_host, but asynchronous, for applying the operator to a
 * sequence of host vectors: enqueues the copy of u_host to one of two device
 * input buffers (alternating from call to call) on a copy stream of the plan,
 * the apply on `stream` once that copy has landed, and the result into v_host
 * (written by the gather through the device mapping of a page-locked v_host,
 * else copied back from a staging buffer on `stream`), and returns. The copy of
 * call k + 1 runs while call k's apply executes. v_host is valid, and u_host and
 * v_host may be reused or freed, only after `stream` has been synchronised. The
 * two input buffers and the copy stream are created at setup. Errors: as
 * igasf_apply_host.
 */
int igasf_apply_host_async(igasf_handle h, int op, int prec, const void *u_host, void *v_host,
                           void *stream);

/* Synchronise the device and free everything the handle owns. NULL is a no-op. */
int igasf_destroy(igasf_handle h);

int64_t igasf_num_dofs(igasf_handle h);          /* -1 on a NULL handle */
int64_t igasf_num_quad_points(igasf_handle h);   /* p^d per element (non-empty span); -1 on a NULL handle */

/* Plan description for one stored precision. */
int igasf_describe(igasf_handle h, int prec, igasf_plan_desc *out);

/*
 * Univariate tables of direction `dir` (0-based) as computed on the device, in
 * FP64 (Sec. 6.1): nodes[Q], weights[Q], B[Q*p], dB[Q*p] with Q = K*p, K the
 * number of non-empty knot spans of the direction, where B[q*p + j] is the
 * value of the j-th function active on the element of quadrature point q
 * (function index = k - p + 1 + j for the element's span [t_k, t_k+1), 0-based
 * knots; element index + j for simple knots) and dB its derivative. Host
 * outputs; any may be NULL. Synchronous. Errors: INVALID_ARG, CUDA, OOM.
 */
int igasf_get_tables(igasf_handle h, int dir, double *nodes, double *weights, double *B,
                     double *dB);

/*
 * The stored factors w F of `op` at precision `prec`, converted to FP64, in
 * lexicographic quadrature order: mass out[q]; stiffness out[q*nf + f] with
 * nf = d(d+1)/2 upper-triangle entries in row order (11,12,13,22,23,33 or
 * 11,12,22). Host output of num_quad_points*nf doubles. Synchronous.
 * Errors: INVALID_ARG, UNSUPPORTED (precision not stored, or factors evaluated
 * on the fly), CUDA, OOM.
 */
int igasf_get_factors(igasf_handle h, int op, int prec, double *out);

/*
 * The physical quadrature points G(x_q) (Sec. 6.2: G = sum_n c_n phi_n,
 * evaluated by the same sum factorization as the factors, in FP64 on the
 * device), for callers that evaluate a coefficient on the physical domain
 * (Example 1: A lives on Omega and is pulled back through G) and pass it per
 * quadrature point with IGASF_COEF_VALUES. Host output xyz_host of
 * num_quad_points * d doubles: point q (lexicographic, first index fastest,
 * the order IGASF_COEF_VALUES expects) at xyz_host[q*d .. q*d + d - 1].
 * Synchronous; allocates a temporary device buffer of the output's size.
 * Errors: INVALID_ARG, CUDA, OOM.
 */
int igasf_quad_points(igasf_handle h, double *xyz_host);

/*
 * Per-kernel timing with CUDA events, for benchmarks. igasf_profile_begin
 * creates events for up to `max_applies` later applies on this handle; each of
 * those applies then records an event before its tile kernel, between the tile
 * kernel and the gather, and after the gather, on the apply's own stream.
 * igasf_profile_end waits for the events, returns the summed durations in
 * milliseconds (ms[0] tile kernel, ms[1] gather) and the number of applies
 * timed, and destroys the events. Applies beyond max_applies are not timed.
 * Errors: INVALID_ARG, CUDA, OOM.
 */
int igasf_profile_begin(igasf_handle h, int max_applies);
int igasf_profile_end(igasf_handle h, double *ms, int *applies);

/*
 * Device status of the plan. Kernels that wait on shared-memory barriers (the
 * FP32/BF16 3D tile kernels whose factor stream arrives by bulk copies) bound every
 * wait by a clock-cycle limit; a wait that runs out sets a status word on the
 * device and the kernel finishes without hanging, but its result is invalid.
 * This call waits for the device, then returns IGASF_ERR_TIMEOUT if the word is
 * set (and clears it if `clear` is non-zero), IGASF_OK otherwise.
 */
int igasf_device_status(igasf_handle h, int clear);

/*
 * Test hook for the bounded waits: from now on, in every FP32/BF16 3D apply on
 * this handle whose tile kernel streams its factors by bulk copies
 * (IGASF_KERNEL_RING), tile 0 never receives factor slab `skip_slab` nor any
 * later slab (its producer stops issuing copies there, after waiting for the
 * ones already issued; -1 turns this off), and every wait gives up after
 * `wait_limit_cycles` clock cycles (default 2e9, about one second; minimum
 * 1000). Results of applies made while slabs are withheld are invalid.
 * Errors: INVALID_ARG.
 */
int igasf_set_test_fault(igasf_handle h, int skip_slab, long long wait_limit_cycles);

/*
 * No counterpart in the paper: a deployment variant of igasf_apply_prec for
 * callers that must not allocate device memory when they apply the operator,
 * for instance code that hands all device memory to its own arena and forbids
 * further cudaMalloc/cudaFree calls (both can synchronize the whole device).
 *
 * It computes the same v = A u with the same kernels, in the same order, so
 * its result equals igasf_apply_prec's bit for bit; but its per-tile scratch
 * (the partial results that the gather sums) lives in one static device array
 * of IGASF_NOALLOC_SCRATCH_BYTES instead of the plan's own workspace, and it
 * allocates nothing. The array is reserved on a device when the library's
 * module holding it is loaded there, which igasf_setup forces (it looks the
 * array's device address up for the plan's device and caches it), and stays
 * reserved until the process exits. Plans whose scratch need exceeds that
 * size (igasf_describe().workspace_bytes) are rejected with
 * IGASF_ERR_UNSUPPORTED; a call with another device current than the plan's
 * is rejected with IGASF_ERR_INVALID_ARG. All calls on a device share the
 * array: calls whose kernels may run at the same time on the GPU race and
 * give wrong results, so order them (one stream). The array keeps the last
 * call's contents; nothing in it needs to start at zero. Arguments, ordering
 * and other errors are those of igasf_apply_prec.
 */
#define IGASF_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int igasf_apply_noalloc(igasf_handle h, int op, int prec, const void *u, void *v, void *stream);

/* Outcome of igasf_cg_solve. */
typedef struct {
  int converged;             /* 1 if ||b - K x|| <= rtol ||b|| was reached */
  int outer_iterations;      /* FP64 residual evaluations r = b - K x */
  int inner_iterations;      /* preconditioned CG iterations, all precisions */
  double final_relres;       /* ||b - K x|| / ||b|| over the interior dofs, FP64 */
  double seconds;            /* wall time of the solve, device synchronised */
} igasf_cg_report;

/*
 * Jacobi-preconditioned conjugate gradients for K u = b with homogeneous
 * Dirichlet conditions: the unknowns are the interior dofs (index 1..N_a - 2 in
 * every direction; on open knot vectors only the first and last function of a
 * direction are non-zero on the boundary), boundary dofs are held at zero. The
 * operator is applied matrix-free (the paper's motivation for matrix-free
 * application, Sec. 3.3 and Sec. 8: iterative solvers need only v = A u).
 *
 *   inner_prec = IGASF_FP64: PCG in FP64 (FP64 apply) until ||r|| <= rtol ||b||.
 *   inner_prec = IGASF_FP32: iterative refinement. Outer loop in FP64:
 *     r = b - K x with the FP64 apply; inner PCG on K d = r with the FP32 apply,
 *     FP32 vectors and FP64 dot products, to ||r_inner|| <= inner_rtol ||r||;
 *     x += d. Stops when the FP64 residual satisfies ||r|| <= rtol ||b||.
 *   inner_prec = IGASF_BF16: the same refinement with the BF16 apply inside
 *     (factors in bfloat16: the inner operator differs from K by about 2^-9
 *     relative, which the FP64 outer residual corrects; more outer steps,
 *     cheaper inner iterations).
 * The Jacobi diagonal of K is computed on the device in FP64 at the first call
 * and kept in the plan.
 *
 * b, x: device arrays of num_dofs doubles (boundary entries of b are ignored);
 * x is overwritten (the solve starts from zero). The plan must store FP64 (and
 * inner_prec for the refined solve). max_iterations bounds the total inner
 * iterations. Synchronous; allocates its vectors for the duration of the call.
 * report may be NULL. Errors: INVALID_ARG, UNSUPPORTED (d != 3 or a missing
 * precision), CUDA, OOM. Not converging is not an error: see report->converged.
 */
int igasf_cg_solve(igasf_handle h, int inner_prec, const double *b, double *x, double rtol,
                   double inner_rtol, int max_iterations, igasf_cg_report *report, void *stream);

/*
 * Many independent 3D patches applied together (the multipatch setting of
 * Sec. 4, Example multipatch, with the patches kept independent: no interface
 * gluing). igasf_batch_create takes already set-up plans (which must outlive
 * the batch and must not be applied on their own while a batch apply may be
 * running: they share their workspace with it), groups them by tile kernel
 * (order, tile shape, factor-stream variant) and captures one launch per group
 * plus one gather for all patches into a CUDA graph. igasf_batch_apply then
 * applies every patch's operator `op` in precision `prec` with one graph
 * launch on `stream`:
 *   u, v: device arrays holding the patches' vectors back to back in plan
 *         order (patch i starts at the sum of num_dofs of patches 0..i-1),
 *         element type of `prec`, not overlapping. v is overwritten.
 * The first apply with a given (u, v), and every change of them, uploads the
 * per-patch pointer tables (a short synchronous copy). Results equal the
 * patches' individual applies bit for bit. Errors: INVALID_ARG, UNSUPPORTED
 * (a plan lacks `prec`, or is 2D), CUDA, OOM. igasf_batch_info reports 1 launch
 * group for the persistent schedule.
 */
typedef struct igasf_batch_s *igasf_batch;
int igasf_batch_create(int nplans, const igasf_handle *plans, int op, int prec, igasf_batch *out);

/*
 * As igasf_batch_create with a choice of schedule:
 *   IGASF_BATCH_GRAPH: the graph of one launch per tile kernel described above
 *     (what igasf_batch_create builds);
 *   IGASF_BATCH_PERSISTENT: one persistent launch (as many blocks as fit on the
 *     GPU) whose blocks walk a work list of every patch's tiles, highest order
 *     first, then the gather, captured as one graph. It runs FP32 or BF16 3D
 *     plans of order 2..6 set up with the persistent tile shape of their order
 *     (igasf_batch_persistent_tile; pass it as options.tile), other plans give
 *     IGASF_ERR_UNSUPPORTED. Each tile runs the register-prefetch kernel's
 *     arithmetic: results equal the individual applies of plans set up with
 *     that variant (options.kernel_variant = IGASF_KERNEL_REGISTERS) bit for
 *     bit.
 */
enum { IGASF_BATCH_GRAPH = 0, IGASF_BATCH_PERSISTENT = 1 };
int igasf_batch_create_ex(int nplans, const igasf_handle *plans, int op, int prec, int schedule,
                          igasf_batch *out);
/* The tile shape (3 ints) the persistent schedule runs for order p in precision
 * prec; IGASF_ERR_UNSUPPORTED if it runs none. Host-only. */
int igasf_batch_persistent_tile(int p, int prec, int *tile);
int igasf_batch_apply(igasf_batch b, const void *u, void *v, void *stream);
int igasf_batch_info(igasf_batch b, int64_t *total_dofs, int64_t *total_quad_points,
                     int64_t *factor_bytes, int *launch_groups);
int igasf_batch_destroy(igasf_batch b);

/*
 * Tile autotuner: sets the given patch up with every compiled (tile shape,
 * factor-stream variant) candidate of its order for `prec`, times `repeats`
 * applies of `op` of each with CUDA events (after two warm-up applies), and
 * returns the fastest candidate in tile[3] (1 in unused directions) and
 * *kernel_variant, and its time per apply in *best_ms (may be NULL). Patch
 * arguments as for igasf_setup. Synchronous; allocates temporarily.
 */
int igasf_autotune(int d, const int *orders, const int *knot_lengths, const double *const *knots,
                   const double *ctrl, const igasf_coef *coef, int op, int prec, int repeats,
                   int *tile, int *kernel_variant, double *best_ms);

/*
 * The compiled tile-kernel candidates of (d, p, prec) for the given geometry
 * mode (IGASF_GEOMETRY_STORED or IGASF_GEOMETRY_ON_THE_FLY, the latter FP32
 * and d = 3 only), in the order igasf_setup tries them (the first is the
 * default). Writes, for candidate i < max_out, its tile shape to
 * tiles[3 i .. 3 i + 2] (1 in unused directions) and its IGASF_KERNEL_* to
 * variants[i]; either array may be NULL to only count. Each candidate is
 * selected by passing that tile and variant in igasf_options. Host-only: no
 * device is touched. Returns the number of candidates (0 when none is built
 * for the combination), or a negative status for an invalid argument.
 */
int igasf_list_kernels(int d, int p, int prec, int geometry, int *tiles, int *variants, int max_out);

/*
 * Number of stored entries of the assembled matrix: the pairs (m, n) whose
 * functions share a non-empty element in every direction, which for simple
 * interior knots is prod_a ((2p - 1) K_a + (p - 1)^2) (Sec. 3.2, Corollary on
 * nnz of B-spline matrices). Returns a negative status on error.
 */
int64_t igasf_assembled_nnz(igasf_handle h);

/*
 * Assembles the matrix of `op` (the quadrature operator itself, eq.
 * quadrature:1) in FP64 CSR on the device by sum factorization over the whole
 * patch (Sec. 3, Alg. 1: the sums over the quadrature points of direction 1,
 * then 2, then d are carried out one direction at a time, with the partial
 * results of each level kept for all pairs of the later directions).
 * Intermediate levels are processed in chunks of element layers along the
 * last direction, so that they stay within `workspace_limit_bytes` of device
 * memory (0 = 2 GiB); every chunk adds to the values in a fixed order, so the
 * result is bitwise reproducible.
 *
 *   rowptr  device, num_dofs + 1 int64 (rowptr[0] = 0)
 *   colind  device, nnz int64, ascending within each row (lexicographic dof
 *           numbering, first index fastest)
 *   values  device, nnz doubles
 * nnz = igasf_assembled_nnz(h); the arrays are caller-owned, 8-byte aligned.
 * Uses the plan's FP64 factors w F (the plan must store FP64). Synchronous on
 * `stream`; allocates its workspace for the duration of the call. Errors:
 * INVALID_ARG, UNSUPPORTED (FP64 not stored), CUDA, OOM.
 */
int igasf_assemble_csr(igasf_handle h, int op, int64_t *rowptr, int64_t *colind, double *values,
                       size_t workspace_limit_bytes, void *stream);

/* Message for the last error on this host thread ("" if none). */
const char *igasf_last_error_message(void);

int igasf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IGASF_H */
