/*
 * Plain FP64 CPU oracle for the isogeometric mass and stiffness operators.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the product path never does. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes is the plain definition of the quadrature operator
 * (Sec. 2, eq. quadrature:1 and eq. ass:0):
 *
 *     A_mn = sum_{x in X} w(x) F(x) d^theta phi_n(x) d^eta phi_m(x),
 *
 * with the pull-back coefficient of Example 1 (eq. cdr:1) for c = 1, b = 0 and
 * an isotropic diffusion A = a I:
 *     mass:      F = |det J|                      (theta = eta = 0)
 *     stiffness: F = a(G(x)) |det J| J^-1 J^-T    (|theta| = |eta| = 1)
 * where J_ij = dG_i / dxi_j and G = sum_n c_n phi_n (Sec. 6.2).
 *
 * Every entry is a direct sum over quadrature points of products of basis
 * values; there is no sum factorization, no blocking and no reordering.
 * Steps, each in the paper's notation:
 *   - elements: the non-empty knot spans of each open knot vector (Ex. gauss);
 *   - Gauss-Legendre rule with p points per element per direction (Ex. gauss),
 *     nodes by Newton's method on the three-term Legendre recurrence;
 *   - univariate B-splines by the Cox-de Boor recursion over the whole index
 *     range (Ex. 1), derivatives by the standard differentiation formula;
 *   - tensor-product basis phi_n = prod_delta phi^delta_{pi_delta(n)} with the
 *     lexicographic order pi, first index fastest (Sec. 3.1);
 *   - tensor-product quadrature X = X_1 x ... x X_d, w = prod w_delta (Sec. 3.1).
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp (OpenMP runs independent pieces on
 * several cores: the rows of the row-wise apply and assembly, the rows of the
 * CSR product, and race-free classes of element layers of the point-by-point
 * apply; no piece's arithmetic depends on the thread count).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 3
#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_KNOTS -2
#define ORC_ERR_MEM -6

enum { ORC_MASS = 0, ORC_STIFFNESS = 1 };
enum { ORC_COEF_CONSTANT = 0, ORC_COEF_EXP_SIN_COS = 1, ORC_COEF_VALUES = 2 };

/* ------------------------------------------------------------------------ */
/* Univariate pieces                                                         */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1, 1], n points, ascending.
 * Newton's method on P_n, with P_n and P_{n-1} from the recurrence
 * (k+1) P_{k+1}(x) = (2k+1) x P_k(x) - k P_{k-1}(x),
 * P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1), weight 2 / ((1 - x^2) P_n'(x)^2). */
int orc_gauss_legendre(int n, double *x, double *w) {
  if (n < 1) return ORC_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));   /* initial guess */
    double pn = 0.0, pnm1 = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      /* P_0 = 1, P_1 = z, then the recurrence up to P_n */
      pnm1 = 1.0;
      pn = z;
      for (int k = 1; k < n; ++k) {
        double next = ((2.0 * k + 1.0) * z * pn - k * pnm1) / (k + 1.0);
        pnm1 = pn;
        pn = next;
      }
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    /* derivative at the final node, for the weight */
    pnm1 = 1.0;
    pn = z;
    for (int k = 1; k < n; ++k) {
      double next = ((2.0 * k + 1.0) * z * pn - k * pnm1) / (k + 1.0);
      pnm1 = pn;
      pn = next;
    }
    dp = n * (z * pn - pnm1) / (z * z - 1.0);
    x[n - 1 - i] = z;                 /* the guesses decrease with i: store ascending */
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return ORC_OK;
}

/* All B-splines of order p on knot vector t (nk knots) at x, by the
 * Cox-de Boor recursion over the whole index range:
 *   b_{i,1}(x) = 1 if t_i <= x < t_{i+1}, else 0,
 *   b_{i,k}(x) = (x - t_i)/(t_{i+k-1} - t_i) b_{i,k-1}(x)
 *              + (t_{i+k} - x)/(t_{i+k} - t_{i+1}) b_{i+1,k-1}(x),   0/0 := 0.
 * Derivative of the order-p functions:
 *   b'_{i,p} = (p-1) [ b_{i,p-1}/(t_{i+p-1} - t_i) - b_{i+1,p-1}/(t_{i+p} - t_{i+1}) ].
 * val and der receive nk - p values. x must lie strictly inside a non-empty
 * span (Gauss nodes always do), so the half-open convention never matters.
 * cox_de_boor() leaves the order-k values of all functions in b (nk - 1 slots). */
static void cox_de_boor(const double *t, int nk, int k_order, double x, double *b, double *tmp) {
  int n1 = nk - 1;
  for (int i = 0; i < n1; ++i) b[i] = (t[i] <= x && x < t[i + 1]) ? 1.0 : 0.0;
  for (int k = 2; k <= k_order; ++k) {
    memcpy(tmp, b, sizeof(double) * (size_t)n1);
    int nfun = nk - k;             /* number of order-k functions */
    for (int i = 0; i < nfun; ++i) {
      double left = 0.0, right = 0.0;
      double dl = t[i + k - 1] - t[i];
      double dr = t[i + k] - t[i + 1];
      if (dl > 0.0) left = (x - t[i]) / dl * tmp[i];
      if (dr > 0.0) right = (t[i + k] - x) / dr * tmp[i + 1];
      b[i] = left + right;
    }
    for (int i = nfun; i < n1; ++i) b[i] = 0.0;
  }
}

int orc_bspline_all(const double *t, int nk, int p, double x, double *val, double *der) {
  if (p < 1 || nk < 2 * p) return ORC_ERR_ARG;
  int n1 = nk - 1;
  int N = nk - p;
  double *b = (double *)calloc((size_t)n1 + 1, sizeof(double));
  double *tmp = (double *)calloc((size_t)n1 + 1, sizeof(double));
  if (!b || !tmp) { free(b); free(tmp); return ORC_ERR_MEM; }
  cox_de_boor(t, nk, p, x, b, tmp);
  for (int i = 0; i < N; ++i) val[i] = b[i];
  if (der) {
    if (p == 1) {
      for (int i = 0; i < N; ++i) der[i] = 0.0;
    } else {
      cox_de_boor(t, nk, p - 1, x, b, tmp);   /* order p-1 values */
      for (int i = 0; i < N; ++i) {
        double dl = t[i + p - 1] - t[i];
        double dr = t[i + p] - t[i + 1];
        double a = (dl > 0.0) ? b[i] / dl : 0.0;
        double c = (dr > 0.0) ? b[i + 1] / dr : 0.0;
        der[i] = (p - 1) * (a - c);
      }
    }
  }
  free(b);
  free(tmp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Patch: univariate tables per direction, dense (all functions at all points) */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d;
  int p[ORC_MAXD];        /* orders */
  int nk[ORC_MAXD];       /* knot counts */
  const double *t[ORC_MAXD];
  int N[ORC_MAXD];        /* functions per direction, nk - p */
  int K[ORC_MAXD];        /* non-empty spans (elements) */
  int *span[ORC_MAXD];    /* knot index k of element e: t_k < t_{k+1} */
  int *elem_of_span[ORC_MAXD]; /* inverse map, -1 for empty spans */
  int Q[ORC_MAXD];        /* quadrature points, K * p */
  double *xq[ORC_MAXD];   /* nodes */
  double *wq[ORC_MAXD];   /* weights */
  double *B[ORC_MAXD];    /* B[q * N + n] = phi_n(x_q) */
  double *dB[ORC_MAXD];   /* derivative */
  const double *ctrl;     /* N x d */
  int coef_kind;
  double coef_const, coef_alpha;
  const double *coef_values;
  int64_t Ntot, Qtot;
} orc_patch;

static void patch_free(orc_patch *P) {
  for (int a = 0; a < ORC_MAXD; ++a) {
    free(P->span[a]); free(P->elem_of_span[a]); free(P->xq[a]); free(P->wq[a]);
    free(P->B[a]); free(P->dB[a]);
  }
}

/* knots: d vectors concatenated; nks[a] entries each */
static int patch_build(orc_patch *P, int d, const int *orders, const int *nks,
                       const double *knots, const double *ctrl, int coef_kind,
                       double coef_const, double coef_alpha, const double *coef_values) {
  memset(P, 0, sizeof(*P));
  if (d < 1 || d > ORC_MAXD) return ORC_ERR_ARG;
  P->d = d;
  P->ctrl = ctrl;
  P->coef_kind = coef_kind;
  P->coef_const = coef_const;
  P->coef_alpha = coef_alpha;
  P->coef_values = coef_values;
  const double *tp = knots;
  P->Ntot = 1;
  P->Qtot = 1;
  for (int a = 0; a < d; ++a) {
    int p = orders[a], nk = nks[a];
    if (p < 1 || nk < 2 * p) return ORC_ERR_KNOTS;
    for (int i = 0; i + 1 < nk; ++i) if (tp[i + 1] < tp[i]) return ORC_ERR_KNOTS;
    P->p[a] = p;
    P->nk[a] = nk;
    P->t[a] = tp;
    P->N[a] = nk - p;
    int K = 0;
    P->span[a] = (int *)malloc(sizeof(int) * (size_t)nk);
    P->elem_of_span[a] = (int *)malloc(sizeof(int) * (size_t)nk);
    for (int k = 0; k < nk; ++k) P->elem_of_span[a][k] = -1;
    for (int k = p - 1; k < nk - p; ++k) {
      if (tp[k + 1] > tp[k]) { P->span[a][K] = k; P->elem_of_span[a][k] = K; ++K; }
    }
    if (K == 0) return ORC_ERR_KNOTS;
    P->K[a] = K;
    P->Q[a] = K * p;
    P->xq[a] = (double *)malloc(sizeof(double) * (size_t)P->Q[a]);
    P->wq[a] = (double *)malloc(sizeof(double) * (size_t)P->Q[a]);
    P->B[a] = (double *)calloc((size_t)P->Q[a] * (size_t)P->N[a], sizeof(double));
    P->dB[a] = (double *)calloc((size_t)P->Q[a] * (size_t)P->N[a], sizeof(double));
    double *gx = (double *)malloc(sizeof(double) * (size_t)p);
    double *gw = (double *)malloc(sizeof(double) * (size_t)p);
    orc_gauss_legendre(p, gx, gw);
    for (int e = 0; e < K; ++e) {
      double lo = tp[P->span[a][e]], hi = tp[P->span[a][e] + 1];
      for (int j = 0; j < p; ++j) {
        int q = e * p + j;
        P->xq[a][q] = lo + (gx[j] + 1.0) * (hi - lo) / 2.0;
        P->wq[a][q] = gw[j] * (hi - lo) / 2.0;
        orc_bspline_all(tp, nk, p, P->xq[a][q], P->B[a] + (size_t)q * P->N[a],
                        P->dB[a] + (size_t)q * P->N[a]);
      }
    }
    free(gx);
    free(gw);
    P->Ntot *= P->N[a];
    P->Qtot *= P->Q[a];
    tp += nk;
  }
  return ORC_OK;
}

/* functions active on element e of direction a: n in [k - p + 1, k], k = span */
static int first_active(const orc_patch *P, int a, int e) { return P->span[a][e] - P->p[a] + 1; }

/* ------------------------------------------------------------------------ */
/* Geometry and coefficient at one quadrature point (Sec. 6.2, Example 1)    */
/* ------------------------------------------------------------------------ */

typedef struct {
  double w;                 /* prod_delta w_delta */
  double G[ORC_MAXD];       /* physical point */
  double J[ORC_MAXD][ORC_MAXD];
  double detJ;
  double a;                 /* coefficient a(G(x)) */
  double FM;                /* |det J| */
  double FK[ORC_MAXD][ORC_MAXD]; /* a |det J| J^-1 J^-T */
} orc_qp;

/* q[a] = per-direction quadrature index */
static void eval_qp(const orc_patch *P, const int *q, orc_qp *out) {
  int d = P->d;
  memset(out, 0, sizeof(*out));
  out->w = 1.0;
  for (int a = 0; a < d; ++a) out->w *= P->wq[a][q[a]];
  int e[ORC_MAXD], f[ORC_MAXD];
  for (int a = 0; a < d; ++a) { e[a] = q[a] / P->p[a]; f[a] = first_active(P, a, e[a]); }
  /* G = sum_n c_n phi_n, J_ij = sum_n c_{n,i} d phi_n / d xi_j, over active n */
  int cnt[ORC_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) cnt[a] = P->p[a];
  for (int j3 = 0; j3 < (d > 2 ? cnt[2] : 1); ++j3)
    for (int j2 = 0; j2 < (d > 1 ? cnt[1] : 1); ++j2)
      for (int j1 = 0; j1 < cnt[0]; ++j1) {
        int n_[ORC_MAXD] = {f[0] + j1, d > 1 ? f[1] + j2 : 0, d > 2 ? f[2] + j3 : 0};
        int64_t n = n_[0];
        if (d > 1) n += (int64_t)P->N[0] * n_[1];
        if (d > 2) n += (int64_t)P->N[0] * P->N[1] * n_[2];
        double val[ORC_MAXD], der[ORC_MAXD];
        for (int a = 0; a < d; ++a) {
          val[a] = P->B[a][(size_t)q[a] * P->N[a] + n_[a]];
          der[a] = P->dB[a][(size_t)q[a] * P->N[a] + n_[a]];
        }
        double phi = 1.0;
        for (int a = 0; a < d; ++a) phi *= val[a];
        for (int i = 0; i < d; ++i) {
          double c = P->ctrl[n * d + i];
          out->G[i] += c * phi;
          for (int j = 0; j < d; ++j) {
            double dphi = 1.0;
            for (int a = 0; a < d; ++a) dphi *= (a == j) ? der[a] : val[a];
            out->J[i][j] += c * dphi;
          }
        }
      }
  /* determinant and inverse by cofactors */
  double inv[ORC_MAXD][ORC_MAXD];
  if (d == 1) {
    out->detJ = out->J[0][0];
    inv[0][0] = 1.0 / out->detJ;
  } else if (d == 2) {
    double (*J)[ORC_MAXD] = out->J;
    out->detJ = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    inv[0][0] = J[1][1] / out->detJ;
    inv[0][1] = -J[0][1] / out->detJ;
    inv[1][0] = -J[1][0] / out->detJ;
    inv[1][1] = J[0][0] / out->detJ;
  } else {
    double (*J)[ORC_MAXD] = out->J;
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double c10 = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
    double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    double c12 = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
    double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    double c21 = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
    double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    out->detJ = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    /* inverse = transpose of the cofactor matrix / det */
    inv[0][0] = c00 / out->detJ; inv[0][1] = c10 / out->detJ; inv[0][2] = c20 / out->detJ;
    inv[1][0] = c01 / out->detJ; inv[1][1] = c11 / out->detJ; inv[1][2] = c21 / out->detJ;
    inv[2][0] = c02 / out->detJ; inv[2][1] = c12 / out->detJ; inv[2][2] = c22 / out->detJ;
  }
  /* coefficient, evaluated at the physical point G(x) */
  switch (P->coef_kind) {
    case ORC_COEF_EXP_SIN_COS:
      out->a = exp(P->coef_alpha * sin(2.0 * M_PI * out->G[0]) *
                   (d > 1 ? cos(2.0 * M_PI * out->G[1]) : 1.0));
      break;
    case ORC_COEF_VALUES: {
      int64_t qi = q[0];
      if (d > 1) qi += (int64_t)P->Q[0] * q[1];
      if (d > 2) qi += (int64_t)P->Q[0] * P->Q[1] * q[2];
      out->a = P->coef_values[qi];
      break;
    }
    default:
      out->a = P->coef_const;
  }
  double adet = fabs(out->detJ);
  out->FM = adet;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += inv[i][k] * inv[j][k];
      out->FK[i][j] = out->a * adet * s;
    }
}

/* value (deriv_dir < 0) or partial derivative d/dxi_{deriv_dir} of phi_n at
 * quadrature point q, n given by per-direction indices */
static double basis_at(const orc_patch *P, const int *q, const int *n, int deriv_dir) {
  double r = 1.0;
  for (int a = 0; a < P->d; ++a) {
    size_t o = (size_t)q[a] * P->N[a] + n[a];
    r *= (a == deriv_dir) ? P->dB[a][o] : P->B[a][o];
  }
  return r;
}

/* ------------------------------------------------------------------------ */
/* Stored factors in a narrower format                                       */
/* ------------------------------------------------------------------------ */

/* A matrix-free apply stores the weighted factors w F at every quadrature
 * point (Sec. 6.2) and may store them in a narrower floating-point format than
 * FP64. The operator it applies is then the quadrature operator whose factors
 * are the rounded values. With stored_bits > 0 the oracle computes exactly that
 * operator: each stored product (w |det J| for the mass, each entry of
 * w a |det J| J^-1 J^-T for the stiffness) is rounded to stored_bits
 * significant bits, ties to even, before it enters the sums. 8 bits is the
 * significand of bfloat16; the exponent range is not limited (the factors lie
 * far inside bfloat16's range). 0 (the default) keeps every factor in FP64. */
static int stored_bits = 0;

/* x rounded to `bits` significant bits, ties to even (x = m 2^e with
 * 1/2 <= |m| < 1, so m 2^bits lies in [2^(bits-1), 2^bits) and rounding it to
 * an integer keeps `bits` significant bits). */
double orc_round_significand(double x, int bits) {
  if (bits <= 0 || bits >= 53 || x == 0.0 || !isfinite(x)) return x;
  int e;
  double m = frexp(x, &e);
  return ldexp(nearbyint(ldexp(m, bits)), e - bits);
}

int orc_set_stored_factor_bits(int bits) {
  if (bits < 0 || bits > 53) return ORC_ERR_ARG;
  stored_bits = bits;
  return ORC_OK;
}

/* integrand of A_mn at one quadrature point: w F d^theta phi_n d^eta phi_m */
static double integrand(const orc_patch *P, const orc_qp *g, const int *q, const int *m,
                        const int *n, int op) {
  if (stored_bits > 0) {
    if (op == ORC_MASS)
      return orc_round_significand(g->w * g->FM, stored_bits) * basis_at(P, q, m, -1) *
             basis_at(P, q, n, -1);
    double s = 0.0;
    for (int i = 0; i < P->d; ++i) {
      double dm = basis_at(P, q, m, i);
      for (int j = 0; j < P->d; ++j)
        s += dm * orc_round_significand(g->w * g->FK[i][j], stored_bits) * basis_at(P, q, n, j);
    }
    return s;
  }
  if (op == ORC_MASS) return g->w * g->FM * basis_at(P, q, m, -1) * basis_at(P, q, n, -1);
  double s = 0.0;
  for (int i = 0; i < P->d; ++i) {
    double dm = basis_at(P, q, m, i);
    for (int j = 0; j < P->d; ++j) s += dm * g->FK[i][j] * basis_at(P, q, n, j);
  }
  return g->w * s;
}

static int64_t lin(const orc_patch *P, const int *n) {
  int64_t r = 0, s = 1;
  for (int a = 0; a < P->d; ++a) { r += s * n[a]; s *= P->N[a]; }
  return r;
}

static void unlin(const orc_patch *P, int64_t r, int *n) {
  for (int a = 0; a < P->d; ++a) { n[a] = (int)(r % P->N[a]); r /= P->N[a]; }
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */

#define PATCH_ARGS int d, const int *orders, const int *nks, const double *knots, \
  const double *ctrl, int coef_kind, double coef_const, double coef_alpha, const double *coef_values
#define PATCH_PASS d, orders, nks, knots, ctrl, coef_kind, coef_const, coef_alpha, coef_values

/* Univariate data of one direction: nodes, weights and dense Q x N tables. */
int orc_tables_1d(int p, int nk, const double *t, double *xq, double *wq, double *B, double *dB) {
  orc_patch P;
  int orders[1] = {p}, nks[1] = {nk};
  int rc = patch_build(&P, 1, orders, nks, t, NULL, 0, 1.0, 0.0, NULL);
  if (rc) { patch_free(&P); return rc; }
  memcpy(xq, P.xq[0], sizeof(double) * (size_t)P.Q[0]);
  memcpy(wq, P.wq[0], sizeof(double) * (size_t)P.Q[0]);
  memcpy(B, P.B[0], sizeof(double) * (size_t)P.Q[0] * P.N[0]);
  memcpy(dB, P.dB[0], sizeof(double) * (size_t)P.Q[0] * P.N[0]);
  patch_free(&P);
  return ORC_OK;
}

/* Per-quadrature-point data in lexicographic quadrature order:
 * w (Qtot), G (Qtot x d), detJ (Qtot), a (Qtot), FM (Qtot),
 * FK (Qtot x d x d, unweighted: a |det J| J^-1 J^-T). Any output may be NULL. */
int orc_quad_data(PATCH_ARGS, double *w, double *G, double *detJ, double *a, double *FM,
                  double *FK) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
  for (int64_t qi = 0; qi < P.Qtot; ++qi) {
    int q[ORC_MAXD] = {0, 0, 0};
    int64_t r = qi;
    for (int k = 0; k < d; ++k) { q[k] = (int)(r % P.Q[k]); r /= P.Q[k]; }
    orc_qp g;
    eval_qp(&P, q, &g);
    if (w) w[qi] = g.w;
    if (G) for (int i = 0; i < d; ++i) G[qi * d + i] = g.G[i];
    if (detJ) detJ[qi] = g.detJ;
    if (a) a[qi] = g.a;
    if (FM) FM[qi] = g.FM;
    if (FK)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) FK[(qi * d + i) * d + j] = g.FK[i][j];
  }
  patch_free(&P);
  return ORC_OK;
}

/* 1D column set of row m in direction a: n with a common non-empty span
 * (the sparsity pattern NZ of Sec. 3.2, which for B-splines is exact). */
static int cols_1d(const orc_patch *P, int a, int m, int *cols) {
  int c = 0;
  int p = P->p[a];
  for (int n = 0; n < P->N[a]; ++n) {
    int lo = m > n ? m : n;
    int hi = (m < n ? m : n) + p - 1;
    int share = 0;
    for (int k = lo; k <= hi; ++k)
      if (k >= 0 && k < P->nk[a] && P->elem_of_span[a][k] >= 0) share = 1;
    if (share) cols[c++] = n;
  }
  return c;
}

/* Number of structurally non-zero entries of the assembled matrix. */
int64_t orc_nnz(PATCH_ARGS) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
  int64_t total = 1;
  for (int a = 0; a < d; ++a) {
    int *cols = (int *)malloc(sizeof(int) * (size_t)P.N[a]);
    int64_t s = 0;
    for (int m = 0; m < P.N[a]; ++m) s += cols_1d(&P, a, m, cols);
    free(cols);
    total *= s;
  }
  patch_free(&P);
  return total;
}

/* CSR assembly. Call with val == NULL to get rowptr (N+1) only; then allocate
 * colind/val of size rowptr[N] and call again. Entries are accumulated element
 * by element, quadrature point by quadrature point, pair by pair. */
int orc_assemble_csr(PATCH_ARGS, int op, int64_t *rowptr, int64_t *colind, double *val) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
  int *c1[ORC_MAXD], *n1[ORC_MAXD];
  for (int a = 0; a < d; ++a) {
    c1[a] = (int *)malloc(sizeof(int) * (size_t)P.N[a] * P.N[a]);
    n1[a] = (int *)malloc(sizeof(int) * (size_t)P.N[a]);
    for (int m = 0; m < P.N[a]; ++m) n1[a][m] = cols_1d(&P, a, m, c1[a] + (size_t)m * P.N[a]);
  }
  /* pattern: row m = product of the 1D column sets, in increasing n */
  rowptr[0] = 0;
  for (int64_t r = 0; r < P.Ntot; ++r) {
    int m[ORC_MAXD];
    unlin(&P, r, m);
    int64_t cnt = 1;
    for (int a = 0; a < d; ++a) cnt *= n1[a][m[a]];
    rowptr[r + 1] = rowptr[r] + cnt;
  }
  if (colind) {
    for (int64_t r = 0; r < P.Ntot; ++r) {
      int m[ORC_MAXD];
      unlin(&P, r, m);
      int64_t pos = rowptr[r];
      int cnt3 = d > 2 ? n1[2][m[2]] : 1, cnt2 = d > 1 ? n1[1][m[1]] : 1;
      for (int k3 = 0; k3 < cnt3; ++k3)
        for (int k2 = 0; k2 < cnt2; ++k2)
          for (int k1 = 0; k1 < n1[0][m[0]]; ++k1) {
            int n[ORC_MAXD] = {c1[0][(size_t)m[0] * P.N[0] + k1],
                               d > 1 ? c1[1][(size_t)m[1] * P.N[1] + k2] : 0,
                               d > 2 ? c1[2][(size_t)m[2] * P.N[2] + k3] : 0};
            colind[pos++] = lin(&P, n);
          }
    }
  }
  if (val) {
    memset(val, 0, sizeof(double) * (size_t)rowptr[P.Ntot]);
    int Ke[ORC_MAXD] = {1, 1, 1}, pe[ORC_MAXD] = {1, 1, 1};
    for (int a = 0; a < d; ++a) { Ke[a] = P.K[a]; pe[a] = P.p[a]; }
    int64_t nel = (int64_t)Ke[0] * Ke[1] * Ke[2];
    for (int64_t el = 0; el < nel; ++el) {
      int e[ORC_MAXD] = {(int)(el % Ke[0]), (int)((el / Ke[0]) % Ke[1]), (int)(el / Ke[0] / Ke[1])};
      int f[ORC_MAXD] = {0, 0, 0};
      for (int a = 0; a < d; ++a) f[a] = first_active(&P, a, e[a]);
      int nloc = 1;
      for (int a = 0; a < d; ++a) nloc *= pe[a];
      for (int g3 = 0; g3 < pe[2]; ++g3)
        for (int g2 = 0; g2 < pe[1]; ++g2)
          for (int g1 = 0; g1 < pe[0]; ++g1) {
            int q[ORC_MAXD] = {e[0] * pe[0] + g1, e[1] * pe[1] + g2, e[2] * pe[2] + g3};
            orc_qp g;
            eval_qp(&P, q, &g);
            for (int im = 0; im < nloc; ++im) {
              int m[ORC_MAXD] = {f[0] + im % pe[0], f[1] + (im / pe[0]) % pe[1],
                                 f[2] + im / (pe[0] * pe[1])};
              int64_t row = lin(&P, m);
              for (int in = 0; in < nloc; ++in) {
                int n[ORC_MAXD] = {f[0] + in % pe[0], f[1] + (in / pe[0]) % pe[1],
                                   f[2] + in / (pe[0] * pe[1])};
                int64_t col = lin(&P, n);
                /* binary search of col in row */
                int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
                while (lo < hi) {
                  int64_t mid = (lo + hi) / 2;
                  if (colind[mid] < col) lo = mid + 1; else hi = mid;
                }
                val[lo] += integrand(&P, &g, q, m, n, op);
              }
            }
          }
    }
  }
  for (int a = 0; a < d; ++a) { free(c1[a]); free(n1[a]); }
  patch_free(&P);
  return ORC_OK;
}

/* y = A x for a CSR matrix, rows spread over the OpenMP threads (each row is
 * summed in column order by one thread, so the result does not depend on the
 * thread count). */
int orc_spmv(int64_t nrows, const int64_t *rowptr, const int64_t *colind, const double *val,
             const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += val[k] * x[colind[k]];
    y[r] = s;
  }
  return ORC_OK;
}

/* The entries A_mn of one row m (per-direction indices m[]) for every n in the
 * window |n_a - m_a| <= p_a - 1, each summed from the definition over the
 * quadrature points of the elements in the support of phi_m, into
 * loc[sum_a (n_a - m_a + p_a - 1) prod_{b<a} W_b], W_a = 2 p_a - 1 (entries
 * with n outside the patch stay zero). */
static void row_window(const orc_patch *P, const int *m, int op, const int *W, double *loc) {
  const int d = P->d;
  int pe[ORC_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) pe[a] = P->p[a];
  memset(loc, 0, sizeof(double) * (size_t)W[0] * W[1] * W[2]);
  /* elements in the support of phi_m: spans k in [m_a, m_a + p_a - 1] */
  int elo[ORC_MAXD] = {0, 0, 0}, ehi[ORC_MAXD] = {0, 0, 0};
  for (int a = 0; a < d; ++a) { elo[a] = m[a]; ehi[a] = m[a] + P->p[a] - 1; }
  for (int k3 = elo[2]; k3 <= ehi[2]; ++k3)
    for (int k2 = elo[1]; k2 <= ehi[1]; ++k2)
      for (int k1 = elo[0]; k1 <= ehi[0]; ++k1) {
        int k[ORC_MAXD] = {k1, k2, k3};
        int e[ORC_MAXD] = {0, 0, 0}, f[ORC_MAXD] = {0, 0, 0}, ok = 1;
        for (int a = 0; a < d; ++a) {
          if (k[a] < 0 || k[a] >= P->nk[a] || P->elem_of_span[a][k[a]] < 0) { ok = 0; break; }
          e[a] = P->elem_of_span[a][k[a]];
          f[a] = first_active(P, a, e[a]);
        }
        if (!ok) continue;
        for (int g3 = 0; g3 < pe[2]; ++g3)
          for (int g2 = 0; g2 < pe[1]; ++g2)
            for (int g1 = 0; g1 < pe[0]; ++g1) {
              int q[ORC_MAXD] = {e[0] * pe[0] + g1, e[1] * pe[1] + g2, e[2] * pe[2] + g3};
              orc_qp g;
              eval_qp(P, q, &g);
              for (int j3 = 0; j3 < pe[2]; ++j3)
                for (int j2 = 0; j2 < pe[1]; ++j2)
                  for (int j1 = 0; j1 < pe[0]; ++j1) {
                    int n[ORC_MAXD] = {f[0] + j1, d > 1 ? f[1] + j2 : 0, d > 2 ? f[2] + j3 : 0};
                    int64_t widx = 0, s = 1;
                    for (int a = 0; a < d; ++a) {
                      widx += s * (n[a] - m[a] + P->p[a] - 1);
                      s *= W[a];
                    }
                    loc[widx] += integrand(P, &g, q, m, n, op);
                  }
            }
      }
}

/* Column n of window entry widx of row m; 0 if n lies outside the patch. */
static int window_col(const orc_patch *P, const int *m, const int *W, int64_t widx, int64_t *col) {
  int n[ORC_MAXD] = {0, 0, 0};
  int64_t r = widx;
  for (int a = 0; a < P->d; ++a) {
    n[a] = (int)(r % W[a]) + m[a] - P->p[a] + 1;
    r /= W[a];
    if (n[a] < 0 || n[a] >= P->N[a]) return 0;
  }
  *col = lin(P, n);
  return 1;
}

/* Selected rows of v = A u, each row assembled on its own from the definition:
 * v_m = sum_n A_mn u_n with A_mn summed over the quadrature points of the
 * elements in the support of phi_m. Also returns sum_n |A_mn| per row.
 * Rows are independent, so they are spread over `threads` OpenMP threads
 * (0 = the runtime default). */
int orc_apply_rows(PATCH_ARGS, int op, const double *u, int64_t nrows, const int64_t *rows,
                   double *v, double *rowabs, int threads) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  int W[ORC_MAXD] = {1, 1, 1};      /* width of the local column window, 2p - 1 */
  for (int a = 0; a < d; ++a) W[a] = 2 * P.p[a] - 1;
  int64_t wsize = (int64_t)W[0] * W[1] * W[2];
#pragma omp parallel
  {
    double *loc = (double *)malloc(sizeof(double) * (size_t)wsize);
#pragma omp for schedule(dynamic, 1)
    for (int64_t ir = 0; ir < nrows; ++ir) {
      int m[ORC_MAXD] = {0, 0, 0};
      unlin(&P, rows[ir], m);
      row_window(&P, m, op, W, loc);
      double sum = 0.0, sabs = 0.0;
      for (int64_t widx = 0; widx < wsize; ++widx) {
        int64_t col;
        if (!window_col(&P, m, W, widx, &col)) continue;
        sum += loc[widx] * u[col];
        sabs += fabs(loc[widx]);
      }
      v[ir] = sum;
      if (rowabs) rowabs[ir] = sabs;
    }
    free(loc);
  }
  patch_free(&P);
  return ORC_OK;
}

/* CSR of selected rows of A, each row assembled on its own from the definition
 * (as in orc_apply_rows): row ir of the output holds A_{rows[ir], n} for every
 * n with |n_a - m_a| <= p_a - 1 inside the patch (the support pattern of the
 * nnz Corollary, Sec. 3.2), columns ascending. Call with colind == NULL to get
 * rowptr (nrows + 1 entries) only; then again with colind and val of rowptr[nrows]
 * entries. Rows run on `threads` OpenMP threads (0 = the runtime default). */
int orc_assemble_rows(PATCH_ARGS, int op, int64_t nrows, const int64_t *rows, int64_t *rowptr,
                      int64_t *colind, double *val, int threads) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  int W[ORC_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) W[a] = 2 * P.p[a] - 1;
  int64_t wsize = (int64_t)W[0] * W[1] * W[2];
  if (!colind) {
    rowptr[0] = 0;
    for (int64_t ir = 0; ir < nrows; ++ir) {
      int m[ORC_MAXD] = {0, 0, 0};
      unlin(&P, rows[ir], m);
      int64_t cnt = 0, col;
      for (int64_t widx = 0; widx < wsize; ++widx) cnt += window_col(&P, m, W, widx, &col);
      rowptr[ir + 1] = rowptr[ir] + cnt;
    }
    patch_free(&P);
    return ORC_OK;
  }
#pragma omp parallel
  {
    double *loc = (double *)malloc(sizeof(double) * (size_t)wsize);
#pragma omp for schedule(dynamic, 1)
    for (int64_t ir = 0; ir < nrows; ++ir) {
      int m[ORC_MAXD] = {0, 0, 0};
      unlin(&P, rows[ir], m);
      row_window(&P, m, op, W, loc);
      int64_t pos = rowptr[ir], col;
      /* window index order is lexicographic in n with the first index
         fastest, i.e. ascending global column */
      for (int64_t widx = 0; widx < wsize; ++widx) {
        if (!window_col(&P, m, W, widx, &col)) continue;
        colind[pos] = col;
        val[pos] = loc[widx];
        ++pos;
      }
    }
    free(loc);
  }
  patch_free(&P);
  return ORC_OK;
}

/* Whole v = A u without a global matrix: for each element, the local matrix
 * A_e from the definition, then v_m += sum_n (A_e)_mn u_n. Serial. */
int orc_apply_elementwise(PATCH_ARGS, int op, const double *u, double *v) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
  int Ke[ORC_MAXD] = {1, 1, 1}, pe[ORC_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) { Ke[a] = P.K[a]; pe[a] = P.p[a]; }
  int nloc = pe[0] * pe[1] * pe[2];
  double *Ae = (double *)malloc(sizeof(double) * (size_t)nloc * nloc);
  memset(v, 0, sizeof(double) * (size_t)P.Ntot);
  int64_t nel = (int64_t)Ke[0] * Ke[1] * Ke[2];
  for (int64_t el = 0; el < nel; ++el) {
    int e[ORC_MAXD] = {(int)(el % Ke[0]), (int)((el / Ke[0]) % Ke[1]), (int)(el / Ke[0] / Ke[1])};
    int f[ORC_MAXD] = {0, 0, 0};
    for (int a = 0; a < d; ++a) f[a] = first_active(&P, a, e[a]);
    memset(Ae, 0, sizeof(double) * (size_t)nloc * nloc);
    for (int g3 = 0; g3 < pe[2]; ++g3)
      for (int g2 = 0; g2 < pe[1]; ++g2)
        for (int g1 = 0; g1 < pe[0]; ++g1) {
          int q[ORC_MAXD] = {e[0] * pe[0] + g1, e[1] * pe[1] + g2, e[2] * pe[2] + g3};
          orc_qp g;
          eval_qp(&P, q, &g);
          for (int im = 0; im < nloc; ++im) {
            int m[ORC_MAXD] = {f[0] + im % pe[0], f[1] + (im / pe[0]) % pe[1],
                               f[2] + im / (pe[0] * pe[1])};
            for (int in = 0; in < nloc; ++in) {
              int n[ORC_MAXD] = {f[0] + in % pe[0], f[1] + (in / pe[0]) % pe[1],
                                 f[2] + in / (pe[0] * pe[1])};
              Ae[im * nloc + in] += integrand(&P, &g, q, m, n, op);
            }
          }
        }
    for (int im = 0; im < nloc; ++im) {
      int m[ORC_MAXD] = {f[0] + im % pe[0], f[1] + (im / pe[0]) % pe[1],
                         f[2] + im / (pe[0] * pe[1])};
      double s = 0.0;
      for (int in = 0; in < nloc; ++in) {
        int n[ORC_MAXD] = {f[0] + in % pe[0], f[1] + (in / pe[0]) % pe[1],
                           f[2] + in / (pe[0] * pe[1])};
        s += Ae[im * nloc + in] * u[lin(&P, n)];
      }
      v[lin(&P, m)] += s;
    }
  }
  free(Ae);
  patch_free(&P);
  return ORC_OK;
}

/* Whole v = A u point by point, without a matrix: for every element and every
 * one of its quadrature points x, first the value of u at x (mass) or its
 * partial derivatives d u / d xi_j (stiffness), each by the direct sum over
 * the p^d functions active on the element (every basis value the full tensor
 * product, as in basis_at: no sum factorization); then the weighted factor
 * times that, g = w F(x) d^theta u(x); then v_m += d^eta phi_m(x) g for every
 * active test function m. Summed over all points this is
 * v_m = sum_n sum_x w F d^theta phi_n d^eta phi_m u_n = (A u)_m, the definition
 * (eq. quadrature:1) with the sum over n taken first, i.e. the local matrix
 * B_e^T D_e B_e applied to u_e without being formed. Stored-factor rounding
 * (stored_bits) applies to w F exactly as in integrand().
 * Parallel without races and in a fixed order: element layers of the last
 * direction whose indices agree modulo p touch disjoint dof layers, so the
 * layers of one residue class run in parallel (one thread per layer) and the
 * classes run one after another; inside a layer elements run in order. */
int orc_apply_qp(PATCH_ARGS, int op, const double *u, double *v, int threads) {
  orc_patch P;
  int rc = patch_build(&P, PATCH_PASS);
  if (rc) { patch_free(&P); return rc; }
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  int Ke[ORC_MAXD] = {1, 1, 1}, pe[ORC_MAXD] = {1, 1, 1};
  for (int a = 0; a < d; ++a) { Ke[a] = P.K[a]; pe[a] = P.p[a]; }
  const int last = d - 1;
  const int nloc = pe[0] * pe[1] * pe[2];
  memset(v, 0, sizeof(double) * (size_t)P.Ntot);
  for (int cls = 0; cls < pe[last]; ++cls) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int layer = cls; layer < Ke[last]; layer += pe[last]) {
      int elo[ORC_MAXD] = {0, 0, 0}, ehi[ORC_MAXD] = {1, 1, 1};
      for (int a = 0; a < d; ++a) { elo[a] = 0; ehi[a] = Ke[a]; }
      elo[last] = layer;
      ehi[last] = layer + 1;
      for (int e3 = elo[2]; e3 < ehi[2]; ++e3)
        for (int e2 = elo[1]; e2 < ehi[1]; ++e2)
          for (int e1 = elo[0]; e1 < ehi[0]; ++e1) {
            int e[ORC_MAXD] = {e1, e2, e3}, f[ORC_MAXD] = {0, 0, 0};
            for (int a = 0; a < d; ++a) f[a] = first_active(&P, a, e[a]);
            for (int g3 = 0; g3 < pe[2]; ++g3)
              for (int g2 = 0; g2 < pe[1]; ++g2)
                for (int g1 = 0; g1 < pe[0]; ++g1) {
                  int q[ORC_MAXD] = {e[0] * pe[0] + g1, e[1] * pe[1] + g2, e[2] * pe[2] + g3};
                  orc_qp g;
                  eval_qp(&P, q, &g);
                  /* d^theta u at x: value, or reference partial derivatives */
                  double du[ORC_MAXD] = {0.0, 0.0, 0.0}, uval = 0.0;
                  for (int in = 0; in < nloc; ++in) {
                    int n[ORC_MAXD] = {f[0] + in % pe[0], f[1] + (in / pe[0]) % pe[1],
                                       f[2] + in / (pe[0] * pe[1])};
                    double un = u[lin(&P, n)];
                    if (op == ORC_MASS) uval += basis_at(&P, q, n, -1) * un;
                    else for (int j = 0; j < d; ++j) du[j] += basis_at(&P, q, n, j) * un;
                  }
                  /* g = w F d^theta u */
                  double gm = 0.0, gk[ORC_MAXD] = {0.0, 0.0, 0.0};
                  if (op == ORC_MASS) {
                    double wf = g.w * g.FM;
                    if (stored_bits > 0) wf = orc_round_significand(wf, stored_bits);
                    gm = wf * uval;
                  } else {
                    for (int i = 0; i < d; ++i)
                      for (int j = 0; j < d; ++j) {
                        double wf = g.w * g.FK[i][j];
                        if (stored_bits > 0) wf = orc_round_significand(wf, stored_bits);
                        gk[i] += wf * du[j];
                      }
                  }
                  /* v_m += d^eta phi_m g */
                  for (int im = 0; im < nloc; ++im) {
                    int m[ORC_MAXD] = {f[0] + im % pe[0], f[1] + (im / pe[0]) % pe[1],
                                       f[2] + im / (pe[0] * pe[1])};
                    double c = 0.0;
                    if (op == ORC_MASS) c = basis_at(&P, q, m, -1) * gm;
                    else for (int i = 0; i < d; ++i) c += basis_at(&P, q, m, i) * gk[i];
                    v[lin(&P, m)] += c;
                  }
                }
          }
    }
  }
  patch_free(&P);
  return ORC_OK;
}

int orc_set_threads(int n) {
  if (n < 1) return ORC_ERR_ARG;
#ifdef _OPENMP
  omp_set_num_threads(n);
#endif
  return ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
