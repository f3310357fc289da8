"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test compares the oracle with a library routine, a closed form, the
paper's own count formula, an invariant of the operator, or an independent
numpy/scipy brute force on tiny patches, so that a dropped term, a wrong sign
or index, or a transposed operand anywhere in the oracle fails at least one.
"""
from fractions import Fraction
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle as O
from paper_1809_05471_gb300 import inputs as I
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Gauss rule (Example gauss: p points per element per direction) ----------

@pytest.mark.parametrize("n", range(1, 14))
def test_gauss_matches_numpy_leggauss(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9])
def test_gauss_exact_on_monomials(n):
    x, w = O.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


# --- univariate B-splines (Cox-de Boor, Example 1) ---------------------------

def _knots_cases():
    rng = np.random.default_rng(3)
    cases = []
    for p in range(1, 8):
        cases.append((I.open_uniform_knots(p, 5), p))
        br = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0.05, 0.95, 4)]))
        mult = [int(rng.integers(1, max(p, 1) + 0)) if p > 1 else 1 for _ in range(4)]
        mult = [min(m, max(p - 1, 1)) for m in mult]
        cases.append((I.open_knots_from_breaks(p, br, mult), p))
    return cases


@pytest.mark.parametrize("t,p", _knots_cases())
def test_bspline_values_and_derivatives_match_scipy(t, p):
    xs = np.linspace(t[0], t[-1], 41)[1:-1] + 1e-3
    for x in xs:
        if np.any(np.isclose(x, t)):
            continue
        val, der = O.bspline_all(t, p, x)
        ref = BSpline.design_matrix([x], t, p - 1).toarray()[0]
        assert np.max(np.abs(val - ref)) < 1e-14
        if p > 1:
            dref = np.array([BSpline(t, np.eye(len(t) - p)[n], p - 1).derivative()(x)
                             for n in range(len(t) - p)])
            assert np.max(np.abs(der - dref)) < 1e-12 * max(1.0, np.max(np.abs(dref)))


@pytest.mark.parametrize("t,p", _knots_cases())
def test_partition_of_unity_and_derivative_sum(t, p):
    xq, wq, B, dB = O.tables_1d(t, p)
    assert np.max(np.abs(B.sum(axis=1) - 1.0)) < 1e-14
    assert np.max(np.abs(dB.sum(axis=1))) < 1e-11
    assert np.all(B >= -1e-15)
    # weights of one element sum to its length; all of them to the interval
    assert abs(wq.sum() - (t[-1] - t[0])) < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_derivative_matches_central_difference(p):
    t = I.open_knots_from_breaks(p, [0.0, 0.13, 0.4, 0.41, 0.77, 1.0])
    h = 1e-6
    for x in [0.05, 0.2, 0.405, 0.6, 0.9]:
        _, der = O.bspline_all(t, p, x)
        vp = O.bspline_all(t, p, x + h, deriv=False)
        vm = O.bspline_all(t, p, x - h, deriv=False)
        fd = (vp - vm) / (2 * h)
        assert np.max(np.abs(der - fd)) < 1e-6 * max(1, np.max(np.abs(der)))


# --- 1D matrices against closed forms ----------------------------------------

def _cardinal_values(order):
    """Exact values M(j), M''(j) at the integers of the cardinal B-spline of the
    given order on knots 0..order, from the recurrence
    M_k(x) = (x M_{k-1}(x) + (k - x) M_{k-1}(x - 1)) / (k - 1) written over
    piecewise polynomials with exact rationals."""
    # piecewise polynomials: pieces[i] = coefficients (ascending) on [i, i+1)
    pieces = {0: [Fraction(1)]}
    for k in range(2, order + 1):
        new = {}
        for i in range(k):
            acc = [Fraction(0)] * k
            # x * M_{k-1}(x) on [i, i+1)
            if i in pieces:
                for e, c in enumerate(pieces[i]):
                    acc[e + 1] += c / (k - 1)
            # (k - x) * M_{k-1}(x - 1) on [i, i+1): shift piece i-1 by 1
            if (i - 1) in pieces:
                c_shift = _shift(pieces[i - 1], 1)
                for e, c in enumerate(c_shift):
                    acc[e] += Fraction(k) * c / (k - 1)
                    acc[e + 1] -= c / (k - 1)
            new[i] = acc
        pieces = new
    def ev(poly, x, der=0):
        s = Fraction(0)
        for e, c in enumerate(poly):
            if e < der:
                continue
            f = 1
            for r in range(der):
                f *= (e - r)
            s += c * f * Fraction(x) ** (e - der)
        return s
    vals = [ev(pieces[j], j) if j in pieces else Fraction(0) for j in range(order + 1)]
    d2 = [ev(pieces[j], j, 2) if j in pieces else Fraction(0) for j in range(order + 1)]
    return vals, d2


def _shift(poly, s):
    """Coefficients of q(x) = poly(x - s)."""
    from math import comb
    out = [Fraction(0)] * len(poly)
    for e, c in enumerate(poly):
        for r in range(e + 1):
            out[r] += c * comb(e, r) * Fraction(-s) ** (e - r)
    return out


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_uniform_1d_rows_match_cardinal_closed_form(p):
    """Interior rows of the uniform 1D mass (stiffness) matrix are h times
    (minus 1/h times the second derivative of) the order-2p cardinal B-spline
    at the integers p + k, k = -(p-1)..(p-1) (autocorrelation identity)."""
    K = 12
    h = 1.0 / K
    t = I.open_uniform_knots(p, K)
    patch = I.Patch(d=1, orders=[p], knots=[t], ctrl=I.greville(t, p)[:, None].copy())
    M = O.csr_to_dense(*O.assemble_csr(patch, O.MASS), patch.num_dofs)
    Kst = O.csr_to_dense(*O.assemble_csr(patch, O.STIFFNESS), patch.num_dofs)
    vals, d2 = _cardinal_values(2 * p)
    i = patch.num_dofs // 2
    for k in range(-(p - 1), p):
        assert abs(M[i, i + k] - h * float(vals[p + k])) < 1e-15
        assert abs(Kst[i, i + k] - (-float(d2[p + k]) / h)) < 1e-12
    # the table often quoted for p = 2..4 (row / h and row * h)
    if p == 2:
        assert np.allclose(M[i, i - 1:i + 2] / h, [1 / 6, 4 / 6, 1 / 6], atol=1e-14)
        assert np.allclose(Kst[i, i - 1:i + 2] * h, [-1, 2, -1], atol=1e-12)
    if p == 4:
        ref = np.array([1, 120, 1191, 2416, 1191, 120, 1]) / 5040
        assert np.allclose(M[i, i - 3:i + 4] / h, ref, atol=1e-14)
        refk = np.array([-1, -24, -15, 80, -15, -24, -1]) / 120
        assert np.allclose(Kst[i, i - 3:i + 4] * h, refk, atol=1e-12)


# --- sparsity: the paper's Corollary lem:nnz-B-spline ------------------------

def _golden_nnz():
    rows = []
    with open(os.path.join(GOLDEN, "nnz_open_knots.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, _, tail = line.partition(":")
            p, K, nz = (int(x) for x in head.split())
            mult = [int(x) for x in tail.split()] if tail else [1] * (K - 1)
            rows.append((p, K, nz, mult))
    return rows


@pytest.mark.parametrize("p,K,nz,mult", _golden_nnz())
def test_nnz_1d_equals_corollary(p, K, nz, mult):
    breaks = np.linspace(0, 1, K + 1) ** 1.3
    t = I.open_knots_from_breaks(p, breaks, mult)
    patch = I.Patch(d=1, orders=[p], knots=[t], ctrl=I.greville(t, p)[:, None].copy())
    assert O.nnz(patch) == nz
    rp, ci, va = O.assemble_csr(patch, O.MASS)
    assert rp[-1] == nz


def test_nnz_3d_is_product_of_corollary():
    p = 3
    ks = [2, 3, 4]
    patch, _ = I.make_patch(3, p, ks, noise_amp=0.02, seed=1)
    expect = 1
    for K in ks:
        expect *= (2 * p - 1) * K + (p - 1) ** 2
    assert O.nnz(patch) == expect
    rp, _, _ = O.assemble_csr(patch, O.MASS)
    assert rp[-1] == expect


# --- whole operator vs an independent brute force (tiny patches) -------------

def _tiny_cases():
    cases = []
    for d in (2, 3):
        for p in (2, 3, 4) if d == 3 else (2, 3, 5, 6):
            for K in (1, 2) if d == 3 else (1, 2, 3):
                cases.append((d, p, K))
    return cases


@pytest.mark.parametrize("d,p,K", _tiny_cases())
@pytest.mark.parametrize("op", [O.MASS, O.STIFFNESS])
def test_dense_matches_brute_force(d, p, K, op):
    breaks = np.array([0.0, 0.3, 0.45, 1.0])[: K + 1] if K < 3 else np.array([0, .2, .5, 1.])
    breaks = np.concatenate([breaks[:-1], [1.0]]) if K > 1 else np.array([0.0, 1.0])
    knots = [I.open_knots_from_breaks(p, breaks * (1 + 0.1 * a)) for a in range(d)]
    patch, u = I.make_patch(d, p, K, noise_amp=0.04, seed=11 + d + p, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    A = O.csr_to_dense(*O.assemble_csr(patch, op), patch.num_dofs)
    Ab = brute.dense_operator(patch, op)
    assert np.max(np.abs(A - Ab)) < 1e-13 * np.max(np.abs(Ab))


def test_dense_matches_brute_force_repeated_knots():
    p = 4
    knots = [I.open_knots_from_breaks(p, [0, 0.3, 0.6, 1.0], [2, 3]),
             I.open_knots_from_breaks(p, [0, 0.5, 1.0], [1]),
             I.open_knots_from_breaks(p, [0, 0.25, 1.0], [2])]
    patch, u = I.make_patch(3, p, [3, 2, 2], noise_amp=0.01, seed=5, knots=knots)
    for op in (O.MASS, O.STIFFNESS):
        A = O.csr_to_dense(*O.assemble_csr(patch, op), patch.num_dofs)
        Ab = brute.dense_operator(patch, op)
        assert np.max(np.abs(A - Ab)) < 1e-13 * np.max(np.abs(Ab))


@pytest.mark.parametrize("bits", [0, O.BF16_BITS])
def test_point_and_row_apply_match_brute_force_repeated_knots(bits):
    # the two matrix-free oracle applies on empty spans: nothing of a repeated
    # knot's zero-length span may enter, with exact or bfloat16-rounded factors
    p = 4
    knots = [I.open_knots_from_breaks(p, [0, 0.3, 0.6, 1.0], [2, 3]),
             I.open_knots_from_breaks(p, [0, 0.5, 1.0], [1]),
             I.open_knots_from_breaks(p, [0, 0.25, 1.0], [2])]
    patch, u = I.make_patch(3, p, [3, 2, 2], noise_amp=0.01, seed=5, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rf = None if bits == 0 else (lambda x: np.ldexp(np.round(np.frexp(x)[0] * 256.0),
                                                    np.frexp(x)[1] - 8))
    rows = np.arange(patch.num_dofs)
    for op in (O.MASS, O.STIFFNESS):
        Ab = brute.dense_operator(patch, op, round_factor=rf)
        with O.stored_factor_bits(bits):
            vq = O.apply_qp(patch, op, u)
            vr, ra = O.apply_rows(patch, op, u, rows)
        s = np.max(np.abs(Ab)) * np.max(np.abs(u))
        assert np.max(np.abs(vq - Ab @ u)) < 1e-13 * s
        assert np.max(np.abs(vr - Ab @ u)) < 1e-13 * s
        assert np.max(np.abs(ra - np.abs(Ab).sum(axis=1))) < 1e-13 * np.max(ra)


# --- Kronecker identity for the identity geometry (Sec. 5) -------------------

@pytest.mark.parametrize("p", [2, 3, 4])
def test_identity_geometry_is_kronecker_of_1d_matrices(p):
    knots = [I.open_knots_from_breaks(p, [0, 0.2, 0.7, 1.0]),
             I.open_knots_from_breaks(p, [0, 0.5, 1.0]),
             I.open_knots_from_breaks(p, [0, 0.1, 0.3, 0.6, 1.0])]
    a = 1.7
    patch, _ = I.make_patch(3, p, [3, 2, 4], knots=knots, coef_constant=a)
    M1, K1 = zip(*[brute.univariate_matrices(t, p) for t in knots])
    # lexicographic with the first index fastest: kron(M3, kron(M2, M1))
    Mk = np.kron(M1[2], np.kron(M1[1], M1[0]))
    Kk = a * (np.kron(M1[2], np.kron(M1[1], K1[0])) + np.kron(M1[2], np.kron(K1[1], M1[0]))
              + np.kron(K1[2], np.kron(M1[1], M1[0])))
    M = O.csr_to_dense(*O.assemble_csr(patch, O.MASS), patch.num_dofs)
    K = O.csr_to_dense(*O.assemble_csr(patch, O.STIFFNESS), patch.num_dofs)
    assert np.max(np.abs(M - Mk)) < 1e-15
    assert np.max(np.abs(K - Kk)) < 1e-12 * np.max(np.abs(Kk))


# --- invariants --------------------------------------------------------------

@pytest.mark.parametrize("d,p,K", [(2, 3, 6), (2, 5, 3), (3, 2, 4), (3, 3, 3)])
def test_mass_sums_to_volume(d, p, K):
    """1^T M 1 = sum_x w |det J|; for the perturbed unit cube that is the
    volume 1 exactly whenever Gauss integrates det J exactly (d = 2 for all p,
    d = 3 for p <= 3)."""
    patch, _ = I.make_patch(d, p, K, noise_amp=0.2 / K, seed=2)
    rp, ci, va = O.assemble_csr(patch, O.MASS)
    assert abs(va.sum() - 1.0) < 1e-13


def test_mass_volume_of_affine_map():
    patch, _ = I.make_patch(3, 4, 2, seed=0)
    Aff = np.array([[2.0, 0.3, 0.0], [0.1, 1.5, 0.2], [0.0, -0.4, 0.7]])
    patch.ctrl = patch.ctrl @ Aff.T + np.array([1.0, -2.0, 0.5])
    rp, ci, va = O.assemble_csr(patch, O.MASS)
    assert abs(va.sum() - abs(np.linalg.det(Aff))) < 1e-13


@pytest.mark.parametrize("d,p,K", [(2, 3, 5), (3, 2, 3), (3, 4, 2)])
def test_stiffness_annihilates_constants_symmetric_psd(d, p, K):
    patch, _ = I.make_patch(d, p, K, noise_amp=0.2 / K, seed=4,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    A = O.csr_to_dense(*O.assemble_csr(patch, O.STIFFNESS), patch.num_dofs)
    nrm = np.max(np.abs(A).sum(axis=1))
    assert np.max(np.abs(A @ np.ones(len(A)))) < 1e-13 * nrm
    assert np.max(np.abs(A - A.T)) < 1e-15 * nrm
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > -1e-12 * nrm
    assert np.sum(ev < 1e-10 * nrm) == 1          # only the constants
    M = O.csr_to_dense(*O.assemble_csr(patch, O.MASS), patch.num_dofs)
    assert np.linalg.eigvalsh(M)[0] > 0


@pytest.mark.parametrize("p", [2, 3, 4])
def test_patch_test_affine_geometry(p):
    """For an affine G and constant a, the linear function x_k (coefficients
    c_{., k}) has zero stiffness residual on rows whose support avoids the
    boundary, and c_k^T K c_k = a * volume."""
    patch, _ = I.make_patch(3, p, 3, seed=0, coef_constant=0.8)
    Aff = np.array([[1.2, 0.2, -0.1], [0.0, 0.9, 0.3], [0.2, 0.0, 1.1]])
    patch.ctrl = patch.ctrl @ Aff.T
    A = O.csr_to_dense(*O.assemble_csr(patch, O.STIFFNESS), patch.num_dofs)
    Ns = patch.dofs_per_dir
    idx = np.arange(patch.num_dofs)
    i1, i2, i3 = idx % Ns[0], (idx // Ns[0]) % Ns[1], idx // (Ns[0] * Ns[1])
    interior = (i1 > 0) & (i1 < Ns[0] - 1) & (i2 > 0) & (i2 < Ns[1] - 1) & (i3 > 0) & (i3 < Ns[2] - 1)
    vol = abs(np.linalg.det(Aff))
    for k in range(3):
        c = patch.ctrl[:, k]
        r = A @ c
        assert np.max(np.abs(r[interior])) < 1e-12
        assert abs(c @ r - 0.8 * vol) < 1e-12


def test_patch_test_2d_perturbed():
    """In 2D the Gauss rule integrates cof(J) grad phi exactly for constant a,
    so interior rows of K x_k vanish even on a perturbed geometry."""
    patch, _ = I.make_patch(2, 3, 5, noise_amp=0.04, seed=9)
    A = O.csr_to_dense(*O.assemble_csr(patch, O.STIFFNESS), patch.num_dofs)
    Ns = patch.dofs_per_dir
    idx = np.arange(patch.num_dofs)
    i1, i2 = idx % Ns[0], idx // Ns[0]
    interior = (i1 > 0) & (i1 < Ns[0] - 1) & (i2 > 0) & (i2 < Ns[1] - 1)
    for k in range(2):
        r = A @ patch.ctrl[:, k]
        assert np.max(np.abs(r[interior])) < 1e-12


# --- the oracle's three apply modes agree ------------------------------------

@pytest.mark.parametrize("op", [O.MASS, O.STIFFNESS])
def test_row_and_elementwise_apply_match_spmv(op):
    patch, u = I.make_patch(3, 3, [3, 2, 4], noise_amp=0.05, seed=6,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rp, ci, va = O.assemble_csr(patch, op)
    v = O.spmv(rp, ci, va, u)
    rows = np.arange(patch.num_dofs)
    vr, ra = O.apply_rows(patch, op, u, rows)
    ve = O.apply_elementwise(patch, op, u)
    s = np.max(np.abs(v))
    assert np.max(np.abs(vr - v)) < 1e-14 * s
    assert np.max(np.abs(ve - v)) < 1e-14 * s
    assert np.max(np.abs(ra - np.add.reduceat(np.abs(va), rp[:-1]))) < 1e-14 * np.max(ra)


@pytest.mark.parametrize("d,p,K", [(2, 2, (5, 4)), (2, 4, (4, 3)), (3, 2, (4, 3, 5)),
                                   (3, 3, (3, 2, 4)), (3, 5, (2, 3, 2))])
@pytest.mark.parametrize("op", [O.MASS, O.STIFFNESS])
@pytest.mark.parametrize("bits", [0, O.BF16_BITS])
def test_point_apply_matches_brute_force_and_is_thread_independent(d, p, K, op, bits):
    rng = np.random.default_rng(40 + d + p)
    knots = [I.open_knots_from_breaks(p, np.concatenate(
        [[0.0], np.cumsum(h := rng.uniform(0.5, 1.5, k)) / h.sum()])) for k in K]
    patch, u = I.make_patch(d, p, list(K), noise_amp=0.3 / max(K), seed=9, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rf = None if bits == 0 else (lambda x: np.ldexp(np.round(np.frexp(x)[0] * 256.0),
                                                    np.frexp(x)[1] - 8))
    Ab = brute.dense_operator(patch, op, round_factor=rf)
    with O.stored_factor_bits(bits):
        v1 = O.apply_qp(patch, op, u, threads=1)
        v4 = O.apply_qp(patch, op, u, threads=4)
    ref = Ab @ u
    assert np.max(np.abs(v1 - ref)) < 1e-13 * np.max(np.abs(Ab)) * np.max(np.abs(u))
    assert np.array_equal(v1, v4)


@pytest.mark.parametrize("op", [O.MASS, O.STIFFNESS])
def test_assembled_rows_match_csr(op):
    patch, u = I.make_patch(3, 3, [4, 3, 5], noise_amp=0.05, seed=6,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rp, ci, va = O.assemble_csr(patch, op)
    rows = np.array([0, 7, 31, 32, 33, patch.num_dofs - 1], dtype=np.int64)
    srp, sci, sva = O.assemble_rows(patch, op, rows, threads=3)
    s = np.max(np.abs(va))
    for i, r in enumerate(rows):
        a, b = rp[r], rp[r + 1]
        assert np.array_equal(sci[srp[i]:srp[i + 1]], ci[a:b])      # the Corollary's pattern
        assert np.max(np.abs(sva[srp[i]:srp[i + 1]] - va[a:b])) < 1e-14 * s
    # the product of the sampled rows is the sampled rows of the product
    O.set_threads(2)
    y = O.spmv(srp, sci, sva, u)
    assert np.max(np.abs(y - O.spmv(rp, ci, va, u)[rows])) < 1e-14 * s * np.max(np.abs(u))


def test_quad_data_coefficient_at_physical_point():
    patch, _ = I.config_cube(p=3, K=3)
    qd = O.quad_data(patch)
    G = qd["G"]
    a = np.exp(0.5 * np.sin(2 * np.pi * G[:, 0]) * np.cos(2 * np.pi * G[:, 1]))
    assert np.max(np.abs(qd["a"] - a)) < 1e-15
    assert np.all(qd["detJ"] > 0)


# --- factors stored in a narrower format (bfloat16) ---------------------------

def _bf16_numpy(x):
    """Round to 8 significant bits, ties to even, with numpy (frexp, and
    np.round, which rounds halves to even)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def test_round_significand_matches_torch_bfloat16():
    """The oracle's rounding to 8 significant bits is bfloat16's round to
    nearest even: compared with torch's float32 -> bfloat16 conversion on
    float32 values (exact in float64, so there is no double rounding), ties
    included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x32 = (rng.standard_normal(4000) * np.exp2(rng.integers(-60, 60, 4000))).astype(np.float32)
    bits = x32.view(np.uint32)
    ties = (bits[:500] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)   # exact halfway cases
    x32 = np.concatenate([x32, ties.view(np.float32)])
    ref = torch.from_numpy(x32.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.round_significand(float(v), O.BF16_BITS) for v in x32.astype(np.float64)])
    assert np.array_equal(got, ref)


def test_round_significand_24_bits_is_float32():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(2000) * np.exp2(rng.integers(-100, 100, 2000))
    got = np.array([O.round_significand(float(v), 24) for v in x])
    assert np.array_equal(got, x.astype(np.float32).astype(np.float64))
    assert O.round_significand(0.0, 8) == 0.0


@pytest.mark.parametrize("d,p,K,op", [(2, 3, 2, 0), (2, 4, 2, 1), (3, 2, 2, 1), (3, 3, 2, 0),
                                      (3, 3, 2, 1)])
def test_bf16_stored_factors_match_brute_force(d, p, K, op):
    """With stored_factor_bits(8) the oracle's operator is the quadrature
    operator whose weighted factors w F are rounded to bfloat16: the numpy
    brute force with the same rounding applied to w |det J| and to each
    w a |det J| (J^-1 J^-T)_ij agrees, and both differ from the FP64 operator
    by about the bfloat16 rounding."""
    patch, _ = I.make_patch(d, p, K, noise_amp=0.1, seed=21,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    N = patch.num_dofs
    with O.stored_factor_bits(O.BF16_BITS):
        A = O.csr_to_dense(*O.assemble_csr(patch, op), N)
    A64 = O.csr_to_dense(*O.assemble_csr(patch, op), N)
    Ab = brute.dense_operator(patch, op, round_factor=_bf16_numpy)
    s = np.max(np.abs(Ab))
    assert np.max(np.abs(A - Ab)) < 1e-13 * s
    rel = np.max(np.abs(A - A64)) / s
    assert 1e-5 < rel < 2.0 ** -7


def test_bf16_stored_mass_sums_to_rounded_weights():
    """1^T M 1 with bfloat16-stored factors is the sum over quadrature points of
    the rounded w |det J| (the rounded quantity is the weighted factor, not
    |det J| alone)."""
    patch, _ = I.config_cube(p=3, K=3)
    qd = O.quad_data(patch)
    with O.stored_factor_bits(O.BF16_BITS):
        rp, ci, va = O.assemble_csr(patch, O.MASS)
    expect = np.sum(_bf16_numpy(qd["w"] * qd["FM"]))
    assert abs(va.sum() - expect) < 1e-14 * expect
    assert abs(va.sum() - 1.0) > 1e-6     # no longer the exact volume
