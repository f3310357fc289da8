"""Repeated interior knots on the CUDA path, against the FP64 oracle (GPU).

An interior knot of multiplicity m (1 <= m <= p - 1) lowers the continuity
there to C^(p-1-m) and adds m - 1 functions (Sec. 2); the elements are the
non-empty knot spans (Sec. 3). The device keeps the empty spans as elements of
zero weight, so these tests check that nothing of them leaks out: tables,
factors, quadrature points and per-point coefficients of the non-empty spans
only, the apply in every precision against the oracle (which never sees an
empty span), the assembled CSR against the oracle's pattern of Cor. 3 (pairs
that share a non-empty element), the solver, the batched apply and the factors
evaluated on the fly. Bars as in the other parity tests (tests/gpu_helpers.py,
tol).
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import gpu_apply, sample_rows, scaled_err, tol

pytestmark = pytest.mark.gpu


def _rep_knots(p, K, seed):
    """Open knot vector over K non-empty spans of random lengths whose interior
    knots have random multiplicities in 1..p-1, the middle one p - 1."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    mult = [int(m) for m in rng.integers(1, p, K - 1)] if p > 1 else [1] * (K - 1)
    if K > 1:
        mult[(K - 1) // 2] = p - 1
    return I.open_knots_from_breaks(p, br, mult)


def _patch(d, p, K, seed, coef=True, noise=1.0 / 3.0):
    knots = [_rep_knots(p, k, seed + 10 * a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    kw = dict(coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5) if coef else {}
    return I.make_patch(d, p, list(K), noise_amp=gap * noise, seed=seed, knots=knots, **kw)


def _spans(t, p):
    """Knot index k of every non-empty span [t_k, t_k+1) (the oracle's elements)."""
    return [k for k in range(p - 1, len(t) - p) if t[k + 1] > t[k]]


def _bits(prec):
    return O.BF16_BITS if prec in (G.BF16, G.BF16_MMA) else 0


def test_knot_vectors_have_repeated_knots():
    for p in range(3, 10):
        t = _rep_knots(p, 5, p)
        vals, counts = np.unique(t, return_counts=True)
        assert counts[0] == p and counts[-1] == p
        assert counts[1:-1].max() == p - 1 and counts[1:-1].min() >= 1


@pytest.mark.parametrize("p", range(2, 10))
def test_tables_of_the_non_empty_spans(p):
    patch, _ = _patch(3, p, (5, 3, 4), seed=p, coef=False)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        for a in range(3):
            t = patch.knots[a]
            nodes, weights, B, dB = plan.tables(a)
            xq, wq, Bo, dBo = O.tables_1d(t, p)
            assert len(nodes) == len(xq) == len(_spans(t, p)) * p
            assert np.max(np.abs(nodes - xq)) < 1e-15
            assert np.max(np.abs(weights - wq)) < 1e-15
            first = np.repeat([k - p + 1 for k in _spans(t, p)], p)
            Q = np.arange(len(xq))
            scale = np.max(np.abs(dBo))
            for j in range(p):
                assert np.max(np.abs(B[:, j] - Bo[Q, first + j])) < 1e-14
                assert np.max(np.abs(dB[:, j] - dBo[Q, first + j])) < 1e-13 * scale


@pytest.mark.parametrize("d,p,K", [(3, 3, (5, 4, 3)), (3, 5, (3, 4, 3)), (3, 9, (2, 3, 2)),
                                   (2, 4, (9, 5)), (2, 8, (4, 3))])
def test_factors_and_points_of_the_non_empty_spans(d, p, K):
    patch, _ = _patch(d, p, K, seed=20 + p)
    qd = O.quad_data(patch)
    fm = qd["w"] * qd["FM"]
    iu = np.triu_indices(d)
    fk = (qd["w"][:, None, None] * qd["FK"])[:, iu[0], iu[1]]
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16)) as plan:
        assert plan.num_quad_points == patch.num_quad_points == len(fm)
        assert plan.describe(G.FP64)["num_quad_points"] == patch.num_quad_points
        assert np.max(np.abs(plan.factors(G.MASS, G.FP64) - fm)) < 1e-13 * np.max(np.abs(fm))
        assert np.max(np.abs(plan.factors(G.STIFFNESS, G.FP64) - fk)) < 1e-12 * np.max(np.abs(fk))
        assert np.max(np.abs(plan.factors(G.MASS, G.FP32) - fm) / np.abs(fm)) < 1e-7
        assert np.max(np.abs(plan.factors(G.MASS, G.BF16) - fm) / np.abs(fm)) < 2.0 ** -8
        x = plan.quad_points()
    assert x.shape == (patch.num_quad_points, d)
    assert np.max(np.abs(x - qd["G"])) < 1e-14


# (d, p, K): K non-empty spans per direction; with the empty spans of the
# repeated knots every case covers two or more tiles (ragged tails included) in
# at least one direction for every precision's default kernel, and empty spans
# fall both inside tiles and on their edges
APPLY_CASES = [(3, 3, (7, 5, 6)), (3, 4, (6, 5, 4)), (3, 5, (4, 5, 3)), (3, 6, (3, 4, 3)),
               (3, 7, (3, 3, 2)), (3, 8, (2, 3, 2)), (3, 9, (2, 2, 3)),
               (2, 3, (9, 7)), (2, 6, (5, 6)), (2, 9, (4, 3))]


@pytest.mark.parametrize("d,p,K", APPLY_CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_apply_whole_vector_every_precision(d, p, K, op):
    patch, u = _patch(d, p, K, seed=30 + p + d)
    precs = (G.FP64, G.FP32, G.BF16) + ((G.TF32, G.BF16_MMA) if d == 3 else ())
    rows = sample_rows(patch, 24, seed=p)
    ref = {}
    for bits in (0, O.BF16_BITS):
        with O.stored_factor_bits(bits):
            ref[bits] = (O.apply_qp(patch, op, u), O.apply_rows(patch, op, u, rows))
    with G.Plan.from_patch(patch, precisions=precs) as plan:
        for prec in precs:
            v_ref, (vr, ra) = ref[_bits(prec)]
            assert np.max(np.abs(v_ref[rows] - vr)) < 1e-13 * ra.max() * np.abs(u).max()
            v = gpu_apply(plan, op, u, prec)
            err = scaled_err(v, v_ref, float(ra.max()), u)
            assert err < tol(prec, patch), (prec, err)


def test_candidates_and_variants_with_repeated_knots():
    # every compiled tile shape and factor-stream variant of two orders
    for p, K in ((4, (5, 4, 6)), (7, (2, 3, 3))):
        patch, u = _patch(3, p, K, seed=40 + p)
        v_ref = O.apply_qp(patch, O.STIFFNESS, u)
        _, ra = O.apply_rows(patch, O.STIFFNESS, u, sample_rows(patch, 16, seed=1))
        for prec in (G.FP32, G.FP64):
            for tile, variant in G.list_kernels(3, p, prec):
                with G.Plan.from_patch(patch, precisions=(prec,), tile=tuple(tile),
                                       kernel_variant=variant) as plan:
                    v = gpu_apply(plan, G.STIFFNESS, u, prec)
                    assert scaled_err(v, v_ref, ra.max(), u) < tol(prec, patch), (p, prec, tile, variant)


def test_per_point_coefficient_with_repeated_knots():
    # the coefficient given at the device's own physical quadrature points
    # reproduces the oracle's operator with the same coefficient function
    patch, u = _patch(3, 4, (5, 4, 3), seed=50)
    v_ref = O.apply_qp(patch, G.STIFFNESS, u)
    _, ra = O.apply_rows(patch, G.STIFFNESS, u, sample_rows(patch, 16, seed=2))
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as probe:
        x = probe.quad_points()
    vals = np.exp(0.5 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]))
    patch.coef_kind, patch.coef_values = I.COEF_VALUES, vals
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec in (G.FP64, G.FP32):
            v = gpu_apply(plan, G.STIFFNESS, u, prec)
            assert scaled_err(v, v_ref, ra.max(), u) < tol(prec, patch), prec


@pytest.mark.parametrize("d,p,K", [(3, 3, (4, 3, 5)), (3, 5, (3, 2, 3)), (2, 4, (6, 5)),
                                   (2, 7, (3, 4))])
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_assembly_pattern_and_values_match_oracle(d, p, K, op):
    patch, u = _patch(d, p, K, seed=60 + p)
    rp, ci, va = O.assemble_csr(patch, op)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        assert plan.assembled_nnz() == len(va) == O.nnz(patch)
        # whole, and one element layer of the last direction per chunk
        for limit in (0, 1):
            grp, gci, gva = (x.cpu().numpy() for x in plan.assemble_csr(op, workspace_limit_bytes=limit))
            assert np.array_equal(grp, rp) and np.array_equal(gci, ci)
            assert np.max(np.abs(gva - va)) <= 1e-12 * O.csr_inf_norm(rp, va), limit


def test_solver_with_repeated_knots():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    patch, _ = _patch(3, 4, (4, 5, 4), seed=70)
    rp, ci, va = O.assemble_csr(patch, O.STIFFNESS)
    A = sp.csr_matrix((va, ci, rp), shape=(patch.num_dofs,) * 2)
    Ns = patch.dofs_per_dir
    idx = np.arange(patch.num_dofs)
    i0, i1, i2 = idx % Ns[0], (idx // Ns[0]) % Ns[1], idx // (Ns[0] * Ns[1])
    m = (i0 > 0) & (i0 < Ns[0] - 1) & (i1 > 0) & (i1 < Ns[1] - 1) & (i2 > 0) & (i2 < Ns[2] - 1)
    b = np.random.default_rng(5).uniform(-1, 1, patch.num_dofs)
    b[~m] = 0.0
    x_ref = np.zeros(patch.num_dofs)
    x_ref[m] = spla.spsolve(A[m][:, m].tocsc(), b[m])
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        bd = torch.as_tensor(b, device="cuda")
        xd = torch.zeros_like(bd)
        rep = plan.cg_solve(bd, xd, inner_prec=G.FP32, rtol=1e-11, inner_rtol=1e-4)
        x = xd.cpu().numpy()
    assert rep["converged"], rep
    assert np.max(np.abs(x - x_ref)) < 1e-7 * np.max(np.abs(x_ref))


def test_batch_and_on_the_fly_with_repeated_knots():
    import torch
    patches = [_patch(3, p, K, seed=80 + p) for p, K in ((3, (5, 4, 6)), (4, (4, 5, 3)), (3, (3, 3, 4)))]
    plans = [G.Plan.from_patch(pt, precisions=(G.FP32,)) for pt, _ in patches]
    u = np.concatenate([uk for _, uk in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    try:
        with G.Batch(plans, op=G.STIFFNESS, prec=G.FP32) as batch:
            v = torch.empty_like(ud)
            batch.apply(ud, v)
            torch.cuda.synchronize()
            for k, (pt, uk) in enumerate(patches):
                a = batch.offsets[k]
                vk = v[a:a + pt.num_dofs].double().cpu().numpy()
                _, ra = O.apply_rows(pt, G.STIFFNESS, uk, sample_rows(pt, 16, seed=k))
                assert scaled_err(vk, O.apply_qp(pt, G.STIFFNESS, uk), ra.max(), uk) < tol(G.FP32, pt)
    finally:
        for plan in plans:
            plan.close()
    # factors evaluated on the fly: empty spans have zero weight there too
    for pt, uk in patches[:2]:
        for op in (G.MASS, G.STIFFNESS):
            with G.Plan.from_patch(pt, precisions=(G.FP32,), geometry=G.GEOMETRY_ON_THE_FLY) as plan:
                v = gpu_apply(plan, op, uk, G.FP32)
            _, ra = O.apply_rows(pt, op, uk, sample_rows(pt, 16, seed=3))
            assert scaled_err(v, O.apply_qp(pt, op, uk), ra.max(), uk) < tol(G.FP32, pt), op
