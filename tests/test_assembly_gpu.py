"""GPU sum-factorized assembly (Alg. 1 over the whole patch) against the
oracle's CSR, through the C-ABI (GPU).

The oracle assembles every entry from the definition (eq. quadrature:1),
element by element and quadrature point by quadrature point; the GPU sums one
direction at a time. Both give the same quadrature matrix up to rounding, so
indices must agree exactly and values within 1e-12 ||A||_inf (the FP64 bar of
the apply, applied entrywise)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import gpu_apply, sample_rows, scaled_err

pytestmark = pytest.mark.gpu


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


def _patch(d, p, K, seed=50):
    knots = [_nonuniform_knots(p, k, seed + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    return I.make_patch(d, p, list(K), noise_amp=min(0.2 / max(K), gap / 3), seed=seed,
                        knots=knots, coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)


def _gpu_csr(plan, op, limit=0):
    rp, ci, va = plan.assemble_csr(op, workspace_limit_bytes=limit)
    return rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy()


CASES = [(2, 2, (5, 4)), (2, 3, (6, 5)), (2, 5, (4, 3)), (2, 9, (3, 2)),
         (3, 2, (4, 3, 3)), (3, 3, (3, 4, 2)), (3, 4, (3, 3, 3)), (3, 6, (2, 2, 3)),
         (3, 9, (1, 2, 1))]


@pytest.mark.parametrize("d,p,K", CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_assembly_matches_oracle_csr(d, p, K, op):
    patch, _ = _patch(d, p, K)
    rp_o, ci_o, va_o = O.assemble_csr(patch, op)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        assert plan.assembled_nnz() == len(ci_o) == O.nnz(patch)
        rp, ci, va = _gpu_csr(plan, op)
    assert np.array_equal(rp, rp_o)
    assert np.array_equal(ci, ci_o)
    a_inf = O.csr_inf_norm(rp_o, va_o)
    assert np.max(np.abs(va - va_o)) <= 1e-12 * a_inf


def test_assembly_chunking_is_deterministic():
    """One element layer per chunk (a tiny workspace limit) against a single
    chunk: the same matrix up to rounding; repeated calls bitwise equal."""
    patch, _ = _patch(3, 3, (4, 3, 5), seed=61)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        _, _, v_one = _gpu_csr(plan, G.STIFFNESS)
        _, _, v_small = _gpu_csr(plan, G.STIFFNESS, limit=1)
        _, _, v_small2 = _gpu_csr(plan, G.STIFFNESS, limit=1)
    assert np.array_equal(v_small, v_small2)
    assert np.max(np.abs(v_one - v_small)) <= 1e-14 * np.max(np.abs(v_one))


@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_assembled_matrix_times_u_equals_matrix_free_apply(op):
    """At a size the oracle's CSR would be slow for: the assembled matrix times
    u equals the FP64 matrix-free apply, and sampled rows equal the oracle's."""
    patch, u = I.config_cube(p=4, K=16)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        rp, ci, va = _gpu_csr(plan, op)
        v_mf = gpu_apply(plan, op, u, G.FP64)
    A = sp.csr_matrix((va, ci, rp), shape=(patch.num_dofs,) * 2)
    a_inf = float(np.max(np.abs(A).sum(axis=1)))
    assert scaled_err(A @ u, v_mf, a_inf, u) < 1e-13
    rows = sample_rows(patch, 64, seed=3)
    vr, ra = O.apply_rows(patch, op, u, rows)
    assert scaled_err((A @ u)[rows], vr, ra.max(), u) < 1e-12


def test_assembly_config_cube_64_p4_sampled_rows():
    """The 64^3, p = 4 benchmark patch: sampled rows of the assembled K times u
    against the oracle's rows."""
    patch, u = I.config_cube(p=4, K=64)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        rp, ci, va = plan.assemble_csr(G.STIFFNESS)
        rows = sample_rows(patch, 64, seed=4)
        rp_h = rp.cpu().numpy()
        lo, hi = rp_h[rows], rp_h[rows + 1]
        ci_h, va_h = ci.cpu().numpy(), va.cpu().numpy()
    v = np.array([np.dot(va_h[a:b], u[ci_h[a:b]]) for a, b in zip(lo, hi)])
    vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    assert scaled_err(v, vr, ra.max(), u) < 1e-12


def test_assembly_argument_errors():
    patch, _ = I.make_patch(3, 2, 3, seed=1)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        with pytest.raises(G.IgasfError) as ei:
            plan.assemble_csr(G.STIFFNESS)
        assert ei.value.code == -4          # UNSUPPORTED: no FP64 factors
    lib = G.load_library()
    assert lib.igasf_assemble_csr(None, 0, None, None, None, 0, None) == -1
