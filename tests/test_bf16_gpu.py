"""The BF16 precision (factors w F stored in bfloat16, FP32 vectors, tables and
arithmetic) against the oracle, through the C-ABI (GPU).

The operator this precision applies is the quadrature operator whose stored
factors are the FP64 factors rounded once to bfloat16 (Sec. 6.2 stores w F at
the quadrature points). The oracle computes exactly that operator under
``stored_factor_bits(8)``, so the parity bar is the FP32 one (1e-5 scaled
max-norm error: only FP32 arithmetic separates the two). Against the FP64
operator the error is the bfloat16 rounding of the factors, about 2^-9
relative per factor; it is checked to stay below 2^-7.
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import tol, gpu_apply, oracle_full, sample_rows, scaled_err

pytestmark = pytest.mark.gpu

BF16_VS_FP64 = 2.0 ** -7


def _bf16(x):
    """Round to 8 significant bits, ties to even (numpy; see the oracle pins)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


def _assert_rounded(got, exact):
    """got == bfloat16(exact), except where exact lies within FP64 noise of a
    rounding tie (the device and the oracle compute w F in different orders)."""
    want = _bf16(exact)
    bad = got != want
    if np.any(bad):
        m, e = np.frexp(exact[bad])
        frac = m * 256.0 - np.floor(m * 256.0)
        assert np.all(np.abs(frac - 0.5) < 1e-6), "factor not rounded to nearest bfloat16"
    assert np.count_nonzero(bad) <= max(1, bad.size // 100000)


@pytest.mark.parametrize("d,p,K", [(3, 2, (9, 5, 4)), (3, 5, (4, 5, 3)), (3, 9, (2, 3, 2)),
                                   (2, 4, (17, 9))])
def test_bf16_factors_are_the_rounded_fp64_factors(d, p, K):
    knots = [_nonuniform_knots(p, k, 20 + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, _ = I.make_patch(d, p, list(K), noise_amp=min(0.2 / max(K), gap / 3), seed=3,
                            knots=knots, coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    qd = O.quad_data(patch)
    w = qd["w"]
    iu = np.triu_indices(d)
    fm = w * qd["FM"]
    fk = (w[:, None, None] * qd["FK"])[:, iu[0], iu[1]]
    with G.Plan.from_patch(patch, precisions=(G.BF16,)) as plan:
        _assert_rounded(plan.factors(G.MASS, G.BF16).reshape(fm.shape), fm)
        _assert_rounded(plan.factors(G.STIFFNESS, G.BF16).reshape(fk.shape), fk)
        desc = plan.describe(G.BF16)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan32:
        d32 = plan32.describe(G.FP32)
    if d == 3 and desc["tile"] == d32["tile"]:
        assert 2 * desc["factor_bytes"][1] == d32["factor_bytes"][1]


FULL_CASES = [
    (2, 2, (17, 12)), (2, 5, (17, 9)), (2, 9, (9, 10)),
    (3, 2, (17, 9, 10)), (3, 3, (17, 9, 9)), (3, 4, (9, 6, 5)),
]


@pytest.mark.parametrize("d,p,K", FULL_CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_bf16_apply_matches_rounded_factor_oracle(d, p, K, op):
    knots = [_nonuniform_knots(p, k, 30 + a) for a, k in enumerate(K)]
    patch, u = I.make_patch(d, p, list(K), noise_amp=0.2 / max(K), seed=5, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    with O.stored_factor_bits(O.BF16_BITS):
        v_bf, a_bf = oracle_full(patch, op, u)
    v_64, a_64 = oracle_full(patch, op, u)
    with G.Plan.from_patch(patch, precisions=(G.BF16,)) as plan:
        v = gpu_apply(plan, op, u, G.BF16)
    assert scaled_err(v, v_bf, a_bf, u) < tol(G.FP32, patch)
    err64 = scaled_err(v, v_64, a_64, u)
    assert 1e-6 < err64 < BF16_VS_FP64, err64


@pytest.mark.parametrize("variant", [G.KERNEL_REGISTERS, G.KERNEL_RING], ids=["registers", "ring"])
@pytest.mark.parametrize("p,K", [(3, (17, 9, 9)), (5, (9, 9, 5)), (7, (5, 5, 5))])
def test_bf16_both_factor_stream_variants(p, K, variant):
    knots = [_nonuniform_knots(p, k, 40 + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, u = I.make_patch(3, p, list(K), noise_amp=gap / 3, seed=6, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 48, seed=p)
    with O.stored_factor_bits(O.BF16_BITS):
        ref = {op: O.apply_rows(patch, op, u, rows) for op in (G.MASS, G.STIFFNESS)}
    with G.Plan.from_patch(patch, precisions=(G.BF16,), kernel_variant=variant) as plan:
        assert plan.describe(G.BF16)["kernel_variant"] == variant
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = ref[op]
            v = gpu_apply(plan, op, u, G.BF16)[rows]
            assert scaled_err(v, vr, ra.max(), u) < tol(G.FP32, patch)


@pytest.mark.parametrize("p", [2, 4, 6, 9])
def test_bf16_order_sweep_2m_dofs_sampled(p):
    """Order sweep at about 2M dofs (127 - p elements per direction), K apply."""
    patch, u = I.config_sweep(p)
    rows = sample_rows(patch, 16, seed=200 + p)
    with O.stored_factor_bits(O.BF16_BITS):
        vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    with G.Plan.from_patch(patch, precisions=(G.BF16,)) as plan:
        v = gpu_apply(plan, G.STIFFNESS, u, G.BF16)[rows]
    assert scaled_err(v, vr, ra.max(), u) < tol(G.FP32, patch)


def test_bf16_config_cube_64_p4_sampled():
    patch, u = I.config_cube(p=4, K=64)
    rows = sample_rows(patch, 128, seed=1)
    with G.Plan.from_patch(patch, precisions=(G.BF16,), default_prec=G.BF16) as plan:
        for op in (G.MASS, G.STIFFNESS):
            with O.stored_factor_bits(O.BF16_BITS):
                vr, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, G.BF16)[rows]
            assert scaled_err(v, vr, ra.max(), u) < tol(G.FP32, patch)


def test_bf16_tiny_and_single_tile_patches():
    for d, p, K in [(3, 2, (1, 1, 1)), (3, 9, (1, 1, 1)), (3, 4, (1, 2, 3)), (2, 3, (1, 1))]:
        patch, u = I.make_patch(d, p, list(K), noise_amp=0.0, seed=1)
        for op in (G.MASS, G.STIFFNESS):
            with O.stored_factor_bits(O.BF16_BITS):
                v_ref, a_inf = oracle_full(patch, op, u)
            with G.Plan.from_patch(patch, precisions=(G.BF16,)) as plan:
                v = gpu_apply(plan, op, u, G.BF16)
            assert scaled_err(v, v_ref, a_inf, u) < tol(G.FP32, patch), (d, p, K, op)
