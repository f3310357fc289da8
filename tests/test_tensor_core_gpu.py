"""The tensor-core precisions against the oracle (GPU).

IGASF_TF32 (FP32 factors, direction-3 contractions on the tensor cores with
TF32 operands and FP32 accumulation) is compared with the FP64 operator;
IGASF_BF16_MMA (bfloat16-stored factors, direction-3 contractions with bfloat16
operands) with the oracle's operator whose factors are rounded to bfloat16, so
that the test sees the error of the tensor-core arithmetic itself. The bar,
4u plus the FP32 bar (u the operand format's unit roundoff), is the first-order
bound of tests/gpu_helpers.py, tol. Every compiled candidate is checked (the
autotuner may return any), on multi-tile patches with ragged tiles in every
direction, whole vectors and sampled rows of the order-sweep workload.
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import gpu_apply, sample_rows, scaled_err, tol

pytestmark = pytest.mark.gpu

TC = (G.TF32, G.BF16_MMA)


def _bits(prec):
    return O.BF16_BITS if prec == G.BF16_MMA else 0


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


@pytest.mark.parametrize("p", range(2, 10))
def test_every_tensor_core_candidate_matches_oracle(p):
    cands = [(prec, tuple(t), v) for prec in TC for t, v in G.list_kernels(3, p, prec)]
    assert len(cands) >= 2 and all(v == G.KERNEL_MMA for _, _, v in cands)
    K = [2 * max(c[1][a] for c in cands) + 1 for a in range(3)]
    knots = [_nonuniform_knots(p, k, 80 + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, u = I.make_patch(3, p, K, noise_amp=gap / 3, seed=11, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 24 if p >= 8 else 40, seed=400 + p)
    ref = {}
    for bits in (0, O.BF16_BITS):
        with O.stored_factor_bits(bits):
            for op in (G.MASS, G.STIFFNESS):
                ref[bits, op] = O.apply_rows(patch, op, u, rows)
    for prec, tile, variant in cands:
        with G.Plan.from_patch(patch, precisions=(prec,), tile=tile) as plan:
            desc = plan.describe(prec)
            assert tuple(desc["tile"]) == tile and desc["kernel_variant"] == G.KERNEL_MMA
            for op in (G.MASS, G.STIFFNESS):
                vr, ra = ref[_bits(prec), op]
                v = gpu_apply(plan, op, u, prec)[rows]
                err = scaled_err(v, vr, ra.max(), u)
                assert err < tol(prec, patch), (prec, tile, op, err)


@pytest.mark.parametrize("p,K", [(2, (17, 9, 10)), (3, (9, 10, 9)), (4, (9, 6, 11)),
                                 (6, (5, 5, 17)), (7, (3, 5, 9)), (9, (5, 3, 13))])
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_tensor_core_whole_vector(p, K, op):
    knots = [_nonuniform_knots(p, k, 90 + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, u = I.make_patch(3, p, list(K), noise_amp=gap / 3, seed=13, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 32, seed=p)
    with G.Plan.from_patch(patch, precisions=TC) as plan:
        for prec in TC:
            with O.stored_factor_bits(_bits(prec)):
                v_ref = O.apply_qp(patch, op, u)
                _, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, prec)
            err = scaled_err(v, v_ref, float(ra.max()), u)
            assert err < tol(prec, patch), (prec, err)


@pytest.mark.parametrize("p", [2, 4, 6, 9])
def test_tensor_core_order_sweep_2m_dofs_sampled(p):
    patch, u = I.config_sweep(p)
    rows = sample_rows(patch, 16 if p >= 8 else 32, seed=500 + p)
    with G.Plan.from_patch(patch, precisions=TC) as plan:
        for prec in TC:
            with O.stored_factor_bits(_bits(prec)):
                vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
            v = gpu_apply(plan, G.STIFFNESS, u, prec)[rows]
            assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch), prec


def test_tensor_core_config_cube_64_p4_sampled_and_deterministic():
    import torch
    patch, u = I.config_cube(p=4, K=64)
    rows = sample_rows(patch, 128, seed=7)
    with G.Plan.from_patch(patch, precisions=TC) as plan:
        for prec in TC:
            for op in (G.MASS, G.STIFFNESS):
                with O.stored_factor_bits(_bits(prec)):
                    vr, ra = O.apply_rows(patch, op, u, rows)
                ud = torch.as_tensor(u, device="cuda").float()
                v1, v2 = torch.empty_like(ud), torch.empty_like(ud)
                plan.apply(op, ud, v1, prec=prec)
                plan.apply(op, ud, v2, prec=prec)
                torch.cuda.synchronize()
                assert torch.equal(v1, v2)
                v = v1.double().cpu().numpy()[rows]
                assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch), (prec, op)


def test_tensor_core_tiny_patches_and_rejections():
    for p, K in ((2, (1, 1, 1)), (5, (1, 2, 3)), (9, (1, 1, 2))):
        patch, u = I.make_patch(3, p, list(K), noise_amp=0.03, seed=2,
                                coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
        with G.Plan.from_patch(patch, precisions=TC) as plan:
            for prec in TC:
                for op in (G.MASS, G.STIFFNESS):
                    with O.stored_factor_bits(_bits(prec)):
                        rp, ci, va = O.assemble_csr(patch, op)
                    v = gpu_apply(plan, op, u, prec)
                    assert scaled_err(v, O.spmv(rp, ci, va, u), O.csr_inf_norm(rp, va), u) \
                        < tol(prec, patch), (p, K, prec, op)
    # two dimensions have no tensor-core kernel
    patch, _ = I.make_patch(2, 3, 6)
    with pytest.raises(G.IgasfError) as ei:
        G.Plan.from_patch(patch, precisions=(G.TF32,))
    assert ei.value.code == -4
