"""The split-lane FP32/BF16 tile kernel (three lanes per pencil pair in the
stiffness' phase C, factors and partial derivatives exchanged by warp
shuffles) against the oracle, through the C-ABI (GPU). Same operator as the
other FP32 kernels, same bar (1e-5 scaled max-norm; BF16 against the oracle's
rounded-factor operator)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import TOL, gpu_apply, oracle_full, sample_rows, scaled_err

pytestmark = pytest.mark.gpu


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


def _patch(p, K, seed):
    knots = [_nonuniform_knots(p, k, seed + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    return I.make_patch(3, p, list(K), noise_amp=min(0.2 / max(K), gap / 3), seed=seed, knots=knots,
                        coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)


CASES = [(4, (9, 6, 5)), (5, (9, 5, 5)), (6, (5, 5, 3))]
SAMPLED = [(7, (5, 3, 5)), (8, (3, 3, 3)), (9, (3, 2, 3))]


@pytest.mark.parametrize("p,K", CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_split_matches_oracle_whole_vector(p, K, op):
    patch, u = _patch(p, K, 110 + p)
    v_ref, a_inf = oracle_full(patch, op, u)
    with O.stored_factor_bits(O.BF16_BITS):
        v_bf, a_bf = oracle_full(patch, op, u)
    with G.Plan.from_patch(patch, precisions=(G.FP32, G.BF16), kernel_variant=G.KERNEL_SPLIT) as plan:
        assert plan.describe(G.FP32)["kernel_variant"] == G.KERNEL_SPLIT
        v = gpu_apply(plan, op, u, G.FP32)
        assert scaled_err(v, v_ref, a_inf, u) < TOL[G.FP32]
        v = gpu_apply(plan, op, u, G.BF16)
        assert scaled_err(v, v_bf, a_bf, u) < TOL[G.FP32]


@pytest.mark.parametrize("p,K", SAMPLED)
def test_split_high_order_sampled_rows(p, K):
    """Orders 7-9: rows on corners, edges, faces and the interior (the oracle's
    whole vector costs p^9 per row)."""
    patch, u = _patch(p, K, 110 + p)
    rows = sample_rows(patch, 24, seed=p)
    with G.Plan.from_patch(patch, precisions=(G.FP32, G.BF16), kernel_variant=G.KERNEL_SPLIT) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, G.FP32)[rows]
            assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]
            with O.stored_factor_bits(O.BF16_BITS):
                vr, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, G.BF16)[rows]
            assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]


@pytest.mark.parametrize("p", [4, 6, 9])
def test_split_order_sweep_2m_dofs_sampled(p):
    patch, u = I.config_sweep(p)
    rows = sample_rows(patch, 16, seed=400 + p)
    vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    with G.Plan.from_patch(patch, precisions=(G.FP32,), kernel_variant=G.KERNEL_SPLIT) as plan:
        v = gpu_apply(plan, G.STIFFNESS, u, G.FP32)[rows]
    assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]


def test_split_batched_equals_individual():
    import torch
    patches = [_patch(p, K, 130 + i) for i, (p, K) in enumerate([(4, (5, 4, 3)), (6, (3, 3, 4)),
                                                                  (6, (4, 2, 3)), (9, (2, 2, 3))])]
    plans = [G.Plan.from_patch(pt, precisions=(G.FP32,), kernel_variant=G.KERNEL_SPLIT)
             for pt, _ in patches]
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    with G.Batch(plans, op=G.STIFFNESS, prec=G.FP32) as batch:
        v = torch.empty_like(ud)
        batch.apply(ud, v)
        torch.cuda.synchronize()
        for k, plan in enumerate(plans):
            a, b = batch.offsets[k], batch.offsets[k + 1]
            vi = torch.empty_like(ud[a:b])
            plan.apply(G.STIFFNESS, ud[a:b].clone(), vi, prec=G.FP32)
            torch.cuda.synchronize()
            assert torch.equal(vi, v[a:b]), k
    for plan in plans:
        plan.close()
