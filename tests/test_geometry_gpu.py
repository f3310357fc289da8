"""FP32 applies that evaluate the factors w F inside the tile kernel from the
control points (Sec. 6.2), against the FP64 oracle, through the C-ABI (GPU).

Same operator as the stored-factor path, so the same bar: 1e-5 scaled max-norm
error (the geometry, det J, the cofactors and the coefficient are FP32 here:
a few ulp of FP32 per factor, well inside the bar for the well-shaped patches
used)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import TOL, gpu_apply, oracle_full, sample_rows, scaled_err

pytestmark = pytest.mark.gpu

ON_THE_FLY = dict(precisions=(G.FP32,), geometry=G.GEOMETRY_ON_THE_FLY)


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


def _patch(p, K, seed, coef_kind=I.COEF_EXP_SIN_COS):
    knots = [_nonuniform_knots(p, k, seed + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    return I.make_patch(3, p, list(K), noise_amp=min(0.2 / max(K), gap / 3), seed=seed, knots=knots,
                        coef_kind=coef_kind, coef_alpha=0.5, coef_constant=1.7)


CASES = [(2, (17, 9, 10)), (3, (17, 9, 9)), (4, (9, 6, 5)), (5, (9, 5, 5)), (6, (5, 5, 3))]
SAMPLED = [(7, (5, 3, 3)), (8, (3, 3, 3)), (9, (3, 2, 3))]


@pytest.mark.parametrize("p,K", CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_on_the_fly_matches_oracle_whole_vector(p, K, op):
    patch, u = _patch(p, K, 70 + p)
    v_ref, a_inf = oracle_full(patch, op, u)
    with G.Plan.from_patch(patch, **ON_THE_FLY) as plan:
        d = plan.describe(G.FP32)
        assert d["kernel_variant"] == G.KERNEL_ON_THE_FLY
        assert d["factor_bytes"] == [0, 0]
        v = gpu_apply(plan, op, u, G.FP32)
    assert scaled_err(v, v_ref, a_inf, u) < TOL[G.FP32]


@pytest.mark.parametrize("p,K", SAMPLED)
def test_on_the_fly_high_order_sampled_rows(p, K):
    patch, u = _patch(p, K, 70 + p)
    rows = sample_rows(patch, 24, seed=p)
    with G.Plan.from_patch(patch, **ON_THE_FLY) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, G.FP32)[rows]
            assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]


@pytest.mark.parametrize("p,second", [(3, [4, 4, 4]), (5, [2, 2, 2])])
def test_on_the_fly_constant_coefficient_and_second_tile(p, second):
    patch, u = _patch(p, (9, 7, 6), 90 + p, coef_kind=I.COEF_CONSTANT)
    v_ref, a_inf = oracle_full(patch, G.STIFFNESS, u)
    for tile in (None, second):
        with G.Plan.from_patch(patch, tile=tile, **ON_THE_FLY) as plan:
            if tile is not None:
                assert plan.describe(G.FP32)["tile"] == second
            v = gpu_apply(plan, G.STIFFNESS, u, G.FP32)
        assert scaled_err(v, v_ref, a_inf, u) < TOL[G.FP32]


def test_on_the_fly_config_cube_64_p4_sampled():
    patch, u = I.config_cube(p=4, K=64)
    rows = sample_rows(patch, 128, seed=1)
    with G.Plan.from_patch(patch, **ON_THE_FLY) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            v = gpu_apply(plan, op, u, G.FP32)[rows]
            assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]


@pytest.mark.parametrize("p", [2, 5, 9])
def test_on_the_fly_order_sweep_2m_dofs_sampled(p):
    patch, u = I.config_sweep(p)
    rows = sample_rows(patch, 16, seed=300 + p)
    vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    with G.Plan.from_patch(patch, **ON_THE_FLY) as plan:
        v = gpu_apply(plan, G.STIFFNESS, u, G.FP32)[rows]
    assert scaled_err(v, vr, ra.max(), u) < TOL[G.FP32]


def test_on_the_fly_with_stored_fp64_solver_and_limits():
    """FP64 stays stored beside an on-the-fly FP32 variant: the refined solver
    uses both; the FP32 variant has no factors to export and no batched form."""
    import torch
    patch, u = I.config_cube(p=3, K=8)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32),
                           geometry=G.GEOMETRY_ON_THE_FLY) as plan:
        assert plan.describe(G.FP64)["kernel_variant"] != G.KERNEL_ON_THE_FLY
        b = torch.as_tensor(np.random.default_rng(2).uniform(-1, 1, plan.num_dofs), device="cuda")
        x = torch.zeros_like(b)
        rep = plan.cg_solve(b, x, inner_prec=G.FP32, rtol=1e-10)
        assert rep["converged"] and rep["outer_iterations"] >= 2
        with pytest.raises(G.IgasfError) as ei:
            plan.factors(G.STIFFNESS, G.FP32)
        assert ei.value.code == -4
        with pytest.raises(G.IgasfError) as ei:
            G.Batch([plan], op=G.STIFFNESS, prec=G.FP32)
        assert ei.value.code == -4
        assert plan.device_status() == 0
