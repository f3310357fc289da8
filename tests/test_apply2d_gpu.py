"""2D applies against the FP64 oracle through the C-ABI (GPU): the packed
FP32x2 kernel (wide tiles along direction 1) on patches spanning at least two
tiles per direction with ragged tails, both tile shapes of each order, the
scalar candidate selected by its tile, and bfloat16-stored factors. FP32 bar:
1e-5 scaled max-norm (BF16 against the oracle's rounded-factor operator)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import tol, gpu_apply, oracle_full, sample_rows, scaled_err

pytestmark = pytest.mark.gpu

# default tile per order (S1, S2): the packed kernel, the scalar one (8 x 8) at p = 9
TILE = {2: (32, 8), 3: (64, 8), 4: (16, 8), 5: (32, 8), 6: (32, 4), 7: (32, 4), 8: (16, 4), 9: (8, 8)}
SECOND = {2: (64, 8), 3: (32, 8), 4: (32, 8), 5: (64, 4), 6: (16, 8), 7: (16, 4), 8: (8, 4), 9: (32, 4)}


def _patch(p, K, seed):
    rng = np.random.default_rng(seed)
    knots = []
    for a, k in enumerate(K):
        h = rng.uniform(0.5, 1.5, k)
        knots.append(I.open_knots_from_breaks(p, np.concatenate([[0.0], np.cumsum(h) / h.sum()])))
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    return I.make_patch(2, p, list(K), noise_amp=min(0.2 / max(K), gap / 3), seed=seed, knots=knots,
                        coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_packed_2d_matches_oracle_whole_vector(p, op):
    S1, S2 = TILE[p]
    K = (2 * S1 + 3, 2 * S2 + 1)                  # three tiles per direction, ragged last
    patch, u = _patch(p, K, 200 + p)
    v_ref, a_inf = oracle_full(patch, op, u)
    with O.stored_factor_bits(O.BF16_BITS):
        v_bf, a_bf = oracle_full(patch, op, u)
    for tile in (None, list(SECOND[p]), [8, 8]):
        with G.Plan.from_patch(patch, precisions=(G.FP32, G.BF16), tile=tile) as plan:
            d = plan.describe(G.FP32)
            assert d["tile"][:2] == list(TILE[p] if tile is None else tile)
            v = gpu_apply(plan, op, u, G.FP32)
            assert scaled_err(v, v_ref, a_inf, u) < tol(G.FP32, patch), tile
            v = gpu_apply(plan, op, u, G.BF16)
            assert scaled_err(v, v_bf, a_bf, u) < tol(G.FP32, patch), tile


@pytest.mark.parametrize("p", [7, 8, 9])
def test_packed_2d_high_order_sampled(p):
    S1, S2 = TILE[p]
    patch, u = _patch(p, (2 * S1 + 3, 2 * S2 + 1), 210 + p)
    rows = sample_rows(patch, 32, seed=p)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            for prec in (G.FP64, G.FP32):
                v = gpu_apply(plan, op, u, prec)[rows]
                assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch)


def test_packed_2d_large_square_sampled():
    """About 4.2M dofs at p = 4: the size `bench.py --dim 2` measures."""
    p, K = 4, 2044
    gap = float(np.diff(I.greville(I.open_uniform_knots(p, K), p)).min())
    patch, u = I.make_patch(2, p, K, noise_amp=min(0.2 / K, gap / 3), seed=0,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 64, seed=9)
    vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        v = gpu_apply(plan, G.STIFFNESS, u, G.FP32)[rows]
    assert scaled_err(v, vr, ra.max(), u) < tol(G.FP32, patch)
