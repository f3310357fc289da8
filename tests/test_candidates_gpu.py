"""Every compiled tile-kernel candidate against the oracle (GPU).

The library lists, per (d, p, precision), the tile shapes and factor-stream
variants it was built with (`igasf_list_kernels`); the first is the default and
the autotuner may return any of them, so each one has to meet the parity bar,
not only the defaults. Per order and dimension one patch spans at least two
tiles of the largest candidate in every direction with a ragged last tile
(non-uniform knots, perturbed geometry, a = exp(0.5 sin 2 pi x cos 2 pi y)); every
candidate applies M and K to the same u and is compared on sampled rows (corners,
edges, faces, interior) with the oracle: FP32 against the FP64 operator, BF16
against the operator with bfloat16-rounded factors (both at the FP32 bar,
1e-5 scaled max-norm), the on-the-fly FP32 kernels against the FP64 operator.
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import tol, gpu_apply, sample_rows, scaled_err

pytestmark = pytest.mark.gpu


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


def _candidates(d, p):
    """[(prec, geometry, tile, variant)] for every compiled candidate."""
    out = []
    for prec in (G.FP32, G.BF16):
        for tile, variant in G.list_kernels(d, p, prec):
            out.append((prec, G.GEOMETRY_STORED, tile[:d], variant))
    if d == 3:
        for tile, variant in G.list_kernels(d, p, G.FP32, G.GEOMETRY_ON_THE_FLY):
            out.append((G.FP32, G.GEOMETRY_ON_THE_FLY, tile[:d], variant))
    return out


@pytest.mark.parametrize("d,p", [(3, p) for p in range(2, 10)] + [(2, p) for p in range(2, 10)])
def test_every_candidate_matches_oracle(d, p):
    cands = _candidates(d, p)
    assert cands, "no kernel compiled for d=%d p=%d" % (d, p)
    K = [2 * max(c[2][a] for c in cands) + 1 for a in range(d)]
    knots = [_nonuniform_knots(p, k, 60 + a) for a, k in enumerate(K)]
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, u = I.make_patch(d, p, K, noise_amp=gap / 3, seed=8, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 24 if p >= 8 else 40, seed=300 + p)
    ops = (G.MASS, G.STIFFNESS)
    ref = {op: O.apply_rows(patch, op, u, rows) for op in ops}
    with O.stored_factor_bits(O.BF16_BITS):
        ref_bf = {op: O.apply_rows(patch, op, u, rows) for op in ops}
    for prec, geometry, tile, variant in cands:
        kv = variant if geometry == G.GEOMETRY_STORED else 0
        with G.Plan.from_patch(patch, precisions=(prec,), tile=tile, kernel_variant=kv,
                               geometry=geometry) as plan:
            desc = plan.describe(prec)
            assert desc["tile"][:d] == tile and desc["kernel_variant"] == variant
            for op in ops:
                vr, ra = (ref_bf if prec == G.BF16 else ref)[op]
                v = gpu_apply(plan, op, u, prec)[rows]
                err = scaled_err(v, vr, ra.max(), u)
                assert err < tol(G.FP32, patch), (prec, geometry, tile, variant, op, err)
