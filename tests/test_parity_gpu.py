"""CUDA path vs the FP64 oracle, through the C-ABI (GPU).

Every test builds the same seeded inputs for both sides. Tolerances (scaled
max-norm error ||v - v_ref||_inf / (||A||_inf ||u||_inf)):
  FP64: 1e-12 (the exactness of sum factorization, Sec. 1 and Sec. 8: the
        factorized apply equals the assembled quadrature operator up to rounding);
  FP32: 2 (6p + 9) 2^-24 (FP32 factors, tables and arithmetic: twice the unit
        roundoff times the ~6p+9 terms of the longest accumulation chain;
        tests/gpu_helpers.py, tol).
"""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import tol, gpu_apply, oracle_full, sample_rows, scaled_err

pytestmark = pytest.mark.gpu

_CACHE = {}


def _oracle_cached(key, fn):
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


def _nonuniform_knots(p, K, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 1.5, K)
    br = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    return I.open_knots_from_breaks(p, br)


# --- row a1: univariate tables ------------------------------------------------

@pytest.mark.parametrize("p", range(2, 10))
def test_tables_match_oracle(p):
    K = (5, 3, 4)
    knots = [_nonuniform_knots(p, k, 10 + a) for a, k in enumerate(K)]
    patch, _ = I.make_patch(3, p, list(K), knots=knots)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        for a in range(3):
            nodes, weights, B, dB = plan.tables(a)
            xq, wq, Bo, dBo = O.tables_1d(knots[a], p)
            assert np.max(np.abs(nodes - xq)) < 1e-15
            assert np.max(np.abs(weights - wq)) < 1e-15
            Q = len(xq)
            e = np.arange(Q) // p
            for j in range(p):
                assert np.max(np.abs(B[:, j] - Bo[np.arange(Q), e + j])) < 1e-14
                scale = np.max(np.abs(dBo))
                assert np.max(np.abs(dB[:, j] - dBo[np.arange(Q), e + j])) < 1e-13 * scale


# --- row a2: geometry factors ------------------------------------------------

@pytest.mark.parametrize("d,p,K", [(3, 2, (9, 5, 4)), (3, 4, (5, 6, 3)), (3, 7, (3, 2, 3)),
                                   (3, 9, (2, 3, 2)), (2, 3, (17, 9)), (2, 6, (9, 4))])
def test_factors_match_oracle(d, p, K):
    knots = [_nonuniform_knots(p, k, 20 + a) for a, k in enumerate(K)]
    patch, _ = I.make_patch(d, p, list(K), noise_amp=0.2 / max(K), seed=3, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    qd = O.quad_data(patch)
    w = qd["w"]
    fm = w * qd["FM"]
    iu = np.triu_indices(d)
    fk = (w[:, None, None] * qd["FK"])[:, iu[0], iu[1]]
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        m64 = plan.factors(G.MASS, G.FP64)
        k64 = plan.factors(G.STIFFNESS, G.FP64)
        assert np.max(np.abs(m64 - fm)) < 1e-13 * np.max(np.abs(fm))
        assert np.max(np.abs(k64 - fk)) < 1e-12 * np.max(np.abs(fk))
        m32 = plan.factors(G.MASS, G.FP32)
        k32 = plan.factors(G.STIFFNESS, G.FP32)
        assert np.max(np.abs(m32 - fm) / np.abs(fm)) < 1e-7       # one FP32 rounding
        assert np.max(np.abs(k32 - fk)) < 1e-7 * np.max(np.abs(fk))


def test_factor_values_per_quad_point_coefficient():
    patch, _ = I.make_patch(3, 3, [4, 3, 5], noise_amp=0.02, seed=8)
    rng = np.random.default_rng(1)
    patch.coef_kind = I.COEF_VALUES
    patch.coef_values = rng.uniform(0.5, 2.0, patch.num_quad_points)
    qd = O.quad_data(patch)
    iu = np.triu_indices(3)
    fk = (qd["w"][:, None, None] * qd["FK"])[:, iu[0], iu[1]]
    with G.Plan.from_patch(patch) as plan:
        assert np.max(np.abs(plan.factors(G.STIFFNESS) - fk)) < 1e-12 * np.max(np.abs(fk))


@pytest.mark.parametrize("d,p,K", [(3, 2, (9, 5, 4)), (3, 5, (4, 5, 3)), (3, 9, (2, 3, 2)),
                                   (2, 3, (17, 9)), (2, 8, (5, 4))])
def test_quad_points_match_oracle(d, p, K):
    knots = [_nonuniform_knots(p, k, 50 + a) for a, k in enumerate(K)]
    patch, _ = I.make_patch(d, p, list(K), noise_amp=0.2 / max(K), seed=4, knots=knots)
    xg = O.quad_data(patch)["G"]
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        x = plan.quad_points()
    assert x.shape == (patch.num_quad_points, d)
    assert np.max(np.abs(x - xg)) < 1e-14


def test_coefficient_from_quad_points_gives_the_oracle_operator():
    # a user evaluates a(x) = exp(0.5 sin 2 pi x cos 2 pi y) at the device's
    # physical quadrature points and passes it per point; the oracle evaluates
    # the same function at its own G(x)
    patch, u = I.make_patch(3, 4, [7, 5, 6], noise_amp=0.03, seed=21,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    v_ref, a_inf = oracle_full(patch, G.STIFFNESS, u)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as probe:
        x = probe.quad_points()
    vals = np.exp(0.5 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]))
    patch.coef_kind, patch.coef_values = I.COEF_VALUES, vals
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec in (G.FP64, G.FP32):
            v = gpu_apply(plan, G.STIFFNESS, u, prec)
            assert scaled_err(v, v_ref, a_inf, u) < tol(prec, patch), prec


# --- rows a3-a7: the apply, whole vectors at sizes spanning several tiles ----

FULL_CASES = [
    # (d, p, K): K spans >= 2 tiles per direction for both precisions, with ragged tails
    (2, 2, (17, 12)), (2, 3, (16, 16)), (2, 5, (17, 9)), (2, 9, (9, 10)),
    (3, 2, (17, 9, 10)), (3, 3, (17, 9, 9)), (3, 4, (9, 6, 5)),
]


@pytest.mark.parametrize("d,p,K", FULL_CASES)
@pytest.mark.parametrize("op", [G.MASS, G.STIFFNESS], ids=["mass", "stiffness"])
def test_apply_matches_oracle_whole_vector(d, p, K, op):
    knots = [_nonuniform_knots(p, k, 30 + a) for a, k in enumerate(K)]
    patch, u = I.make_patch(d, p, list(K), noise_amp=0.2 / max(K), seed=5, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    v_ref, a_inf = _oracle_cached(("full", d, p, K, op), lambda: oracle_full(patch, op, u))
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec in (G.FP64, G.FP32):
            v = gpu_apply(plan, op, u, prec)
            err = scaled_err(v, v_ref, a_inf, u)
            assert err < tol(prec, patch), (prec, err)


def test_config_small_2d_identity_matches_csr():
    """d=2, p=3, 16x16 elements, identity geometry, a=1, FP64, u from seed 0."""
    patch, u = I.config_small_2d()
    for op in (G.MASS, G.STIFFNESS):
        v_ref, a_inf = oracle_full(patch, op, u, mode="csr")
        with G.Plan.from_patch(patch) as plan:
            v = gpu_apply(plan, op, u, G.FP64)
        assert scaled_err(v, v_ref, a_inf, u) < 1e-12


SAMPLED_CASES = [(5, (9, 9, 5)), (6, (9, 5, 5)), (7, (5, 5, 5)), (8, (5, 5, 3)), (9, (5, 3, 5))]


@pytest.mark.parametrize("p,K,fp32_tiles", [(4, 54, (None,)), (8, 24, (None, (2, 2, 2)))])
def test_whole_vector_several_full_waves(p, K, fp32_tiles):
    """Whole vectors at sizes whose default tiles make several full waves of
    resident blocks (p = 4: 14^3 = 2744 tiles of 4^3 elements, 4.5 waves of the
    FP32 kernel's 608 resident blocks; p = 8: 12^3 = 1728 tiles of 2^3 elements
    for FP64 and the FP32 2 x 2 x 2 candidate, and the default 2 x 2 x 8 tiles),
    against the oracle's point-by-point apply on all host cores."""
    patch, u = I.config_cube(p=p, K=K)
    for op in ((G.STIFFNESS, G.MASS) if p < 8 else (G.STIFFNESS,)):
        v_ref = O.apply_qp(patch, op, u)
        rows = sample_rows(patch, 64, seed=p)
        _, ra = O.apply_rows(patch, op, u, rows)
        a_inf = float(ra.max())      # lower bound of ||A||_inf: the bar is conservative
        for tile in fp32_tiles:
            precs = (G.FP64, G.FP32) if tile is None else (G.FP32,)
            with G.Plan.from_patch(patch, precisions=precs, tile=tile) as plan:
                for prec in precs:
                    v = gpu_apply(plan, op, u, prec)
                    err = scaled_err(v, v_ref, a_inf, u)
                    assert err < tol(prec, patch), (p, op, prec, tile, err)


@pytest.mark.parametrize("p,K", SAMPLED_CASES)
def test_apply_high_order_sampled_rows(p, K):
    knots = [_nonuniform_knots(p, k, 40 + a) for a, k in enumerate(K)]
    # noise below a third of the smallest Greville gap keeps G a diffeomorphism
    gap = min(np.diff(I.greville(t, p)).min() for t in knots)
    patch, u = I.make_patch(3, p, list(K), noise_amp=gap / 3, seed=6, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    rows = sample_rows(patch, 48 if p < 8 else 24, seed=p)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            for prec in (G.FP64, G.FP32):
                v = gpu_apply(plan, op, u, prec)[rows]
                assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch)


# --- the benchmark workloads at full size, sampled rows ----------------------

def test_config_cube_64_p4_sampled():
    """d=3, p=4, 64^3 elements, perturbed cube, a = exp(0.5 sin 2pi x cos 2pi y);
    FP64 and FP32 applies of K and M on 256 sampled rows."""
    patch, u = I.config_cube(p=4, K=64)
    rows = sample_rows(patch, 256, seed=1)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for op in (G.MASS, G.STIFFNESS):
            vr, ra = O.apply_rows(patch, op, u, rows)
            for prec in (G.FP64, G.FP32):
                v = gpu_apply(plan, op, u, prec)[rows]
                assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch)


@pytest.mark.parametrize("p", range(2, 10))
def test_order_sweep_2m_dofs_sampled(p):
    """Order sweep at about 2M dofs (127 - p elements per direction), K apply."""
    patch, u = I.config_sweep(p)
    nrows = 16 if p >= 8 else 32
    rows = sample_rows(patch, nrows, seed=100 + p)
    vr, ra = O.apply_rows(patch, G.STIFFNESS, u, rows)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec in (G.FP64, G.FP32):
            v = gpu_apply(plan, G.STIFFNESS, u, prec)[rows]
            assert scaled_err(v, vr, ra.max(), u) < tol(prec, patch)


# --- invariants of the CUDA path alone at full size ---------------------------

def test_invariants_config_cube():
    import torch
    patch, u = I.config_cube(p=4, K=64)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        N = plan.num_dofs
        one = torch.ones(N, dtype=torch.float64, device="cuda")
        out = torch.empty_like(one)
        plan.apply(G.STIFFNESS, one, out)
        k1 = out.abs().max().item()
        rng = np.random.default_rng(2)
        a = torch.as_tensor(rng.uniform(-1, 1, N), device="cuda")
        b = torch.as_tensor(rng.uniform(-1, 1, N), device="cuda")
        ka, kb = torch.empty_like(a), torch.empty_like(b)
        plan.apply(G.STIFFNESS, a, ka)
        plan.apply(G.STIFFNESS, b, kb)
        sym = abs((b @ ka).item() - (a @ kb).item()) / abs((b @ ka).item())
        plan.apply(G.MASS, one, out)
        vol = out.sum().item()
        fm = plan.factors(G.MASS)
        ka_max = ka.abs().max().item()
    # K 1 = 0, K symmetric, 1^T M 1 = sum_x w |det J| = volume of the cube up to quadrature error
    assert k1 < 1e-12 * ka_max
    assert sym < 1e-12
    assert abs(vol - fm.sum()) < 1e-12
    assert abs(vol - 1.0) < 1e-6


# --- edge cases and determinism -----------------------------------------------

@pytest.mark.parametrize("d,p,K", [(3, 2, (1, 1, 1)), (3, 4, (1, 2, 3)), (3, 9, (1, 1, 1)),
                                   (3, 5, (3, 1, 2)), (2, 7, (1, 1)), (2, 2, (1, 30))])
def test_tiny_patches_single_partial_tile(d, p, K):
    patch, u = I.make_patch(d, p, list(K), noise_amp=0.05, seed=12,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for op in (G.MASS, G.STIFFNESS):
            v_ref, a_inf = oracle_full(patch, op, u, mode="csr")
            for prec in (G.FP64, G.FP32):
                assert scaled_err(gpu_apply(plan, op, u, prec), v_ref, a_inf, u) < tol(prec, patch)


def test_apply_is_cuda_graph_capturable():
    """igasf_apply allocates nothing and never synchronizes with the host, so a
    caller can capture it (tile kernel, then the gather with its programmatic
    launch) into a CUDA graph: replays equal direct applies bit for bit, also
    after the input buffer's values change."""
    import torch
    patch, u = I.make_patch(3, 4, [9, 6, 5], noise_amp=0.02, seed=5,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    precs = (G.FP64, G.FP32, G.BF16, G.TF32, G.BF16_MMA)
    with G.Plan.from_patch(patch, precisions=precs) as plan:
        for prec in precs:
            dt = torch.float64 if prec == G.FP64 else torch.float32
            for op in (G.MASS, G.STIFFNESS):
                ud = torch.as_tensor(u, device="cuda").to(dt)
                v = torch.full_like(ud, float("nan"))
                s = torch.cuda.Stream()
                s.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(s):
                    plan.apply(op, ud, v, prec=prec)      # warm-up outside the capture
                torch.cuda.current_stream().wait_stream(s)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    plan.apply(op, ud, v, prec=prec)
                for scale in (1.0, -0.5):
                    ud.mul_(scale)
                    v_ref = torch.empty_like(ud)
                    plan.apply(op, ud, v_ref, prec=prec)
                    v.fill_(float("nan"))
                    g.replay()
                    torch.cuda.synchronize()
                    assert torch.equal(v, v_ref), (prec, op, scale)
                assert plan.device_status() == 0
                del g


def test_apply_is_deterministic_and_host_path_matches():
    import torch
    patch, u = I.config_cube(p=3, K=20)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec, dt, npdt in ((G.FP64, torch.float64, np.float64), (G.FP32, torch.float32, np.float32)):
            ud = torch.as_tensor(u, device="cuda").to(dt)
            v1, v2 = torch.empty_like(ud), torch.empty_like(ud)
            plan.apply(G.STIFFNESS, ud, v1, prec=prec)
            plan.apply(G.STIFFNESS, ud, v2, prec=prec)
            torch.cuda.synchronize()
            assert torch.equal(v1, v2)
            uh = torch.as_tensor(u.astype(npdt)).pin_memory()
            vh = torch.empty_like(uh).pin_memory()
            plan.apply_host(G.STIFFNESS, uh, vh, prec=prec)      # pinned v: written directly
            assert torch.equal(vh, v1.cpu())
            un = u.astype(npdt)
            vn = np.full_like(un, np.nan)                        # pageable v: staged copy
            plan.apply_host(G.STIFFNESS, un, vn, prec=prec)
            assert np.array_equal(vn, v1.cpu().numpy())


def test_async_host_apply_sequence_equals_device_applies():
    """A sequence of asynchronous host-buffer applies (input copies overlapping
    the previous apply, two alternating input buffers) gives each vector's own
    device apply bit for bit, for a page-locked v (written through its mapping)
    and a pageable one (copied back)."""
    import torch
    patch, _ = I.config_cube(p=3, K=12)
    rng = np.random.default_rng(3)
    us = [rng.uniform(-1, 1, patch.num_dofs).astype(np.float32) for _ in range(5)]
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        refs = []
        for u in us:
            ud = torch.as_tensor(u, device="cuda")
            vd = torch.empty_like(ud)
            plan.apply(G.STIFFNESS, ud, vd, prec=G.FP32)
            refs.append(vd.cpu())
        stream = torch.cuda.current_stream()
        uhs = [torch.as_tensor(u).pin_memory() for u in us]
        vhs = [torch.full_like(uh, float("nan")).pin_memory() for uh in uhs]
        for uh, vh in zip(uhs, vhs):
            plan.apply_host_async(G.STIFFNESS, uh, vh, prec=G.FP32, stream=stream)
        stream.synchronize()
        for vh, ref in zip(vhs, refs):
            assert torch.equal(vh, ref)
        vns = [np.full(patch.num_dofs, np.nan, dtype=np.float32) for _ in us]
        for u, vn in zip(us, vns):
            plan.apply_host_async(G.STIFFNESS, u, vn, prec=G.FP32, stream=stream)
        stream.synchronize()
        for vn, ref in zip(vns, refs):
            assert np.array_equal(vn, ref.numpy())


def test_default_precision_apply():
    import torch
    patch, u = I.config_cube(p=2, K=9)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        ud = torch.as_tensor(u, device="cuda").float()
        v1, v2 = torch.empty_like(ud), torch.empty_like(ud)
        plan.apply_default(G.STIFFNESS, ud, v1)
        plan.apply(G.STIFFNESS, ud, v2, prec=G.FP32)
        torch.cuda.synchronize()
        assert torch.equal(v1, v2)
        with pytest.raises(G.IgasfError) as ei:
            plan.apply(G.STIFFNESS, ud.double(), v1.double(), prec=G.FP64)
        assert ei.value.code == -4


def test_apply_argument_errors():
    import torch
    patch, u = I.config_cube(p=2, K=9)
    with G.Plan.from_patch(patch, precisions=(G.FP64,)) as plan:
        ud = torch.as_tensor(u, device="cuda")
        big = torch.zeros(2 * len(u) + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(G.IgasfError) as ei:      # misaligned
            plan.apply(G.STIFFNESS, ud, _misaligned(big, len(u)))
        assert ei.value.code == -1
        with pytest.raises(G.IgasfError) as ei:      # overlap
            plan.apply(G.STIFFNESS, big[:len(u)], big[len(u) // 2:len(u) // 2 + len(u)])
        assert ei.value.code == -1
        with pytest.raises(G.IgasfError) as ei:      # bad op
            plan.apply(5, ud, torch.empty_like(ud))
        assert ei.value.code == -1


class _misaligned:
    """A fake tensor whose data pointer is off by 4 bytes."""

    def __init__(self, base, n):
        self.base = base

    def data_ptr(self):
        return self.base.data_ptr() + 4


def test_setup_rejects_inverted_geometry():
    patch, u = I.make_patch(3, 3, 4)
    patch.ctrl[:, 0] = -patch.ctrl[:, 0]   # mirror: det J < 0 everywhere
    with pytest.raises(G.IgasfError) as ei:
        G.Plan.from_patch(patch)
    assert ei.value.code == -3
