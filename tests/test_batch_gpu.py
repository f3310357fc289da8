"""Batched multi-patch apply and the tile autotuner (GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import sample_rows, scaled_err, tol

pytestmark = pytest.mark.gpu


def _small_batch(n, seed):
    """Patches shaped like the 256-patch workload but smaller (4..14 elements)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        p = int(rng.integers(2, 7))
        K = [int(k) for k in rng.integers(4, 15, size=3)]
        out.append(I.make_patch(3, p, K, noise_amp=0.2 / max(K) / p, seed=100 + i,
                                coef_constant=float(rng.uniform(0.5, 2.0))))
    return out


@pytest.mark.parametrize("prec", [G.FP32, G.FP64, G.BF16, G.TF32, G.BF16_MMA])
def test_batch_equals_individual_applies(prec):
    import torch
    dt = torch.float64 if prec == G.FP64 else torch.float32
    patches = _small_batch(12, 3)
    # force two kernel variants on patches of the same order to get several groups
    plans = []
    for i, (pt, _) in enumerate(patches):
        kv = G.KERNEL_RING if (prec in (G.FP32, G.BF16) and i % 2) else 0
        plans.append(G.Plan.from_patch(pt, precisions=(prec,), kernel_variant=kv))
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").to(dt)
    with G.Batch(plans, op=G.STIFFNESS, prec=prec) as batch:
        assert batch.total_dofs == len(u)
        orders = {pt.orders[0] for pt, _ in patches}
        assert len(orders) <= batch.launch_groups <= 2 * len(orders)
        v = torch.empty_like(ud)
        for _ in range(2):                       # twice: the graph is replayed
            v.fill_(float("nan"))
            batch.apply(ud, v)
            torch.cuda.synchronize()
            for k, plan in enumerate(plans):
                a, b = batch.offsets[k], batch.offsets[k + 1]
                vi = torch.empty_like(ud[a:b])
                plan.apply(G.STIFFNESS, ud[a:b].clone(), vi, prec=prec)
                torch.cuda.synchronize()
                assert torch.equal(vi, v[a:b]), k
        # and against the oracle on a few rows of two patches
        for k in (0, 5):
            pt, uk = patches[k]
            rows = sample_rows(pt, 16, seed=k)
            with O.stored_factor_bits(O.BF16_BITS if prec in (G.BF16, G.BF16_MMA) else 0):
                vr, ra = O.apply_rows(pt, O.STIFFNESS, uk, rows)
            a = batch.offsets[k]
            vk = v[a:a + pt.num_dofs].double().cpu().numpy()[rows]
            assert scaled_err(vk, vr, ra.max(), uk) < tol(prec, pt)
    for plan in plans:
        assert plan.device_status() == 0
        plan.close()


def test_batch_rejects_missing_precision_and_new_vectors_rebind():
    import torch
    patches = _small_batch(3, 9)
    plans = [G.Plan.from_patch(pt, precisions=(G.FP64,)) for pt, _ in patches]
    with pytest.raises(G.IgasfError) as ei:
        G.Batch(plans, prec=G.FP32)
    assert ei.value.code == -4
    u = np.concatenate([u for _, u in patches])
    with G.Batch(plans, prec=G.FP64) as batch:
        u1 = torch.as_tensor(u, device="cuda")
        u2 = 2.0 * u1
        v1, v2 = torch.empty_like(u1), torch.empty_like(u1)
        batch.apply(u1, v1)
        batch.apply(u2, v2)            # other vectors: tables are re-bound
        torch.cuda.synchronize()
        assert torch.allclose(v2, 2.0 * v1, rtol=1e-14, atol=0)
    for plan in plans:
        plan.close()


@pytest.mark.parametrize("p", [2, 5])
def test_autotune_returns_a_built_candidate(p):
    patch, u = I.config_cube(p=p, K=24)
    tile, variant, ms = G.autotune(patch, op=G.STIFFNESS, prec=G.FP32, repeats=3)
    assert ms > 0 and variant in (G.KERNEL_REGISTERS, G.KERNEL_RING)
    with G.Plan.from_patch(patch, precisions=(G.FP32,), tile=tile, kernel_variant=variant) as plan:
        desc = plan.describe(G.FP32)
        assert desc["tile"] == tile and desc["kernel_variant"] == variant


def _persistent_plans(patches, prec):
    """Plans with the persistent tile of their order and the register-prefetch
    kernel, whose per-tile arithmetic the persistent launch runs."""
    return [G.Plan.from_patch(pt, precisions=(prec,), tile=G.batch_persistent_tile(pt.orders[0], prec),
                              kernel_variant=G.KERNEL_REGISTERS) for pt, _ in patches]


@pytest.mark.parametrize("prec", [G.FP32, G.BF16])
@pytest.mark.parametrize("op", [G.STIFFNESS, G.MASS], ids=["stiffness", "mass"])
def test_persistent_batch_equals_individual_applies(prec, op):
    import torch
    patches = _small_batch(12, 5)
    plans = _persistent_plans(patches, prec)
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    with G.Batch(plans, op=op, prec=prec, schedule=G.BATCH_PERSISTENT) as batch:
        assert batch.launch_groups == 1
        v = torch.empty_like(ud)
        for _ in range(2):
            v.fill_(float("nan"))
            batch.apply(ud, v)
            torch.cuda.synchronize()
            for k, plan in enumerate(plans):
                a, b = batch.offsets[k], batch.offsets[k + 1]
                vi = torch.empty_like(ud[a:b])
                plan.apply(op, ud[a:b].clone(), vi, prec=prec)
                torch.cuda.synchronize()
                assert torch.equal(vi, v[a:b]), k
    for plan in plans:
        assert plan.device_status() == 0
        plan.close()


def test_persistent_batch_rejects_other_tiles_and_orders():
    patch, _ = I.make_patch(3, 4, [6, 6, 6], noise_amp=0.01, seed=3)
    with G.Plan.from_patch(patch, precisions=(G.FP32,), tile=(8, 4, 2)) as plan:
        assert plan.describe(G.FP32)["tile"] != G.batch_persistent_tile(4)
        with pytest.raises(G.IgasfError) as ei:
            G.Batch([plan], prec=G.FP32, schedule=G.BATCH_PERSISTENT)
        assert ei.value.code == -4
    with pytest.raises(G.IgasfError):
        G.batch_persistent_tile(8)
    with pytest.raises(G.IgasfError):
        G.batch_persistent_tile(4, G.FP64)


@pytest.mark.parametrize("schedule", [G.BATCH_GRAPH, G.BATCH_PERSISTENT], ids=["graph", "persistent"])
def test_batch_of_the_256_patch_workload_matches_oracle_rows(schedule):
    """The batched workload itself (256 patches from seed 7, 8..48 elements per
    direction, p = 2..6): the graph with the default tiles and the persistent
    launch with its tiles, against the oracle on sampled rows of six patches of
    different orders."""
    import torch
    patches = I.config_batch()
    if schedule == G.BATCH_PERSISTENT:
        plans = _persistent_plans(patches, G.FP32)
    else:
        plans = [G.Plan.from_patch(pt, precisions=(G.FP32,)) for pt, _ in patches]
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    with G.Batch(plans, op=G.STIFFNESS, prec=G.FP32, schedule=schedule) as batch:
        v = torch.empty_like(ud)
        batch.apply(ud, v)
        torch.cuda.synchronize()
        vh = v.double().cpu().numpy()
        picks, seen = [], set()
        for k, (pt, _) in enumerate(patches):
            if pt.orders[0] not in seen:
                seen.add(pt.orders[0])
                picks.append(k)
        picks.append(len(patches) - 1)
        for k in picks:
            pt, uk = patches[k]
            rows = sample_rows(pt, 8, seed=k)
            vr, ra = O.apply_rows(pt, O.STIFFNESS, uk, rows)
            a = batch.offsets[k]
            assert scaled_err(vh[a:a + pt.num_dofs][rows], vr, ra.max(), uk) < tol(G.FP32, pt), k
    for plan in plans:
        assert plan.device_status() == 0
        plan.close()
