"""The apply entry point that allocates nothing (igasf_apply_noalloc).

Some callers must not allocate device memory when they apply the operator,
for example code that gives all device memory to its own arena and forbids
cudaMalloc/cudaFree (both can synchronize the whole device). For them the
library offers an apply whose scratch is a fixed static device array. This
test calls it through the C ABI and checks it against the regular apply,
twice in a row (the shared array keeps the previous call's contents), for
plans of different orders and tile layouts in FP64, FP32 and BF16; checks that
the device's free memory does not change across those calls, the first one
after setup included; and checks that a plan needing more scratch than the
array holds, or a call with another device current, is refused. The two applies
run the same kernels in the same order, so their results must be equal bit
for bit. It is in a file of its own, collected last, and passes alone or after
the other tests.
"""
import pytest

from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LIMIT = 64 << 20   # IGASF_NOALLOC_SCRATCH_BYTES


def _check_plan(plan, u, precs):
    import torch
    dts = {G.FP64: torch.float64, G.FP32: torch.float32, G.BF16: torch.float32}
    for prec in precs:
        assert plan.describe(prec)["workspace_bytes"] <= LIMIT
        for op in (G.STIFFNESS, G.MASS):
            ud = torch.as_tensor(u, device="cuda").to(dts[prec])
            v_ref = torch.empty_like(ud)
            plan.apply(op, ud, v_ref, prec=prec)
            outs = [torch.full_like(ud, float("nan")) for _ in range(2)]
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            for v in outs:
                plan.apply_noalloc(op, ud, v, prec=prec)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            assert free1 == free0, (prec, op, free0 - free1)
            assert plan.device_status() == 0
            for k, v in enumerate(outs):
                assert torch.equal(v, v_ref), (prec, op, k)


def test_noalloc_apply_equals_regular_apply_twice():
    # the first noalloc call right after setup allocates nothing either
    patch, u = I.config_cube(p=4, K=24)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16)) as plan:
        _check_plan(plan, u, (G.FP64, G.FP32, G.BF16))
    # other orders, sizes and tile layouts through the same shared array
    for p, K in ((6, 13), (2, 30), (9, 5)):
        patch, u = I.config_cube(p=p, K=K)
        with G.Plan.from_patch(patch, precisions=(G.FP32, G.BF16)) as plan:
            _check_plan(plan, u, (G.FP32, G.BF16))


def test_noalloc_apply_rejects_plans_beyond_the_scratch_size():
    import torch
    # p = 2 with 232^3 elements needs about 95 MB of per-tile scratch in FP32,
    # more than the 64 MiB static array
    patch, u = I.config_cube(p=2, K=232)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        assert plan.describe(G.FP32)["workspace_bytes"] > LIMIT
        ud = torch.as_tensor(u, device="cuda").float()
        v = torch.empty_like(ud)
        with pytest.raises(G.IgasfError) as ei:
            plan.apply_noalloc(G.STIFFNESS, ud, v, prec=G.FP32)
        assert ei.value.code == -4
        assert "static scratch" in str(ei.value)


def test_noalloc_apply_rejects_another_current_device():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    patch, u = I.config_cube(p=3, K=6)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        ud = torch.as_tensor(u, device="cuda:0").float()
        v = torch.empty_like(ud)
        with torch.cuda.device(1):
            with pytest.raises(G.IgasfError) as ei:
                plan.apply_noalloc(G.STIFFNESS, ud, v, prec=G.FP32)
        assert ei.value.code == -1
