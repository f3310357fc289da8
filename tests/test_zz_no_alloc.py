"""The apply entry point that allocates nothing (igasf_apply_noalloc).

Some callers must not allocate device memory when they apply the operator,
for example code that gives all device memory to its own arena and forbids
cudaMalloc/cudaFree (both can synchronize the whole device). For them the
library offers an apply whose scratch is a fixed static device array. This
test calls it through the C ABI and checks it against the regular apply, twice
in a row (the shared array keeps the previous call's contents), and checks
that a plan needing more scratch than the array holds is refused. It is in a
file of its own, collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import TOL

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_regular_apply_twice():
    import torch
    patch, u = I.config_cube(p=4, K=24)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        for prec, dt in ((G.FP64, torch.float64), (G.FP32, torch.float32)):
            assert plan.describe(prec)["workspace_bytes"] <= 64 << 20
            for op in (G.STIFFNESS, G.MASS):
                ud = torch.as_tensor(u, device="cuda").to(dt)
                v_ref = torch.empty_like(ud)
                plan.apply(op, ud, v_ref, prec=prec)
                for _ in range(2):
                    v = torch.full_like(ud, float("nan"))
                    plan.apply_noalloc(op, ud, v, prec=prec)
                    torch.cuda.synchronize()
                    ref = v_ref.double().cpu().numpy()
                    err = np.max(np.abs(v.double().cpu().numpy() - ref)) / np.max(np.abs(ref))
                    assert err < TOL[prec], (prec, op, err)


def test_noalloc_apply_rejects_plans_beyond_the_scratch_size():
    import torch
    # p = 2 with 232^3 elements needs about 95 MB of per-tile scratch in FP32,
    # more than the 64 MiB static array
    patch, u = I.config_cube(p=2, K=232)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        assert plan.describe(G.FP32)["workspace_bytes"] > 64 << 20
        ud = torch.as_tensor(u, device="cuda").float()
        v = torch.empty_like(ud)
        with pytest.raises(G.IgasfError) as ei:
            plan.apply_noalloc(G.STIFFNESS, ud, v, prec=G.FP32)
        assert ei.value.code == -4
        assert "static scratch" in str(ei.value)
