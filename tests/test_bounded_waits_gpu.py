"""Bounded device waits (GPU): the FP32 tile kernel receives its factor slabs
by bulk copies and waits on shared-memory barriers; every wait has a limit.
A test hook makes tile 0 never receive one slab: the wait must run out, the
kernel must return, the plan's status word must report IGASF_ERR_TIMEOUT, and
the next apply without the fault must be correct again. No GPU fault, trap or
hang is involved: the missing slab is simply never requested."""
import numpy as np
import pytest

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I
from tests.gpu_helpers import tol, oracle_full, scaled_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [G.FP32, G.BF16], ids=["fp32", "bf16"])
def test_missing_slab_times_out_and_reports_status(prec):
    import torch
    patch, u = I.config_cube(p=4, K=9)
    with O.stored_factor_bits(O.BF16_BITS if prec == G.BF16 else 0):
        v_ref, a_inf = oracle_full(patch, G.STIFFNESS, u)
    with G.Plan.from_patch(patch, precisions=(prec,), kernel_variant=G.KERNEL_RING) as plan:
        assert plan.describe(prec)["kernel_variant"] == G.KERNEL_RING
        ud = torch.as_tensor(u, device="cuda").float()
        v = torch.empty_like(ud)
        assert plan.device_status() == 0
        plan.set_test_fault(skip_slab=3, wait_limit_cycles=200000)
        plan.apply(G.STIFFNESS, ud, v, prec=prec)
        assert plan.device_status(clear=True) == -7          # IGASF_ERR_TIMEOUT
        assert plan.device_status() == 0                     # cleared
        plan.set_test_fault(skip_slab=-1)
        for apply in (plan.apply, plan.apply_noalloc):
            apply(G.STIFFNESS, ud, v, prec=prec)
            assert plan.device_status() == 0
            assert scaled_err(v.double().cpu().numpy(), v_ref, a_inf, u) < tol(G.FP32, patch)


def test_fault_hook_argument_check():
    patch, u = I.config_cube(p=2, K=4)
    with G.Plan.from_patch(patch, precisions=(G.FP32,)) as plan:
        with pytest.raises(G.IgasfError) as ei:
            plan.set_test_fault(skip_slab=0, wait_limit_cycles=10)
        assert ei.value.code == -1
