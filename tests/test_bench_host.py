"""Host-side pieces of the benchmark (CPU only): the reference arm prints the
same config as the GPU arm, and the full-size CSR of the CPU baseline is made
of the oracle's sample rows in order."""
import argparse
import contextlib
import io
import json

import numpy as np

import oracle as O
from paper_1809_05471_gb300 import inputs as I


def _args(**kw):
    base = dict(p=4, elements=8, op="stiffness", steps=2, warmup=1, gpus=1, prec="fp32", dim=3)
    base.update(kw)
    return argparse.Namespace(**base)


def test_reference_arm_prints_the_gpu_arm_config(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    out = io.StringIO()
    args = _args()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args)
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.bench_config(args, 1)
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle CSR SpMV" and line["value"] > 0


def test_full_size_csr_repeats_the_sample_rows():
    import bench
    patch, u = I.config_cube(p=3, K=5)
    rows = np.arange(30, 70, dtype=np.int64)
    rp, ci, va = O.assemble_rows(patch, O.STIFFNESS, rows)
    big = bench.full_size_csr(rp, ci, va, 95)
    assert len(big[0]) == 96
    y = O.spmv(*big, u)
    ys = O.spmv(rp, ci, va, u)
    assert np.array_equal(y, np.tile(ys, 3)[:95])


def test_algorithmic_bytes_are_the_stated_per_unit_figures():
    # the roofline's bytes per launch: every stored factor once, u once, v once;
    # per quadrature point and per dof as stated for each precision and operator
    import bench
    per_qp = {("stiffness", "fp32"): 24, ("stiffness", "fp64"): 48, ("stiffness", "bf16"): 12,
              ("mass", "fp32"): 4, ("mass", "fp64"): 8, ("mass", "bf16"): 2}
    per_dof = {"fp32": 8, "fp64": 16, "bf16": 8}
    for (op, prec), b in per_qp.items():
        assert bench.algorithmic_bytes(op, prec, 1, 0) == b, (op, prec)
        assert bench.algorithmic_bytes(op, prec, 0, 1) == per_dof[prec], (op, prec)
    assert bench.algorithmic_bytes("stiffness", "fp32", 1, 0, d=2) == 12   # 3 fields in 2D
    # the 64^3, p = 4 headline: 256^3 Gauss points and 67^3 dofs
    assert bench.algorithmic_bytes("stiffness", "fp32", 256 ** 3, 67 ** 3) == 405059288
