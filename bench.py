#!/usr/bin/env python
"""Benchmark of the matrix-free sum-factorized stiffness apply (GDoF/s).

Workload (default): d = 3 perturbed unit cube, order p = 4, 64^3 elements
(67^3 = 300,763 dofs, 256^3 Gauss points), a(x) = exp(0.5 sin 2 pi x cos 2 pi y),
stiffness apply in FP32. One step = one apply v = K u (tile kernel + gather) with
u, v and the factors resident in HBM. Factors (403 MB in FP32) exceed the L2
(129 MB), so no flush is needed between steps.

Also reported: the FP64 stiffness apply and both mass applies, the end-to-end
rate through the host-buffer C-ABI call, the roofline of the tile kernel (its
CUDA-event time on the launching stream over the timed region), the FP64 oracle
timed on the host cores on a bounded sample of rows (and compared with the GPU
result on those rows), and the SM clocks sampled during the timed region.

With torchrun (N > 1) each rank runs its own replica of the workload on its own
GPU (the apply of one patch does not shard: replicas only); value is the total
over ranks divided by the slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D stiffness apply GDoF/s vs p and % HBM roofline; mixed vs FP64 at stated error"
UNIT = "GDoF/s"
# scaled max-norm error bound vs the FP64 oracle; bf16 (factors stored in
# bfloat16) applies a different operator, the quadrature operator with rounded
# factors, which sits about 2^-9 relative from the FP64 one
TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2.0 ** -7, "fp32_on_the_fly": 1e-5}
FACTOR_BYTES = {"fp64": 8, "fp32": 4, "bf16": 2}
VECTOR_BYTES = {"fp64": 8, "fp32": 4, "bf16": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="igasf", choices=["igasf", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--op", default="stiffness", choices=["stiffness", "mass"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--dim", type=int, default=3, choices=[2, 3],
                    help="2: the square counterpart of the workload (no bfloat16 or on-the-fly lines)")
    ap.add_argument("--elements", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the FP64 / mass side runs")
    ap.add_argument("--solve", action="store_true",
                    help="time the Dirichlet solve (p=5, 96^3 elements) instead of the apply")
    ap.add_argument("--solve-elements", type=int, default=96)
    ap.add_argument("--batch", action="store_true",
                    help="time the 256-patch batched apply (seed 7) instead of the single patch")
    ap.add_argument("--assemble", action="store_true",
                    help="time the GPU sum-factorized CSR assembly (FP64) of the --p/--elements cube")
    return ap.parse_args()


def max_over_ranks(x, world, device):
    """The largest x over the ranks (the slowest rank's time); x itself for one
    rank. device: where the all-reduce tensor lives ("cuda" for NCCL, "cpu" for
    gloo)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(dofs_per_rank, world, seconds_per_step):
    """GDoF/s of the whole job: every rank applies its own replica, so the work
    is world x the per-rank dofs in the slowest rank's time."""
    return world * dofs_per_rank / seconds_per_step / 1e9


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_name(p, K, d=3):
    N = (K + p - 1) ** d
    if d == 2:
        return ("perturbed unit square d=2, order p=%d, %d^2 elements (%d dofs, %d^2 Gauss points), "
                "a=exp(0.5 sin 2pi x cos 2pi y), noise min(0.2/%d, Greville gap/3), seed 0"
                % (p, K, N, p * K, K))
    return ("perturbed unit cube d=3, order p=%d, %d^3 elements (%d dofs, %d^3 Gauss points), "
            "a=exp(0.5 sin 2pi x cos 2pi y), noise 0.2/%d, seed 0" % (p, K, N, p * K, K))


def square_patch(p, K):
    """The 2D counterpart of the bench cube: K^2 elements, noise below a third of
    the smallest Greville gap (a diffeomorphism at every order)."""
    import numpy as np
    from paper_1809_05471_gb300 import inputs as I
    gap = float(np.diff(I.greville(I.open_uniform_knots(p, K), p)).min())
    return I.make_patch(2, p, K, noise_amp=min(0.2 / K, gap / 3), seed=0,
                        coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_bytes(op, prec, Qtot, N, d=3):
    """Bytes the apply must move at minimum: the stored factors once, u once, v once."""
    nf = 1 if op == "mass" else d * (d + 1) // 2
    return nf * FACTOR_BYTES[prec] * Qtot + 2 * VECTOR_BYTES[prec] * N


def apply_flops(op, p, K, d=3):
    """Floating-point operations of one sum-factorized apply at the global sizes
    (tile halos excluded): forward sweeps, product, transposed sweeps."""
    N1, Q1 = K + p - 1, K * p
    if op == "mass":
        fwd = 2 * p * (N1 * N1 * Q1 + N1 * Q1 * Q1 + Q1 ** 3)
        return 2 * fwd + 1 * Q1 ** 3
    fwd = 2 * p * (2 * N1 * N1 * Q1 + 3 * N1 * Q1 * Q1 + 3 * Q1 ** 3)
    return 2 * fwd + 15 * Q1 ** 3


def sources_digest(names):
    """First 16 hex digits of the SHA-256 of the named kernel sources, concatenated."""
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1809_05471_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel_key):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current sources of that kernel (the kernel template and what it includes)
    and the default candidate is still the profiled instantiation; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    ent = rec.get(kernel_key)
    if not ent:
        return None
    try:
        h = sources_digest(ent.get("sources", []))
        inst = open(os.path.join(ROOT, "paper_1809_05471_gb300", "csrc",
                                 ent.get("instantiated_in", ""))).read()
    except OSError:
        return None
    if ent.get("sources_sha256_16") != h or ent.get("instantiation", "\0") not in inst:
        return None
    return ent.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def _smi_id():
    import torch
    try:
        pr = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis if vis.isdigit() else "0"


class ClockSampler:
    def __init__(self):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--id=" + _smi_id(), "--query-gpu=" + QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(REASONS, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline); the only oracle use in this file
# ---------------------------------------------------------------------------
def cpu_baseline(patch, op_code, u, seconds, v_gpu=None, seed=0):
    import numpy as np
    import oracle as O

    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    t_rows = 0.0
    done = 0
    batch = 4 * cores
    rows_all, v_all, ra_all = [], [], []
    while t_rows < seconds:
        rows = np.sort(rng.choice(patch.num_dofs, size=batch, replace=False))
        t0 = time.perf_counter()
        v, ra = O.apply_rows(patch, op_code, u, rows, threads=cores)
        t_rows += time.perf_counter() - t0
        done += len(rows)
        rows_all.append(rows)
        v_all.append(v)
        ra_all.append(ra)
        if t_rows < seconds / 4:
            batch *= 2
    rows = np.concatenate(rows_all)
    vref = np.concatenate(v_all)
    a_inf = float(np.concatenate(ra_all).max())
    res = {"value": done / t_rows / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d random rows of v = A u, each assembled from the definition "
                     "(row-wise oracle, OpenMP over rows), %.1f s" % (done, t_rows)}
    errs = {}
    if v_gpu:
        uinf = float(np.max(np.abs(u)))
        for key, vg in v_gpu.items():
            errs[key] = float(np.max(np.abs(vg[rows] - vref))) / (a_inf * uinf)
    return res, errs


# ---------------------------------------------------------------------------
def run_igasf(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    p, K, dim = args.p, args.elements, args.dim
    patch, u = I.config_cube(p=p, K=K) if dim == 3 else square_patch(p, K)
    t0 = time.perf_counter()
    plan = G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    N, Qtot = plan.num_dofs, plan.num_quad_points
    dt = {"fp32": torch.float32, "fp64": torch.float64, "bf16": torch.float32}
    pc = {"fp32": G.FP32, "fp64": G.FP64, "bf16": G.BF16}
    oc = {"stiffness": G.STIFFNESS, "mass": G.MASS}
    stream = torch.cuda.current_stream()

    def timed(op, prec, steps, warmup, sample_clocks=False):
        """Two passes of `steps` applies. The first is the timed region proper
        (barrier and synchronize on both sides, CUDA events on the launching
        stream around all steps, nothing between the kernels, so the gather
        keeps its programmatic overlap with the tile kernel). The second repeats
        the same steps with CUDA events around each kernel, for the per-kernel
        durations of the roofline."""
        ud = torch.as_tensor(u, device="cuda").to(dt[prec])
        vd = torch.empty_like(ud)
        for _ in range(warmup):
            plan.apply(oc[op], ud, vd, prec=pc[prec], stream=stream)
        torch.cuda.synchronize()
        barrier()
        clocks = ClockSampler() if sample_clocks and rank == 0 else None
        if clocks is not None:
            time.sleep(0.3)   # let the sampler start before the timed region
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(steps):
            plan.apply(oc[op], ud, vd, prec=pc[prec], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        # second pass: per-kernel events
        plan.profile_begin(steps)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            plan.apply(oc[op], ud, vd, prec=pc[prec], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_events = e0.elapsed_time(e1)
        k_ms, g_ms, n_timed = plan.profile_end()
        ck = clocks.stop() if clocks is not None else None
        ms = max_over_ranks(ms, world, "cuda")
        return ms, k_ms / max(n_timed, 1), g_ms / max(n_timed, 1), vd, ck, ms_events

    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])

    def roofline(op, prec, kernel_ms):
        ab = algorithmic_bytes(op, prec, Qtot, N, dim)
        ach = ab / (kernel_ms * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
             "frac": round(ach / hbm, 4), "traffic": traffic_record("%s_%s_p%d" % (op, prec, p)),
             "algorithmic_bytes_per_launch": ab, "kernel_ms": round(kernel_ms, 5),
             "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src}
        if prec == "fp64":
            fl = apply_flops(op, p, K)
            r["fp64_tflops"] = round(fl / (kernel_ms * 1e-3) / 1e12, 3)
        return r

    # headline
    ms, k_ms, g_ms, vd, clocks, ms_ev = timed(args.op, args.prec, args.steps, args.warmup, True)
    per_step = ms / args.steps
    value = whole_job_rate(N, world, per_step * 1e-3)
    v_main = vd.double().cpu().numpy()

    # end to end through the host-buffer call (pinned host memory)
    uh = torch.as_tensor(u).to(dt[args.prec]).pin_memory()
    vh = torch.empty_like(uh).pin_memory()
    for _ in range(max(3, min(args.warmup, 20))):
        plan.apply_host(oc[args.op], uh, vh, prec=pc[args.prec], stream=stream)
    e2e_steps = max(10, min(args.steps, 2000))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.apply_host(oc[args.op], uh, vh, prec=pc[args.prec], stream=stream)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    bio = VECTOR_BYTES[args.prec]
    e2e = {"value": round(world * N * e2e_steps / e2e_s / 1e9, 4), "unit": UNIT,
           "h2d_bytes_per_step": N * bio, "d2h_bytes_per_step": N * bio,
           "ms_per_step": round(e2e_s / e2e_steps * 1e3, 4),
           "api": "igasf_apply_host (pinned host u, v)"}

    extra = []
    v_gpu = {"%s_%s" % (args.op, args.prec): v_main}
    if not args.no_extra:
        for op, prec in (("stiffness", "fp64"), ("mass", "fp32"), ("mass", "fp64"),
                         ("stiffness", "fp32"), ("stiffness", "bf16"), ("mass", "bf16")):
            if (op, prec) == (args.op, args.prec):
                continue
            steps = 300 if prec == "fp64" else 1000
            ms2, k2, g2, vd2, _, _ = timed(op, prec, steps, 10)
            if op == args.op:
                v_gpu["%s_%s" % (op, prec)] = vd2.double().cpu().numpy()
            extra.append({"op": op, "prec": prec, "value": round(world * N / (ms2 / steps * 1e-3) / 1e9, 4),
                          "ms_per_step": round(ms2 / steps, 5), "roofline": roofline(op, prec, k2),
                          "gather_ms": round(g2, 5)})
        # FP32 with the factors evaluated inside the tile kernel (nothing stored, 3D)
        geo = G.Plan.from_patch(patch, precisions=(G.FP32,), geometry=G.GEOMETRY_ON_THE_FLY) \
            if dim == 3 else None
        for op in (("stiffness", "mass") if geo is not None else ()):
            ud = torch.as_tensor(u, device="cuda").float()
            vd2 = torch.empty_like(ud)
            for _ in range(10):
                geo.apply(oc[op], ud, vd2, prec=G.FP32, stream=stream)
            steps = 1000
            geo.profile_begin(steps)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                geo.apply(oc[op], ud, vd2, prec=G.FP32, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1)
            k2, g2, n2 = geo.profile_end()
            if op == args.op:
                v_gpu["%s_fp32_on_the_fly" % op] = vd2.double().cpu().numpy()
            extra.append({"op": op, "prec": "fp32", "geometry": "on the fly",
                          "value": round(world * N / (ms2 / steps * 1e-3) / 1e9, 4),
                          "ms_per_step": round(ms2 / steps, 5), "kernel_ms": round(k2 / max(n2, 1), 5),
                          "gather_ms": round(g2 / max(n2, 1), 5),
                          "bytes_per_launch": 4 * 5 * N,
                          "note": "no stored factors: reads u and the control points, writes v"})
        if geo is not None:
            geo.close()

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "f32 (bf16-stored factors)"}[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(p, K, dim), "op": args.op, "precision": args.prec,
                   "d": dim, "order": p, "elements_per_dir": K, "dofs": N, "quad_points": Qtot,
                   "tile": plan.describe(pc[args.prec])["tile"],
                   "l2": "no flush: factors (%.0f MB) larger than L2 (129 MB)"
                         % (algorithmic_bytes(args.op, args.prec, Qtot, 0, dim) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline(args.op, args.prec, k_ms),
        "gather_ms": round(g_ms, 5),
        "ms_per_step_with_kernel_events": round(ms_ev / args.steps, 5),
        "kernel_timing": ("tile kernel and gather durations from CUDA events around each kernel, "
                          "over a second pass of the same steps right after the timed one (events "
                          "between the two kernels serialise their programmatic overlap)"),
        "e2e": e2e,
        "gpu_launches": 2 * args.steps * world,
        "setup_s": round(setup_s, 3),
        "clocks": clocks,
        "also": extra,
    }
    if rank == 0 and not args.no_cpu_baseline:
        cb, errs = cpu_baseline(patch, oc[args.op], u, args.cpu_seconds, v_gpu)
        result["cpu_baseline"] = cb
        result["error_vs_oracle"] = {"rows": "the cpu_baseline sample", "scaled_max_norm": errs,
                                     "tolerance": TOL}
    result["device_status"] = "ok" if plan.device_status() == 0 else "a bounded wait ran out"
    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_solve(args):
    """Homogeneous-Dirichlet Poisson solve on the perturbed cube, order p = 5,
    96^3 elements (100^3 = 1M dofs), a = 1, b = M u* with u* ~ U[-1, 1] (seed 0),
    Jacobi-PCG to a 1e-10 relative residual: FP32 inner solves inside FP64
    iterative refinement against all-FP64 PCG, on the same GPU (and, reported
    beside them, inner solves with bfloat16-stored factors). b is formed with
    the FP64 mass apply (the row oracle would need hours at this size)."""
    import numpy as np
    import torch

    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    K = args.solve_elements
    patch, ustar = I.make_patch(3, 5, K, noise_amp=0.2 / K, seed=0)
    t0 = time.perf_counter()
    plan = G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16))
    setup_s = time.perf_counter() - t0
    us = torch.as_tensor(ustar, device="cuda")
    b = torch.empty_like(us)
    plan.apply(G.MASS, us, b, prec=G.FP64)
    # warm-up (also computes the Jacobi diagonal once)
    x = torch.zeros_like(b)
    plan.cg_solve(b, x, inner_prec=G.FP32, rtol=1e-2)
    runs = {}
    for name, prec in (("mixed_fp32_in_fp64_ir", G.FP32), ("all_fp64", G.FP64),
                       ("mixed_bf16_in_fp64_ir", G.BF16)):
        x = torch.zeros_like(b)
        rep = plan.cg_solve(b, x, inner_prec=prec, rtol=1e-10, inner_rtol=1e-4)
        runs[name] = rep
    mixed, full = runs["mixed_fp32_in_fp64_ir"], runs["all_fp64"]
    ok = plan.device_status() == 0
    plan.close()
    print(json.dumps({
        "metric": "time to 1e-10 relative residual, Jacobi-PCG, homogeneous Dirichlet",
        "value": round(mixed["seconds"], 4), "unit": "s", "n_gpus": 1,
        "higher_is_better": False, "data": "synthetic",
        "config": {"workload": "perturbed unit cube d=3, order p=5, %d^3 elements (%d dofs), "
                               "a=1, b = M u*, u* ~ U[-1,1] seed 0" % (K, plan.num_dofs),
                   "tolerance": 1e-10, "inner_rtol": 1e-4},
        "mixed": mixed, "fp64": full, "mixed_bf16": runs["mixed_bf16_in_fp64_ir"],
        "speedup_vs_fp64": round(full["seconds"] / mixed["seconds"], 3),
        "setup_s": round(setup_s, 3), "device_status": "ok" if ok else "a bounded wait ran out",
    }), flush=True)


def run_batch(args):
    """256 independent d=3 patches (seed 7; 8..48 elements per direction, p = 2..6,
    constant a ~ U[0.5, 2]), FP32 stiffness, applied as one CUDA graph launch.
    Tile shape and kernel variant per order come from the library autotuner run on
    the largest patch of that order."""
    import numpy as np
    import torch

    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    patches = I.config_batch()
    t0 = time.perf_counter()
    tuned = {}
    for p in sorted({pt.orders[0] for pt, _ in patches}):
        big = max((pt for pt, _ in patches if pt.orders[0] == p), key=lambda q: q.num_quad_points)
        tile, variant, ms = G.autotune(big, op=G.STIFFNESS, prec=G.FP32, repeats=5)
        tuned[p] = {"tile": tile, "variant": variant, "ms_on_largest": round(ms, 4)}
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    plans = [G.Plan.from_patch(pt, precisions=(G.FP32,), tile=tuned[pt.orders[0]]["tile"],
                               kernel_variant=tuned[pt.orders[0]]["variant"]) for pt, _ in patches]
    setup_s = time.perf_counter() - t0
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    vd = torch.empty_like(ud)
    batch = G.Batch(plans, op=G.STIFFNESS, prec=G.FP32)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup // 10)):
        batch.apply(ud, vd, stream=stream)
    steps = max(10, args.steps // 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        batch.apply(ud, vd, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the same work as individual applies, one after another (no graph)
    e0.record(stream)
    for _ in range(3):
        for k, plan in enumerate(plans):
            a, b = int(batch.offsets[k]), int(batch.offsets[k + 1])
            plan.apply(G.STIFFNESS, ud[a:b], vd[a:b], prec=G.FP32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / 3
    peaks, _ = measured_peaks()
    alg = 24 * batch.total_quad_points + 8 * batch.total_dofs
    ok = all(plan.device_status() == 0 for plan in plans)
    print(json.dumps({
        "metric": "batched 3D stiffness apply GDoF/s (256 uneven patches, one graph launch)",
        "value": round(batch.total_dofs / (ms * 1e-3) / 1e9, 4), "unit": "GDoF/s", "n_gpus": 1,
        "steps": steps, "ms_per_step": round(ms, 4), "higher_is_better": True, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "256 patches from seed 7: 8..48 elements per direction, p = 2..6, "
                               "a ~ U[0.5, 2]; %d dofs, %d quadrature points" % (batch.total_dofs,
                                                                                batch.total_quad_points),
                   "launch_groups": batch.launch_groups, "tuned": {str(k): v for k, v in tuned.items()}},
        "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1),
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                     "note": "whole graph (tile kernels + gather), algorithmic bytes 24 B/qp + 8 B/dof"},
        "sequential_individual_applies_ms": round(ms_seq, 4),
        "autotune_s": round(tune_s, 2), "setup_s": round(setup_s, 2),
        "device_status": "ok" if ok else "a bounded wait ran out",
    }), flush=True)
    batch.close()
    for plan in plans:
        plan.close()


def run_reference(args):
    """The oracle as it stands, on the host cores, on the same workload and metric:
    each step computes a bounded sample of rows of v = A u."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_1809_05471_gb300 import inputs as I

    p, K = args.p, args.elements
    patch, u = I.config_cube(p=p, K=K)
    op = O.STIFFNESS if args.op == "stiffness" else O.MASS
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(0)
    # size each step so that warmup + steps take about 120 s
    t0 = time.perf_counter()
    O.apply_rows(patch, op, u, rng.choice(patch.num_dofs, cores, replace=False), threads=cores)
    per_row = (time.perf_counter() - t0) / cores
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows_per_step = max(1, int(budget / per_row))
    for _ in range(args.warmup):
        O.apply_rows(patch, op, u, rng.choice(patch.num_dofs, rows_per_step, replace=False),
                     threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.apply_rows(patch, op, u, rng.choice(patch.num_dofs, rows_per_step, replace=False),
                     threads=cores)
    dt_s = time.perf_counter() - t0
    value = rows_per_step * args.steps / dt_s / 1e9
    sample = ("%d random rows of v = A u per step (row-wise FP64 oracle, OpenMP over rows)"
              % rows_per_step)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(p, K), "op": args.op, "precision": args.prec},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def assembly_flops(d, p, K, op):
    """Floating-point operations of the sum-factorized assembly as implemented
    (one FMA, 2 flop, per inner term: the product of the two univariate tables is
    precomputed per pair), counted from the loop bounds."""
    W = 2 * p - 1
    N = K + p - 1
    # sum over (m, o) valid of (#shared elements) * p, one direction
    C = 0
    nnz1 = 0
    for m in range(N):
        for o in range(W):
            n = m + o - (p - 1)
            if 0 <= n < N:
                nnz1 += 1
                lo, hi = max(max(m, n) - p + 1, 0), min(min(m, n), K - 1)
                C += max(0, hi - lo + 1) * p
    Q = K * p
    nterms, ngroups = (d * d, 4) if op == "stiffness" else (1, 1)
    if d == 3:
        it = nterms * Q * Q * C + nterms * Q * C * N * W + ngroups * C * nnz1 * nnz1
    else:
        it = nterms * Q * C + ngroups * C * nnz1
    return 2 * it


def run_assemble(args):
    """FP64 CSR assembly by sum factorization over the whole patch (Alg. 1) on
    the GPU: the perturbed cube, order p, K^3 elements, a = exp(0.5 sin cos);
    time per assembly of K and of M (synchronous calls, CUDA-synchronised
    wall time), checked on sampled rows against the oracle, with the oracle's
    row assembly timed on the host cores as the CPU baseline."""
    import numpy as np
    import torch

    import oracle as O
    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p, K = args.p, args.elements
    patch, u = I.config_cube(p=p, K=K)
    plan = G.Plan.from_patch(patch, precisions=(G.FP64,))
    out = {}
    for opname, op in (("stiffness", G.STIFFNESS), ("mass", G.MASS)):
        rp, ci, va = plan.assemble_csr(op)                      # warm-up
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(reps):
            del rp, ci, va
            rp, ci, va = plan.assemble_csr(op)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        fl = assembly_flops(3, p, K, opname)
        rows = np.sort(np.random.default_rng(5).choice(plan.num_dofs, 48, replace=False))
        rp_h, ci_h, va_h = rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy()
        v = np.array([np.dot(va_h[rp_h[r]:rp_h[r + 1]], u[ci_h[rp_h[r]:rp_h[r + 1]]]) for r in rows])
        cores = len(os.sched_getaffinity(0))
        t1 = time.perf_counter()
        vr, ra = O.apply_rows(patch, op, u, rows, threads=cores)
        t_rows = time.perf_counter() - t1
        out[opname] = {"seconds": round(sec, 5), "nnz": int(len(va_h)),
                       "gflops": round(fl / sec / 1e9, 1), "flops_per_assembly": fl,
                       "error_vs_oracle_rows": float(np.max(np.abs(v - vr)) / (ra.max() * np.max(np.abs(u)))),
                       "cpu_baseline": {"kind": "oracle", "cores": cores, "rows": len(rows),
                                        "seconds": round(t_rows, 3),
                                        "full_matrix_seconds_extrapolated":
                                            round(t_rows / len(rows) * plan.num_dofs, 1)}}
        del rp, ci, va
    ok = plan.device_status() == 0
    plan.close()
    print(json.dumps({
        "metric": "FP64 CSR assembly time (sum factorization over the whole patch, Alg. 1)",
        "value": out["stiffness"]["seconds"], "unit": "s", "n_gpus": 1, "higher_is_better": False,
        "data": "synthetic",
        "config": {"workload": "perturbed unit cube d=3, order p=%d, %d^3 elements (%d dofs), "
                               "a = exp(0.5 sin 2 pi x cos 2 pi y)" % (p, K, (K + p - 1) ** 3)},
        "stiffness": out["stiffness"], "mass": out["mass"],
        "device_status": "ok" if ok else "a bounded wait ran out",
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.solve:
        run_solve(args)
    elif args.batch:
        run_batch(args)
    elif args.assemble:
        run_assemble(args)
    else:
        run_igasf(args)


if __name__ == "__main__":
    main()
