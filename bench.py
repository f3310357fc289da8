#!/usr/bin/env python
"""Benchmark of the matrix-free sum-factorized stiffness apply (GDoF/s).

Headline workload: d = 3 perturbed unit cube, order p = 4, 64^3 elements
(67^3 = 300,763 dofs, 256^3 Gauss points), a(x) = exp(0.5 sin 2 pi x cos 2 pi y),
stiffness apply in FP32. One step = one apply v = K u (tile kernel + gather) with
u, v and the factors resident in HBM. Factors (403 MB in FP32) exceed the L2
(129 MB), so no flush is needed between steps. The K-step timed region is then
repeated back to back (200 windows by default) for the median and spread.

Also reported (single GPU), each as an entry of "also":
  * the 64^3 workload in the other precisions (FP64, BF16-stored factors, the
    tensor-core TF32 and BF16_MMA sweeps, factors on the fly) and the mass apply;
  * the order sweep p = 2..9 at about 2M dofs (127 - p elements per direction):
    GDoF/s, tile-kernel roofline and the scaled error against the FP64 oracle on
    sampled rows, per precision;
  * the Dirichlet solve (p = 5, 96^3 elements): mixed-precision iterative
    refinement against all-FP64 PCG to 1e-10;
  * the 256-patch batched apply (one CUDA-graph launch).
plus the end-to-end rate through the host-buffer C-ABI call, the SM clocks
sampled during the timed windows, and the CPU baseline: the FP64 oracle's CSR
product on the host cores (all of them and one).

With torchrun (N > 1) each rank runs its own replica of the headline workload
on its own GPU (the apply of one patch does not shard: replicas only); value is
the total over ranks divided by the slowest rank's time; the side runs are made
at N = 1 only.

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
PRECS = ("fp64", "fp32", "bf16", "tf32", "bf16_mma")
# scaled max-norm bar against the FP64 oracle (tests/gpu_helpers.py derives the
# per-order bars; these are their largest values over p = 2..9). bf16 and
# bf16_mma store the factors in bfloat16: against the FP64 operator they carry
# that rounding (about 2^-9 relative), against the oracle's operator with the
# same rounded factors only their arithmetic's error.
TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2.0 ** -7, "tf32": 4 * 2.0 ** -11 + 1e-5,
       "bf16_mma": 2.0 ** -7 + 4 * 2.0 ** -8, "fp32_on_the_fly": 1e-5}
FACTOR_BYTES = {"fp64": 8, "fp32": 4, "bf16": 2, "tf32": 4, "bf16_mma": 2}
VECTOR_BYTES = {"fp64": 8, "fp32": 4, "bf16": 4, "tf32": 4, "bf16_mma": 4}
ROUNDED_FACTORS = ("bf16", "bf16_mma")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=200,
                    help="back-to-back repeats of the K-step timed region (median and spread)")
    ap.add_argument("--impl", default="igasf", choices=["igasf", "reference"])
    ap.add_argument("--prec", default="fp32", choices=list(PRECS))
    ap.add_argument("--op", default="stiffness", choices=["stiffness", "mass"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--dim", type=int, default=3, choices=[2, 3],
                    help="2: the square counterpart of the workload (FP64, FP32 and BF16 only)")
    ap.add_argument("--elements", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="only the headline: no other precisions, sweep, solve or batch")
    ap.add_argument("--sweep-orders", default="2,3,4,5,6,7,8,9",
                    help="orders of the 2M-dof order sweep ('' for none)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--solve", action="store_true",
                    help="only the Dirichlet solve (p=5, 96^3 elements)")
    ap.add_argument("--solve-elements", type=int, default=96)
    ap.add_argument("--batch", action="store_true", help="only the 256-patch batched apply")
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


def bench_config(args, world=1):
    """The config object of both arms (computed without a GPU)."""
    p, K, d = args.p, args.elements, args.dim
    N, Q = (K + p - 1) ** d, (K * p) ** d
    return {"workload": workload_name(p, K, d), "op": args.op, "precision": args.prec, "d": d,
            "order": p, "elements_per_dir": K, "dofs": N, "quad_points": Q,
            "l2": "no flush: factors (%.0f MB) larger than L2 (129 MB)"
                  % (algorithmic_bytes(args.op, args.prec, Q, 0, d) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU"}


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
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
# besides the error check of the GPU results and the reference arm
# ---------------------------------------------------------------------------
def csr_sample(patch, op_code, layers, cores):
    """CSR of `layers` consecutive interior dof layers of the last direction (all
    their rows), each row assembled from the definition by the oracle."""
    import numpy as np
    import oracle as O
    N1, N2, N3 = patch.dofs_per_dir
    l0 = max(0, N3 // 2 - layers // 2)
    rows = np.arange(l0 * N1 * N2, (l0 + layers) * N1 * N2, dtype=np.int64)
    t0 = time.perf_counter()
    rp, ci, va = O.assemble_rows(patch, op_code, rows, threads=cores)
    return rows, rp, ci, va, time.perf_counter() - t0


def full_size_csr(rp, ci, va, nrows):
    """A CSR of nrows rows made of copies of the sample's rows, in order (the
    matrix of the workload's size: same rows, same nonzeros per row, the same
    column pattern per row), for timing the product on a matrix larger than the
    host caches."""
    import numpy as np
    ns = len(rp) - 1
    reps = -(-nrows // ns)
    counts = np.diff(rp)
    cnt = np.tile(counts, reps)[:nrows]
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    nz = int(rowptr[-1])
    colind = np.tile(ci, reps)[:nz]
    val = np.tile(va, reps)[:nz]
    return rowptr, colind, val


def time_spmv(rowptr, colind, val, x, threads, min_seconds=1.0, max_reps=50):
    import numpy as np
    import oracle as O
    O.set_threads(threads)
    O.spmv(rowptr, colind, val, x)              # warm-up (first touch of the output)
    reps, t = 0, 0.0
    while t < min_seconds and reps < max_reps:
        t0 = time.perf_counter()
        O.spmv(rowptr, colind, val, x)
        t += time.perf_counter() - t0
        reps += 1
    return t / reps


def cpu_baseline(patch, op_code, u, v_gpu=None, layers=3):
    """The oracle on the host cores: the CSR product v = A u (orc_spmv, OpenMP over
    rows) timed on all cores and on one, on a matrix of the workload's size built
    from `layers` dof layers of oracle-assembled rows; the GPU results are
    compared with the oracle on those rows. Also reported, as a second figure:
    the oracle's row-wise apply, which assembles each row from the definition."""
    import numpy as np
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    rows, rp, ci, va, t_asm = csr_sample(patch, op_code, layers, cores)
    N = patch.num_dofs
    big = full_size_csr(rp, ci, va, N)
    t_all = time_spmv(*big, u, cores)
    t_one = time_spmv(*big, u, 1, min_seconds=0.5, max_reps=3)
    O.set_threads(cores)
    nnz = int(big[0][-1])
    res = {"value": N / t_all / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle CSR SpMV",
           "cores_1": {"value": N / t_one / 1e9, "unit": UNIT, "cores": 1},
           "sample": ("orc_spmv (OpenMP over rows) of a %d-row, %d-nonzero FP64 CSR matrix (the "
                      "workload's size) made of copies of %d rows (%d dof layers of the last "
                      "direction) assembled row by row from the definition by the oracle (%.1f s); "
                      "%.2f ms per product on %d cores, %.1f ms on one"
                      % (N, nnz, len(rows), layers, t_asm, t_all * 1e3, cores, t_one * 1e3))}
    # second figure: the row-wise apply (assembles every row from the definition)
    sub = rows[:: max(1, len(rows) // (4 * cores))][: 4 * cores]
    t0 = time.perf_counter()
    O.apply_rows(patch, op_code, u, sub, threads=cores)
    t_rows = time.perf_counter() - t0
    res["row_assembly_apply"] = {"value": len(sub) / t_rows / 1e9, "unit": UNIT, "cores": cores,
                                 "kind": "oracle row-wise apply (each row assembled from the definition)",
                                 "sample": "%d rows, %.2f s" % (len(sub), t_rows)}
    errs = {}
    if v_gpu:
        vref = O.spmv(rp, ci, va, u)
        a_inf = float(np.max(np.add.reduceat(np.abs(va), rp[:-1])))
        uinf = float(np.max(np.abs(u)))
        for key, vg in v_gpu.items():
            errs[key] = float(np.max(np.abs(vg[rows] - vref))) / (a_inf * uinf)
    return res, errs, {"rows": "%d rows (%d dof layers)" % (len(rows), layers)}


def fp64_peak():
    """Measured FP64 rate of this GPU: the best of five 4096^3 cuBLAS DGEMMs
    through torch.matmul (FP64 tensor-core or FMA path, whichever cuBLAS takes)."""
    import torch
    n = 4096
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# ---------------------------------------------------------------------------
# device timing
# ---------------------------------------------------------------------------
def time_apply(plan, op, prec, u_dev, steps, warmup, stream, barrier=None, repeats=0, clocks=False,
               rank=0):
    """CUDA-event timing of `steps` applies on the launching stream, after
    `warmup` untimed ones, with a synchronize (and barrier) on both sides: the
    timed region proper, nothing between the kernels so that the gather keeps
    its programmatic overlap with the tile kernel. Then `repeats` more windows of
    `steps` applies back to back (for the median and spread), and a last pass
    with CUDA events around each kernel for the per-kernel durations.
    Returns (ms of the timed region, dict of the repeats or None, tile-kernel ms
    per apply, gather ms per apply, v, clock record or None)."""
    import torch
    barrier = barrier or (lambda: None)
    vd = torch.empty_like(u_dev)
    for _ in range(warmup):
        plan.apply(op, u_dev, vd, prec=prec, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler() if clocks and rank == 0 else None
    if sampler is not None:
        time.sleep(0.3)   # let the sampler start before the timed region
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(steps):
        plan.apply(op, u_dev, vd, prec=prec, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    rep = None
    if repeats > 0:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(repeats + 1)]
        evs[0].record(stream)
        for r in range(repeats):
            for _ in range(steps):
                plan.apply(op, u_dev, vd, prec=prec, stream=stream)
            evs[r + 1].record(stream)
        torch.cuda.synchronize()
        per = sorted(evs[r].elapsed_time(evs[r + 1]) / steps for r in range(repeats))
        q = lambda f: per[min(len(per) - 1, int(f * len(per)))]
        rep = {"windows": repeats, "steps_per_window": steps,
               "median_ms_per_step": round(statistics.median(per), 5), "p10": round(q(0.1), 5),
               "p90": round(q(0.9), 5), "min": round(per[0], 5), "max": round(per[-1], 5)}
    ck = sampler.stop() if sampler is not None else None
    n = max(steps, 5)
    plan.profile_begin(n)
    for _ in range(n):
        plan.apply(op, u_dev, vd, prec=prec, stream=stream)
    k_ms, g_ms, n_timed = plan.profile_end()
    return ms, rep, k_ms / max(n_timed, 1), g_ms / max(n_timed, 1), vd, ck


def steps_for(ms_estimate, target_ms=150.0, lo=5, hi=2000):
    return int(max(lo, min(hi, target_ms / max(ms_estimate, 1e-4))))


# ---------------------------------------------------------------------------
def run_igasf(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle as O
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

    pc = {"fp32": G.FP32, "fp64": G.FP64, "bf16": G.BF16, "tf32": G.TF32, "bf16_mma": G.BF16_MMA}
    oc = {"stiffness": G.STIFFNESS, "mass": G.MASS}
    dt = lambda prec: torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.current_stream()
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    extras = not args.no_extra and world == 1

    p, K, dim = args.p, args.elements, args.dim
    patch, u = I.config_cube(p=p, K=K) if dim == 3 else square_patch(p, K)
    precs64 = ("fp64", "fp32", "bf16") + (("tf32", "bf16_mma") if dim == 3 else ())
    if not extras:
        precs64 = tuple(sorted({args.prec}))
    t0 = time.perf_counter()
    plan = G.Plan.from_patch(patch, precisions=tuple(pc[x] for x in precs64))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    N, Qtot = plan.num_dofs, plan.num_quad_points
    fp64_tf = fp64_peak() if extras else None

    def roofline(op, prec, kernel_ms, Qt, Nd, pp, KK, dd=3, cube=True):
        """cube: the bench cube's own launch, whose DRAM traffic a committed ncu
        summary may record (the order sweep's launches have none)."""
        ab = algorithmic_bytes(op, prec, Qt, Nd, dd)
        ach = ab / (kernel_ms * 1e-3) / 1e9
        traffic = traffic_record("%s_%s_p%d_cube%d" % (op, prec, pp, KK)) if cube else None
        r = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
             "frac": round(ach / hbm, 4), "traffic": traffic,
             "algorithmic_bytes_per_launch": ab, "kernel_ms": round(kernel_ms, 5),
             "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src}
        if prec == "fp64":
            fl = apply_flops(op, pp, KK, dd)
            tf = fl / (kernel_ms * 1e-3) / 1e12
            r["fp64_tflops"] = round(tf, 3)
            if fp64_tf:
                r["fp64_peak_tflops"] = round(fp64_tf, 3)
                r["fp64_frac"] = round(tf / fp64_tf, 4)
                r["fp64_peak_source"] = "measured: best of five 4096^3 cuBLAS DGEMMs (torch.matmul)"
        return r

    # ---- headline: the timed region, its repeats, per-kernel durations
    ud = torch.as_tensor(u, device="cuda").to(dt(args.prec))
    ms, rep, k_ms, g_ms, vd, clocks = time_apply(plan, oc[args.op], pc[args.prec], ud, args.steps,
                                                 args.warmup, stream, barrier, args.repeats, True, rank)
    ms = max_over_ranks(ms, world, "cuda")
    per_step = ms / args.steps
    value = whole_job_rate(N, world, per_step * 1e-3)
    v_main = vd.double().cpu().numpy()

    # ---- end to end through the host-buffer calls (pinned host memory): every
    # step copies its u from the host and writes its v into host memory. The
    # asynchronous call lets step k + 1's input copy run during step k's apply
    # (the timed region ends when the stream has finished every step); the
    # synchronous call waits for each step before the next.
    uh = torch.as_tensor(u).to(dt(args.prec)).pin_memory()
    vh = torch.empty_like(uh).pin_memory()
    e2e_steps = max(10, min(args.steps, 2000))
    bio = VECTOR_BYTES[args.prec]

    def e2e_run(call):
        for _ in range(max(3, min(args.warmup, 20))):
            call(oc[args.op], uh, vh, prec=pc[args.prec], stream=stream)
        stream.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            call(oc[args.op], uh, vh, prec=pc[args.prec], stream=stream)
        stream.synchronize()
        return max_over_ranks(time.perf_counter() - t0, world, "cuda")

    e2e_s = e2e_run(plan.apply_host_async)
    e2e_sync_s = e2e_run(plan.apply_host)
    e2e = {"value": round(world * N * e2e_steps / e2e_s / 1e9, 4), "unit": UNIT,
           "h2d_bytes_per_step": N * bio, "d2h_bytes_per_step": N * bio,
           "ms_per_step": round(e2e_s / e2e_steps * 1e3, 4), "steps": e2e_steps,
           "api": "igasf_apply_host_async (pinned host u and v; stream synchronised after "
                  "the last step)",
           "synchronous": {"value": round(world * N * e2e_steps / e2e_sync_s / 1e9, 4),
                           "ms_per_step": round(e2e_sync_s / e2e_steps * 1e3, 4),
                           "api": "igasf_apply_host (waits for each step)"}}

    extra = []
    v_gpu = {"%s_%s" % (args.op, args.prec): v_main}
    if extras:
        for op in ("stiffness", "mass"):
            for prec in precs64:
                if (op, prec) == (args.op, args.prec):
                    continue
                u2 = torch.as_tensor(u, device="cuda").to(dt(prec))
                steps = 300 if prec == "fp64" else 1000
                ms2, _, k2, g2, vd2, _ = time_apply(plan, oc[op], pc[prec], u2, steps, 10, stream)
                if op == args.op:
                    v_gpu["%s_%s" % (op, prec)] = vd2.double().cpu().numpy()
                extra.append({"workload": "bench cube", "op": op, "prec": prec,
                              "value": round(N / (ms2 / steps * 1e-3) / 1e9, 4),
                              "ms_per_step": round(ms2 / steps, 5),
                              "roofline": roofline(op, prec, k2, Qtot, N, p, K, dim),
                              "tile": plan.describe(pc[prec])["tile"], "gather_ms": round(g2, 5)})
                del u2, vd2
        # FP32 with the factors evaluated inside the tile kernel (nothing stored, 3D)
        if dim == 3:
            with G.Plan.from_patch(patch, precisions=(G.FP32,), geometry=G.GEOMETRY_ON_THE_FLY) as geo:
                u2 = torch.as_tensor(u, device="cuda").float()
                for op in ("stiffness", "mass"):
                    ms2, _, k2, g2, vd2, _ = time_apply(geo, oc[op], G.FP32, u2, 1000, 10, stream)
                    if op == args.op:
                        v_gpu["%s_fp32_on_the_fly" % op] = vd2.double().cpu().numpy()
                    extra.append({"workload": "bench cube", "op": op, "prec": "fp32",
                                  "geometry": "on the fly",
                                  "value": round(N / (ms2 / 1000 * 1e-3) / 1e9, 4),
                                  "ms_per_step": round(ms2 / 1000, 5), "kernel_ms": round(k2, 5),
                                  "gather_ms": round(g2, 5), "bytes_per_launch": 4 * 5 * N,
                                  "note": "no stored factors: reads u and the control points, writes v"})
                    del vd2
    device_ok = plan.device_status() == 0
    tile_main = plan.describe(pc[args.prec])["tile"]
    plan.close()
    torch.cuda.empty_cache()

    sweep = []
    if extras and dim == 3 and args.sweep_orders:
        sweep, ok_sw = order_sweep([int(x) for x in args.sweep_orders.split(",")], G, I, O,
                                   torch, stream, roofline)
        device_ok = device_ok and ok_sw
        extra.extend(sweep)
    if extras and dim == 3 and not args.no_solve:
        extra.append(solve_entry(args, G, I, torch))
    if extras and dim == 3 and not args.no_batch:
        extra.append(batch_entry(args, G, I, torch, hbm))

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "f32 (bf16-stored factors)",
                  "tf32": "f32 (tf32 tensor-core direction-3 contractions)",
                  "bf16_mma": "f32 (bf16-stored factors, bf16 tensor-core direction-3 contractions)"}
        [args.prec],
        "data": "synthetic",
        "config": bench_config(args, world),
        "tile": tile_main,
        "roofline": roofline(args.op, args.prec, k_ms, Qtot, N, p, K, dim),
        "repeats": rep,
        "gather_ms": round(g_ms, 5),
        "kernel_timing": ("tile kernel and gather durations from CUDA events around each kernel, "
                          "over a pass of the same applies right after the timed windows (events "
                          "between the two kernels serialise their programmatic overlap)"),
        "e2e": e2e,
        "gpu_launches": 2 * args.steps * world,
        "setup_s": round(setup_s, 3),
        "clocks": clocks,
        "clocks_window": "sampled every 50 ms from before the timed region through its %d repeats"
                         % (args.repeats,),
        "also": extra,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cb, errs, rows_desc = cpu_baseline(patch, oc[args.op], u, v_gpu)
        result["cpu_baseline"] = cb
        result["error_vs_oracle"] = {"rows": rows_desc["rows"], "scaled_max_norm": errs,
                                     "tolerance": TOL,
                                     "note": "against the FP64 operator; bf16 variants carry the "
                                             "bfloat16 rounding of the factors (the order sweep "
                                             "also compares them with the rounded-factor operator)"}
    result["device_status"] = "ok" if device_ok else "a bounded wait ran out"
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


SWEEP_WINDOWS = 4   # timed windows per order-sweep line after the first


def order_sweep(orders, G, I, O, torch, stream, roofline):
    """The order sweep: p = 2..9 at about 2M dofs (127 - p elements per
    direction, the same perturbed cube and coefficient), stiffness in every
    precision (FP64 up to p = 6: its factors alone are 30 to 60 GB beyond), one
    plan per precision at a time; GDoF/s per apply (median of SWEEP_WINDOWS timed
    windows, with the SM clocks sampled meanwhile), tile-kernel roofline and the
    scaled error on sampled rows against the FP64 oracle (and, for the bfloat16
    precisions, against the oracle's operator with the same rounded factors)."""
    import numpy as np
    cores = len(os.sched_getaffinity(0))
    pc = {"fp32": G.FP32, "fp64": G.FP64, "bf16": G.BF16, "tf32": G.TF32, "bf16_mma": G.BF16_MMA}
    out, ok = [], True
    for p in orders:
        patch, u = I.config_sweep(p)
        K = I.sweep_elements(p)
        precs = ("fp32", "bf16", "tf32", "bf16_mma") + (("fp64",) if p <= 6 else ())
        vs, lines = {}, []
        for prec in precs:
            t0 = time.perf_counter()
            plan = G.Plan.from_patch(patch, precisions=(pc[prec],))
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            ud = torch.as_tensor(u, device="cuda").to(torch.float64 if prec == "fp64" else torch.float32)
            ms, _, k_ms, _, _, _ = time_apply(plan, G.STIFFNESS, pc[prec], ud, 3, 2, stream)
            steps = steps_for(ms / 3)
            # the first window, then SWEEP_WINDOWS more: the line reports their median
            # (one window of 30 to 70 steps can catch a passing clock dip)
            ms, rep, k_ms, g_ms, vd, ck = time_apply(plan, G.STIFFNESS, pc[prec], ud, steps, 3, stream,
                                                     repeats=SWEEP_WINDOWS, clocks=True)
            ms_step = rep["median_ms_per_step"]
            vs[prec] = vd.double().cpu().numpy()
            ok = ok and plan.device_status() == 0
            N, Q = plan.num_dofs, plan.num_quad_points
            lines.append({"workload": "order sweep", "p": p, "elements_per_dir": K, "dofs": N,
                          "quad_points": Q, "op": "stiffness", "prec": prec,
                          "tile": plan.describe(pc[prec])["tile"],
                          "value": round(N / (ms_step * 1e-3) / 1e9, 4),
                          "ms_per_step": ms_step, "steps": steps,
                          "windows": {"count": SWEEP_WINDOWS, "first_window_ms_per_step": round(ms / steps, 5),
                                      "min": rep["min"], "max": rep["max"]},
                          "roofline": roofline("stiffness", prec, k_ms, Q, N, p, K, cube=False),
                          "gather_ms": round(g_ms, 5), "setup_s": round(setup_s, 3), "clocks": ck})
            plan.close()
            del ud, vd
            torch.cuda.empty_cache()
        rows = np.sort(np.random.default_rng(600 + p).choice(patch.num_dofs, 8 if p >= 8 else 24,
                                                               replace=False))
        t0 = time.perf_counter()
        ref = {0: O.apply_rows(patch, O.STIFFNESS, u, rows, threads=cores)}
        with O.stored_factor_bits(O.BF16_BITS):
            ref[O.BF16_BITS] = O.apply_rows(patch, O.STIFFNESS, u, rows, threads=cores)
        t_or = time.perf_counter() - t0
        uinf = float(np.max(np.abs(u)))
        for ln in lines:
            v = vs[ln["prec"]][rows]
            vr, ra = ref[0]
            err = {"fp64_operator": float(np.max(np.abs(v - vr)) / (ra.max() * uinf))}
            if ln["prec"] in ROUNDED_FACTORS:
                vb, rb = ref[O.BF16_BITS]
                err["rounded_factor_operator"] = float(np.max(np.abs(v - vb)) / (rb.max() * uinf))
            ln["error_vs_oracle"] = dict(err, rows=len(rows), oracle_seconds=round(t_or, 2))
        out.extend(lines)
        log("sweep p=%d done" % p)
    return out, ok


def solve_entry(args, G, I, torch):
    """Homogeneous-Dirichlet Poisson solve on the perturbed cube, order p = 5,
    96^3 elements (100^3 = 1M dofs), a = 1, b = M u* with u* ~ U[-1, 1] (seed 0),
    Jacobi-PCG to a 1e-10 relative residual: FP32 inner solves inside FP64
    iterative refinement against all-FP64 PCG, on the same GPU (and, beside
    them, inner solves with bfloat16-stored factors and with the TF32
    tensor-core apply). b is formed with the FP64 mass apply (the oracle would
    need minutes at this size; the solves are judged by their own FP64
    residual)."""
    K = args.solve_elements
    patch, ustar = I.make_patch(3, 5, K, noise_amp=0.2 / K, seed=0)
    t0 = time.perf_counter()
    plan = G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16, G.TF32))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    us = torch.as_tensor(ustar, device="cuda")
    b = torch.empty_like(us)
    plan.apply(G.MASS, us, b, prec=G.FP64)
    x = torch.zeros_like(b)
    plan.cg_solve(b, x, inner_prec=G.FP32, rtol=1e-2)      # warm-up; computes the Jacobi diagonal
    runs = {}
    for name, prec in (("mixed_fp32_in_fp64_ir", G.FP32), ("all_fp64", G.FP64),
                       ("mixed_bf16_in_fp64_ir", G.BF16), ("mixed_tf32_in_fp64_ir", G.TF32)):
        x = torch.zeros_like(b)
        runs[name] = plan.cg_solve(b, x, inner_prec=prec, rtol=1e-10, inner_rtol=1e-4)
    ok = plan.device_status() == 0
    N = plan.num_dofs
    plan.close()
    torch.cuda.empty_cache()
    mixed, full = runs["mixed_fp32_in_fp64_ir"], runs["all_fp64"]
    return {"workload": "Dirichlet solve",
            "metric": "time to 1e-10 relative residual, Jacobi-PCG, homogeneous Dirichlet",
            "value": round(mixed["seconds"], 4), "unit": "s", "higher_is_better": False,
            "config": "perturbed unit cube d=3, order p=5, %d^3 elements (%d dofs), a=1, "
                      "b = M u*, u* ~ U[-1,1] seed 0; inner_rtol 1e-4" % (K, N),
            "runs": runs, "speedup_vs_fp64": round(full["seconds"] / mixed["seconds"], 3),
            "faster_than_fp64": bool(mixed["converged"] and mixed["seconds"] < full["seconds"]),
            "setup_s": round(setup_s, 3), "device_status": "ok" if ok else "a bounded wait ran out"}


def batch_entry(args, G, I, torch, hbm):
    """256 independent d=3 patches (seed 7; 8..48 elements per direction, p = 2..6,
    constant a ~ U[0.5, 2]), FP32 stiffness, applied as one CUDA graph launch.
    Tile shape and kernel variant per (order, patch shape class) come from the
    library autotuner run on the largest patch of that class; the persistent
    schedule is timed beside it."""
    import numpy as np
    patches = I.config_batch()

    def shape_class(pt):
        """(order, shape): 'cube' when the element counts differ by at most 2x,
        else the thin direction (the one with the fewest elements)."""
        K = pt.elements_per_dir
        return pt.orders[0], ("cube" if max(K) <= 2 * min(K) else "thin%d" % int(np.argmin(K)))

    t0 = time.perf_counter()
    tuned = {}
    for key in sorted({shape_class(pt) for pt, _ in patches}):
        big = max((pt for pt, _ in patches if shape_class(pt) == key), key=lambda q: q.num_quad_points)
        tile, variant, ms = G.autotune(big, op=G.STIFFNESS, prec=G.FP32, repeats=5)
        tuned[key] = {"tile": tile, "variant": variant, "ms_on_largest": round(ms, 4),
                      "patches": sum(1 for pt, _ in patches if shape_class(pt) == key)}
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    plans = [G.Plan.from_patch(pt, precisions=(G.FP32,), tile=tuned[shape_class(pt)]["tile"],
                               kernel_variant=tuned[shape_class(pt)]["variant"]) for pt, _ in patches]
    setup_s = time.perf_counter() - t0
    u = np.concatenate([u for _, u in patches])
    ud = torch.as_tensor(u, device="cuda").float()
    vd = torch.empty_like(ud)
    stream = torch.cuda.current_stream()
    batch = G.Batch(plans, op=G.STIFFNESS, prec=G.FP32)
    for _ in range(5):
        batch.apply(ud, vd, stream=stream)
    steps = 50
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
    alg = 24 * batch.total_quad_points + 8 * batch.total_dofs
    ok = all(plan.device_status() == 0 for plan in plans)
    batch.close()
    for plan in plans:
        plan.close()
    torch.cuda.empty_cache()
    # the same patches in one persistent launch over the (patch, tile) work list
    # (plans with the persistent tile of their order, register-prefetch kernel)
    pplans = [G.Plan.from_patch(pt, precisions=(G.FP32,), tile=G.batch_persistent_tile(pt.orders[0]),
                                kernel_variant=G.KERNEL_REGISTERS) for pt, _ in patches]
    with G.Batch(pplans, op=G.STIFFNESS, prec=G.FP32, schedule=G.BATCH_PERSISTENT) as pb:
        for _ in range(5):
            pb.apply(ud, vd, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pb.apply(ud, vd, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1) / steps
    ok = ok and all(plan.device_status() == 0 for plan in pplans)
    for plan in pplans:
        plan.close()
    torch.cuda.empty_cache()
    out = {
        "workload": "batched patches",
        "metric": "batched 3D stiffness apply GDoF/s (256 uneven patches, one graph launch)",
        "value": round(batch.total_dofs / (ms * 1e-3) / 1e9, 4), "unit": "GDoF/s",
        "steps": steps, "ms_per_step": round(ms, 4), "prec": "fp32",
        "config": "256 patches from seed 7: 8..48 elements per direction, p = 2..6, a ~ U[0.5, 2]; "
                  "%d dofs, %d quadrature points" % (batch.total_dofs, batch.total_quad_points),
        "launch_groups": batch.launch_groups,
        "tuned": {"p=%d %s" % k: v for k, v in tuned.items()},
        "tuning": "autotuner per (order, patch shape class) on the class's largest patch",
        "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(alg / (ms * 1e-3) / 1e9 / hbm, 4),
                     "note": "whole graph (tile kernels + gather), algorithmic bytes 24 B/qp + 8 B/dof"},
        "sequential_individual_applies_ms": round(ms_seq, 4),
        "persistent": {"ms_per_step": round(ms_p, 4),
                       "value": round(batch.total_dofs / (ms_p * 1e-3) / 1e9, 4),
                       "note": "one persistent launch over the (patch, tile) work list, tiles "
                               "8x8x4 / 8x4x4 / 4x4x4 / 4x4x4 / 2x2x8 for p = 2..6, then the gather"},
        "autotune_s": round(tune_s, 2), "setup_s": round(setup_s, 2),
        "device_status": "ok" if ok else "a bounded wait ran out"}
    return out


def run_solve(args):
    import torch
    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = solve_entry(args, G, I, torch)
    r.update({"n_gpus": 1, "data": "synthetic"})
    print(json.dumps(r), flush=True)


def run_batch(args):
    import torch
    from paper_1809_05471_gb300 import igasf as G
    from paper_1809_05471_gb300 import inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = batch_entry(args, G, I, torch, float(measured_peaks()[0]["hbm_gbs"]))
    r.update({"n_gpus": 1, "data": "synthetic", "dtype": "f32"})
    print(json.dumps(r), flush=True)


def run_reference(args):
    """The oracle as it stands, on the host cores, on the same workload and metric:
    each step is one FP64 CSR product v = A u (orc_spmv, OpenMP over rows, all
    cores) on a matrix of the workload's size whose rows are copies of a sample of
    the workload's rows assembled by the oracle from the definition (the whole
    matrix would take the row-wise oracle minutes to assemble)."""
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
    layers = 3
    rows, rp, ci, va, t_asm = csr_sample(patch, op, layers, cores)
    N = patch.num_dofs
    big = full_size_csr(rp, ci, va, N)
    O.set_threads(cores)
    for _ in range(args.warmup):
        O.spmv(*big, u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.spmv(*big, u)
    dt_s = time.perf_counter() - t0
    value = N * args.steps / dt_s / 1e9
    sample = ("orc_spmv (OpenMP over rows, %d cores) of a %d-row, %d-nonzero FP64 CSR matrix (the "
              "workload's size) made of copies of %d rows (%d dof layers) assembled row by row "
              "from the definition by the oracle (%.1f s, not timed)"
              % (cores, N, int(big[0][-1]), len(rows), layers, t_asm))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle CSR SpMV",
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
