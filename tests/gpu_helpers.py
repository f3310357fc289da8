"""Shared helpers of the GPU tests: run the CUDA path through the C-ABI binding
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I

TOL = {G.FP64: 1e-12, G.FP32: 1e-5}
DTYPE = {G.FP64: "float64", G.FP32: "float32", G.BF16: "float32", G.TF32: "float32",
         G.BF16_MMA: "float32"}
# unit roundoff of the tensor-core operand formats (round to nearest): TF32
# keeps 11 significant bits, bfloat16 8
UNIT_ROUNDOFF = {G.TF32: 2.0 ** -11, G.BF16_MMA: 2.0 ** -8}


def tol(prec, patch_or_p):
    """Scaled max-norm bar of an apply against the oracle at order p.

    FP64: 1e-12 (sum factorization reaches the assembled quadrature operator up
    to rounding, Sec. 1 and Sec. 8).
    FP32 (and BF16 against the oracle's operator with the same rounded factors,
    whose arithmetic is FP32 too): the longest accumulation chain of one output
    has about 6p + 9 terms (three forward sweeps of p terms, the 3-term product
    with the factors, three transposed sweeps), so first-order rounding gives
    (6p + 9) 2^-24 relative to the absolute terms; the bar is twice that
    (2.5e-6 at p = 2, 7.5e-6 at p = 9).
    TF32 and BF16_MMA (tensor-core direction-3 sweeps; BF16_MMA against the
    oracle's operator with bfloat16-rounded factors): every product of the two
    direction-3 contractions has both operands rounded once to the operand
    format, a relative perturbation of at most 2u each, so to first order the
    error is at most 4u times the absolute-value operator applied to |u|; the
    bar takes that bound with the absolute operator's row sums at ||A||_inf,
    i.e. 4u (TF32 2.0e-3, BF16 1.6e-2), plus the FP32 bar for the rest."""
    p = patch_or_p if isinstance(patch_or_p, (int, np.integer)) else int(patch_or_p.orders[0])
    if prec == G.FP64:
        return TOL[G.FP64]
    fp32 = 2.0 * (6 * p + 9) * 2.0 ** -24
    if prec in UNIT_ROUNDOFF:
        return 4.0 * UNIT_ROUNDOFF[prec] + fp32
    return fp32


def gpu_apply(plan, op, u, prec):
    import torch
    dt = getattr(torch, DTYPE[prec])
    ud = torch.as_tensor(np.asarray(u), device="cuda").to(dt)
    vd = torch.empty_like(ud)
    plan.apply(op, ud, vd, prec=prec)
    torch.cuda.synchronize()
    assert plan.device_status() == 0, "a bounded device wait ran out"
    return vd.double().cpu().numpy()


def oracle_full(patch, op, u, mode="elementwise"):
    """Whole v = A u and ||A||_inf from the oracle."""
    if mode == "csr":
        rp, ci, va = O.assemble_csr(patch, op)
        return O.spmv(rp, ci, va, u), O.csr_inf_norm(rp, va)
    rows = np.arange(patch.num_dofs)
    v, ra = O.apply_rows(patch, op, u, rows)
    return v, float(ra.max())


def sample_rows(patch, n, seed=0):
    """Rows on corners, edges and faces of the dof grid plus random interior ones."""
    Ns = patch.dofs_per_dir
    d = patch.d
    rng = np.random.default_rng(seed)
    picks = set()
    for corner in range(2 ** d):
        idx = [(Ns[a] - 1) if (corner >> a) & 1 else 0 for a in range(d)]
        picks.add(tuple(idx))
    while len(picks) < n:
        idx = []
        for a in range(d):
            r = rng.random()
            if r < 0.15:
                idx.append(int(rng.integers(0, min(Ns[a], 3))))
            elif r < 0.3:
                idx.append(int(Ns[a] - 1 - rng.integers(0, min(Ns[a], 3))))
            else:
                idx.append(int(rng.integers(0, Ns[a])))
        picks.add(tuple(idx))
    rows = []
    for idx in sorted(picks):
        lin, s = 0, 1
        for a in range(d):
            lin += s * idx[a]
            s *= Ns[a]
        rows.append(lin)
    return np.array(sorted(rows), dtype=np.int64)


def scaled_err(v, v_ref, a_inf, u):
    return I.scaled_error(v, v_ref, a_inf, u)
