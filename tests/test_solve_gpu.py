"""Jacobi-PCG and mixed-precision iterative refinement (GPU) against a direct
solve of the oracle's assembled stiffness matrix (homogeneous Dirichlet: the
interior block K_II), and against each other."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _interior_mask(patch):
    Ns = patch.dofs_per_dir
    idx = np.arange(patch.num_dofs)
    i0, i1, i2 = idx % Ns[0], (idx // Ns[0]) % Ns[1], idx // (Ns[0] * Ns[1])
    return (i0 > 0) & (i0 < Ns[0] - 1) & (i1 > 0) & (i1 < Ns[1] - 1) & (i2 > 0) & (i2 < Ns[2] - 1)


@pytest.mark.parametrize("p,K", [(3, 6), (4, 5)])
def test_cg_matches_direct_interior_solve(p, K):
    import torch
    patch, u = I.config_cube(p=p, K=K)
    rp, ci, va = O.assemble_csr(patch, O.STIFFNESS)
    A = sp.csr_matrix((va, ci, rp), shape=(patch.num_dofs,) * 2)
    m = _interior_mask(patch)
    rng = np.random.default_rng(4)
    b = rng.uniform(-1, 1, patch.num_dofs)
    b[~m] = 0.0
    x_ref = np.zeros(patch.num_dofs)
    x_ref[m] = spla.spsolve(A[m][:, m].tocsc(), b[m])
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.BF16)) as plan:
        bd = torch.as_tensor(b, device="cuda")
        for inner in (G.FP64, G.FP32, G.BF16):
            xd = torch.zeros_like(bd)
            rep = plan.cg_solve(bd, xd, inner_prec=inner, rtol=1e-11, inner_rtol=1e-4)
            x = xd.cpu().numpy()
            assert rep["converged"], rep
            assert rep["final_relres"] <= 1e-11
            assert np.all(x[~m] == 0.0)
            # residual of the oracle's matrix at the GPU solution
            res = np.linalg.norm((A[m][:, m] @ x[m]) - b[m]) / np.linalg.norm(b[m])
            assert res < 1e-10, (inner, res)
            assert np.max(np.abs(x - x_ref)) < 1e-7 * np.max(np.abs(x_ref)), inner
            if inner != G.FP64:
                assert rep["outer_iterations"] >= 2


def test_cg_is_deterministic_and_reports_non_convergence():
    import torch
    patch, u = I.config_cube(p=3, K=8)
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32)) as plan:
        b = torch.as_tensor(u, device="cuda")
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        r1 = plan.cg_solve(b, x1, inner_prec=G.FP32, rtol=1e-10)
        r2 = plan.cg_solve(b, x2, inner_prec=G.FP32, rtol=1e-10)
        assert torch.equal(x1, x2) and r1["inner_iterations"] == r2["inner_iterations"]
        x3 = torch.zeros_like(b)
        r3 = plan.cg_solve(b, x3, inner_prec=G.FP64, rtol=1e-10, max_iterations=3)
        assert not r3["converged"] and r3["inner_iterations"] == 3


def test_refined_solve_of_the_solver_workload_shape_checked_by_oracle_rows():
    """The solver workload's shape at half its size (p = 5, 48^3 elements, the
    perturbed cube, a = 1, homogeneous Dirichlet) with FP32 and TF32 inner
    solves in FP64 refinement to 1e-10: on sampled interior rows the oracle's
    residual b_m - (K x)_m, with K from the definition, is within the solve's
    own bound (each |r_m| <= ||r||_2 <= 1e-10 ||b||_2) plus the FP64 rounding of
    the two operators (1e-13 ||K||_inf ||x||_inf)."""
    import torch
    patch, _ = I.make_patch(3, 5, 48, noise_amp=0.2 / 48, seed=0)
    m = _interior_mask(patch)
    rng = np.random.default_rng(11)
    b = rng.uniform(-1, 1, patch.num_dofs)
    b[~m] = 0.0
    idx = np.flatnonzero(m)
    rows = np.sort(rng.choice(idx, 32, replace=False))
    with G.Plan.from_patch(patch, precisions=(G.FP64, G.FP32, G.TF32)) as plan:
        bd = torch.as_tensor(b, device="cuda")
        for inner in (G.FP32, G.TF32):
            xd = torch.zeros_like(bd)
            rep = plan.cg_solve(bd, xd, inner_prec=inner, rtol=1e-10, inner_rtol=1e-4)
            assert rep["converged"] and rep["final_relres"] <= 1e-10, (inner, rep)
            x = xd.cpu().numpy()
            assert np.all(x[~m] == 0.0)
            kx, ra = O.apply_rows(patch, O.STIFFNESS, x, rows)
            r = b[rows] - kx
            bound = 1e-10 * np.linalg.norm(b) + 1e-13 * ra.max() * np.max(np.abs(x))
            assert np.max(np.abs(r)) <= bound, (inner, np.max(np.abs(r)), bound)
