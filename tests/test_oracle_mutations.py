"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch every one of them (CPU only; the planted copies are built in a
temporary directory and never touch the real oracle)."""
import os
import subprocess

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle as O
from paper_1809_05471_gb300 import inputs as I
from tests import brute

SRC = os.path.join(os.path.dirname(O.__file__), "igasf_oracle.c")

# (name, text in the source, replacement)
MUTATIONS = [
    ("gauss weight factor", "w[n - 1 - i] = 2.0 /", "w[n - 1 - i] = 1.0 /"),
    ("gauss node map", "(gx[j] + 1.0) * (hi - lo) / 2.0", "(gx[j] + 1.0) * (hi - lo)"),
    ("cox-de boor index", "(t[i + k] - x) / dr * tmp[i + 1]", "(t[i + k] - x) / dr * tmp[i]"),
    ("derivative factor", "der[i] = (p - 1) * (a - c);", "der[i] = p * (a - c);"),
    ("derivative sign", "der[i] = (p - 1) * (a - c);", "der[i] = (p - 1) * (c - a);"),
    ("dropped weight", "out->w *= P->wq[a][q[a]];", "out->w *= 1.0;"),
    ("dropped |det J| in mass", "out->FM = adet;", "out->FM = 1.0;"),
    ("cofactor sign", "double c01 = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);",
     "double c01 = (J[1][0] * J[2][2] - J[1][2] * J[2][0]);"),
    ("transposed inverse", "inv[0][1] = c10 / out->detJ;", "inv[0][1] = c01 / out->detJ;"),
    ("J^-T J^-1 instead of J^-1 J^-T", "s += inv[i][k] * inv[j][k];", "s += inv[k][i] * inv[k][j];"),
    ("coefficient argument", "sin(2.0 * M_PI * out->G[0])", "sin(2.0 * M_PI * out->G[1])"),
    ("stiffness index", "s += dm * g->FK[i][j] * basis_at(P, q, n, j);",
     "s += dm * g->FK[i][j] * basis_at(P, q, n, i);"),
    ("transposed operand in J", "out->J[i][j] += c * dphi;", "out->J[j][i] += c * dphi;"),
    ("row support window", "ehi[a] = m[a] + P->p[a] - 1;", "ehi[a] = m[a] + P->p[a] - 2;"),
    ("point apply: test function derivative direction",
     "else for (int i = 0; i < d; ++i) c += basis_at(&P, q, m, i) * gk[i];",
     "else for (int i = 0; i < d; ++i) c += basis_at(&P, q, m, 0) * gk[i];"),
    ("point apply: transposed factor",
     "double wf = g.w * g.FK[i][j];", "double wf = g.w * g.FK[j][i] * (i == j ? 1.0 : 0.5);"),
    ("point apply: a layer class skipped",
     "for (int cls = 0; cls < pe[last]; ++cls) {", "for (int cls = 1; cls < pe[last]; ++cls) {"),
    ("stored stiffness factor rounded before the weight",
     "orc_round_significand(g->w * g->FK[i][j], stored_bits)",
     "g->w * orc_round_significand(g->FK[i][j], stored_bits)"),
    ("stored mass factor rounded before the weight",
     "orc_round_significand(g->w * g->FM, stored_bits)",
     "g->w * orc_round_significand(g->FM, stored_bits)"),
    ("rounding halves away from zero", "nearbyint(ldexp(m, bits))", "round(ldexp(m, bits))"),
    ("one significant bit too many", "return ldexp(nearbyint(ldexp(m, bits)), e - bits);",
     "return ldexp(nearbyint(ldexp(m, bits + 1)), e - bits - 1);"),
]


def _quick_pins():
    """A subset of the pins, returning the list of those that failed."""
    failed = []
    x, w = O.gauss_legendre(4)
    xr, wr = np.polynomial.legendre.leggauss(4)
    if not (np.allclose(x, xr, atol=1e-14) and np.allclose(w, wr, atol=1e-14)):
        failed.append("gauss")
    t = I.open_knots_from_breaks(4, [0, 0.3, 0.45, 1.0])
    val, der = O.bspline_all(t, 4, 0.37)
    ref = BSpline.design_matrix([0.37], t, 3).toarray()[0]
    dref = np.array([BSpline(t, np.eye(len(t) - 4)[n], 3).derivative()(0.37)
                     for n in range(len(t) - 4)])
    if not (np.allclose(val, ref, atol=1e-14) and np.allclose(der, dref, atol=1e-12)):
        failed.append("bspline")
    knots = [I.open_knots_from_breaks(3, np.array([0, 0.3, 1.0]) * (1 + 0.1 * a)) for a in range(3)]
    patch, u = I.make_patch(3, 3, 2, noise_amp=0.04, seed=17, knots=knots,
                            coef_kind=I.COEF_EXP_SIN_COS, coef_alpha=0.5)
    for op in (O.MASS, O.STIFFNESS):
        A = O.csr_to_dense(*O.assemble_csr(patch, op), patch.num_dofs)
        Ab = brute.dense_operator(patch, op)
        if not np.max(np.abs(A - Ab)) < 1e-13 * np.max(np.abs(Ab)):
            failed.append("brute-force op %d" % op)
        rows = np.arange(patch.num_dofs)
        vr, _ = O.apply_rows(patch, op, u, rows)
        if not np.max(np.abs(vr - Ab @ u)) < 1e-13 * np.max(np.abs(Ab @ u)):
            failed.append("rows op %d" % op)
        vq = O.apply_qp(patch, op, u, threads=3)
        if not np.max(np.abs(vq - Ab @ u)) < 1e-13 * np.max(np.abs(Ab @ u)):
            failed.append("point apply op %d" % op)
    # bfloat16-stored factors: ties to even, and the rounded quantity is w F
    if not (O.round_significand(1 + 2.0 ** -8, 8) == 1.0
            and O.round_significand(1 + 3 * 2.0 ** -8, 8) == 1 + 2.0 ** -6
            and O.round_significand(1 + 2.0 ** -7, 8) == 1 + 2.0 ** -7):
        failed.append("bf16 rounding")
    for op in (O.MASS, O.STIFFNESS):
        with O.stored_factor_bits(O.BF16_BITS):
            A = O.csr_to_dense(*O.assemble_csr(patch, op), patch.num_dofs)
        Ab = brute.dense_operator(patch, op, round_factor=lambda x: np.ldexp(
            np.round(np.frexp(x)[0] * 256.0), np.frexp(x)[1] - 8))
        if not np.max(np.abs(A - Ab)) < 1e-13 * np.max(np.abs(Ab)):
            failed.append("bf16 brute-force op %d" % op)
    return failed


def test_quick_pins_pass_on_the_real_oracle():
    assert _quick_pins() == []


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
                    "-o", str(lib), str(mutated), "-lm"], check=True)
    with O.use_library(str(lib)):
        failed = _quick_pins()
    assert failed, "planted mistake '%s' was not caught by any pin" % name
