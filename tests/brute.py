"""A second, independent dense implementation for tiny patches (tests only).

It shares nothing with the C oracle: the univariate basis comes from
``scipy.interpolate.BSpline``, the Gauss rule from ``numpy.polynomial.legendre``,
determinants and inverses from ``numpy.linalg``. It assembles the dense
quadrature matrix A_mn = sum_x w F d phi_n d phi_m (Sec. 2, eq. quadrature:1)
with einsum over all quadrature points and all functions.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import BSpline


def elements(t, p):
    ks = [k for k in range(p - 1, len(t) - p) if t[k + 1] > t[k]]
    return [(t[k], t[k + 1]) for k in ks]


def tables(t, p):
    """Nodes, weights, dense (Q, N) values and derivatives via scipy."""
    gx, gw = np.polynomial.legendre.leggauss(p)
    xs, ws = [], []
    for lo, hi in elements(t, p):
        xs.append(lo + (gx + 1) * (hi - lo) / 2)
        ws.append(gw * (hi - lo) / 2)
    x = np.concatenate(xs)
    w = np.concatenate(ws)
    N = len(t) - p
    deg = p - 1
    B = np.zeros((len(x), N))
    dB = np.zeros((len(x), N))
    for n in range(N):
        c = np.zeros(N)
        c[n] = 1.0
        s = BSpline(t, c, deg, extrapolate=False)
        B[:, n] = s(x)
        dB[:, n] = s.derivative()(x) if deg > 0 else 0.0
    return x, w, np.nan_to_num(B), np.nan_to_num(dB)


def dense_operator(patch, op, round_factor=None):
    """Dense A (N x N) for op 0 = mass, 1 = stiffness. If given,
    ``round_factor`` maps each array of weighted factors w F (w |det J|, or one
    entry (i, j) of w a |det J| J^-1 J^-T) to the values actually stored."""
    rf = round_factor if round_factor is not None else (lambda x: x)
    d = patch.d
    tabs = [tables(t, p) for t, p in zip(patch.knots, patch.orders)]
    Ns = [tb[2].shape[1] for tb in tabs]
    # full tensor-product basis at all quadrature points, lexicographic (x fastest)
    # value: Phi[q, n]; derivative along direction j: dPhi[j][q, n]
    def kron_rev(mats):
        out = mats[0]
        for M in mats[1:]:
            out = np.kron(M, out)
        return out
    Phi = kron_rev([tb[2] for tb in tabs])
    dPhi = []
    for j in range(d):
        dPhi.append(kron_rev([tabs[a][3] if a == j else tabs[a][2] for a in range(d)]))
    w = kron_rev([tb[1][:, None] for tb in tabs])[:, 0]
    ctrl = patch.ctrl
    G = Phi @ ctrl                                       # (Q, d)
    J = np.stack([dPhi[j] @ ctrl for j in range(d)], axis=2)  # J[q, i, j] = dG_i/dxi_j
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    if patch.coef_kind == 1:
        y = np.cos(2 * np.pi * G[:, 1]) if d > 1 else 1.0
        a = np.exp(patch.coef_alpha * np.sin(2 * np.pi * G[:, 0]) * y)
    elif patch.coef_kind == 2:
        a = np.asarray(patch.coef_values)
    else:
        a = np.full(len(w), patch.coef_constant)
    if op == 0:
        return Phi.T @ (rf(w * np.abs(det))[:, None] * Phi)
    F = (a * np.abs(det))[:, None, None] * np.einsum("qik,qjk->qij", Jinv, Jinv)
    A = np.zeros((Phi.shape[1], Phi.shape[1]))
    for i in range(d):
        for j in range(d):
            A += dPhi[i].T @ (rf(w * F[:, i, j])[:, None] * dPhi[j])
    return A


def univariate_matrices(t, p):
    """1D mass and stiffness (identity geometry) from scipy tables."""
    x, w, B, dB = tables(t, p)
    return B.T @ (w[:, None] * B), dB.T @ (w[:, None] * dB)
