"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only builds inputs: open knot vectors, geometry control points and
the vector u. It holds none of the operator's arithmetic (no basis evaluation,
no quadrature, no geometry factors), so both sides of a parity check can take
their inputs from here without sharing any of the method.

Recipe (the paper's own geometries, a quarter annulus and a bent box of Sec. 7,
are only drawn as figures, so seeded stand-ins are used):

* Knots: open uniform knot vectors on [0, 1] with K elements and order p
  (p = degree + 1, Sec. 1), i.e. p repeats at each end and K - 1 simple interior
  knots, so N = K + p - 1 functions per direction (Sec. 7).
* Identity geometry: control points at the Greville abscissae
  xi*_i = (t_{i+1} + ... + t_{i+p-1}) / (p - 1), which reproduce the map
  G(x) = x exactly.
* Perturbed cube: the identity control points plus uniform noise U[-a, a] on
  every interior control point (all index coordinates in 1..N_delta-2); the
  boundary control points stay put, so the patch is still the unit cube.
* RNG: ``numpy.random.default_rng(seed)``; the noise array of shape
  (N_d, ..., N_1, d) is drawn first (always, also for a = 0), then
  u ~ U[-1, 1] of length N.
* Dofs and quadrature points are lexicographic with the first index fastest
  (the ordering pi of Sec. 3.1): n = n_1 + N_1 (n_2 + N_2 n_3).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

COEF_CONSTANT = 0
COEF_EXP_SIN_COS = 1
COEF_VALUES = 2


@dataclasses.dataclass
class Patch:
    """One tensor-product B-spline patch with its geometry and coefficient."""

    d: int
    orders: List[int]
    knots: List[np.ndarray]          # one open knot vector per direction
    ctrl: np.ndarray                 # (N, d) control points, lexicographic, x fastest
    coef_kind: int = COEF_CONSTANT
    coef_constant: float = 1.0       # a for COEF_CONSTANT
    coef_alpha: float = 0.0          # alpha in exp(alpha sin(2 pi x) cos(2 pi y))
    coef_values: Optional[np.ndarray] = None  # per quadrature point (COEF_VALUES)

    @property
    def dofs_per_dir(self) -> List[int]:
        return [len(t) - p for t, p in zip(self.knots, self.orders)]

    @property
    def num_dofs(self) -> int:
        return int(np.prod(self.dofs_per_dir))

    @property
    def elements_per_dir(self) -> List[int]:
        return [int(np.count_nonzero(np.diff(t) > 0)) for t in self.knots]

    @property
    def quad_per_dir(self) -> List[int]:
        return [k * p for k, p in zip(self.elements_per_dir, self.orders)]

    @property
    def num_quad_points(self) -> int:
        return int(np.prod(self.quad_per_dir))


def open_uniform_knots(p: int, K: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """Open knot vector of order p with K equal elements on [a, b]."""
    if p < 1 or K < 1:
        raise ValueError("need p >= 1 and K >= 1")
    interior = a + (b - a) * np.arange(1, K) / K
    return np.concatenate([np.full(p, a), interior, np.full(p, b)]).astype(np.float64)


def open_knots_from_breaks(p: int, breaks: Sequence[float],
                           mult: Optional[Sequence[int]] = None) -> np.ndarray:
    """Open knot vector of order p over the given break points.

    ``mult`` gives the multiplicity of each interior break (default 1).
    """
    br = np.asarray(breaks, dtype=np.float64)
    if mult is None:
        mult = [1] * (len(br) - 2)
    parts = [np.full(p, br[0])]
    for x, m in zip(br[1:-1], mult):
        parts.append(np.full(m, x))
    parts.append(np.full(p, br[-1]))
    return np.concatenate(parts)


def greville(t: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae of the order-p B-splines on knot vector t."""
    N = len(t) - p
    if p == 1:
        return 0.5 * (t[:N] + t[1:N + 1])
    return np.array([t[i + 1:i + p].mean() for i in range(N)])


def make_patch(d: int, p: int, K, noise_amp: float = 0.0, seed: int = 0,
               coef_kind: int = COEF_CONSTANT, coef_constant: float = 1.0,
               coef_alpha: float = 0.0, knots: Optional[List[np.ndarray]] = None):
    """Build a patch and u from one seeded stream (noise first, then u).

    Returns (patch, u) with u of length N, float64.
    """
    if np.isscalar(K):
        K = [int(K)] * d
    if knots is None:
        knots = [open_uniform_knots(p, int(k)) for k in K]
    orders = [p] * d
    Ns = [len(t) - p for t in knots]
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-noise_amp, noise_amp, size=tuple(reversed(Ns)) + (d,))
    # zero every control point that has an index coordinate on the boundary
    interior = np.ones(tuple(reversed(Ns)), dtype=bool)
    for axis in range(d):
        sl = [slice(None)] * d
        sl[axis] = 0
        interior[tuple(sl)] = False
        sl[axis] = -1
        interior[tuple(sl)] = False
    noise[~interior] = 0.0
    grids = [greville(t, p) for t in knots]
    mesh = np.meshgrid(*reversed(grids), indexing="ij")   # axes (n_d, ..., n_1)
    ctrl = np.stack([mesh[d - 1 - i] for i in range(d)], axis=-1) + noise
    ctrl = np.ascontiguousarray(ctrl.reshape(-1, d))
    N = int(np.prod(Ns))
    u = rng.uniform(-1.0, 1.0, size=N)
    patch = Patch(d=d, orders=orders, knots=[np.asarray(t, np.float64) for t in knots],
                  ctrl=ctrl, coef_kind=coef_kind, coef_constant=coef_constant,
                  coef_alpha=coef_alpha)
    return patch, u


# --- the workloads -----------------------------------------------------------

def config_small_2d():
    """d=2, p=3, 16x16 elements, identity geometry, coefficient 1, seed 0."""
    return make_patch(2, 3, 16, noise_amp=0.0, seed=0)


def config_cube(p: int = 4, K: int = 64, seed: int = 0, coef: bool = True):
    """d=3 perturbed unit cube with noise 0.2/K and a(x)=exp(0.5 sin 2pi x cos 2pi y)."""
    kw = dict(coef_kind=COEF_EXP_SIN_COS, coef_alpha=0.5) if coef else {}
    return make_patch(3, p, K, noise_amp=0.2 / K, seed=seed, **kw)


def sweep_elements(p: int, target_dofs: float = 2.0e6) -> int:
    """Elements per direction so that (K + p - 1)^3 is about the target (K = 127 - p at 2e6)."""
    return int(round(target_dofs ** (1.0 / 3.0))) - p + 1


def config_sweep(p: int, seed: int = 0):
    """Order sweep: d=3, about 2M dofs, same perturbed cube and coefficient."""
    K = sweep_elements(p)
    return config_cube(p=p, K=K, seed=seed)


def scaled_error(v: np.ndarray, v_ref: np.ndarray, a_inf: float, u: np.ndarray) -> float:
    """Max-norm error scaled by ||A||_inf ||u||_inf."""
    den = a_inf * float(np.max(np.abs(u)))
    return float(np.max(np.abs(np.asarray(v, np.float64) - v_ref))) / den


def config_batch(n: int = 256, seed: int = 7):
    """Many independent d=3 patches: elements per direction uniform in 8..48
    (each axis drawn separately), order uniform in 2..6, a constant coefficient
    a ~ U[0.5, 2]. Geometry noise: 0.2 / (largest element count of the patch),
    capped at a third of the patch's smallest Greville gap so that every map stays
    a diffeomorphism. The per-patch parameters come from default_rng(seed); patch i
    draws its noise and u from default_rng(1000 * seed + i)."""
    rng = np.random.default_rng(seed)
    Ks = rng.integers(8, 49, size=(n, 3))
    ps = rng.integers(2, 7, size=n)
    coefs = rng.uniform(0.5, 2.0, size=n)
    out = []
    for i in range(n):
        p, K = int(ps[i]), [int(k) for k in Ks[i]]
        gap = min(np.diff(greville(open_uniform_knots(p, k), p)).min() for k in K)
        amp = min(0.2 / max(K), gap / 3.0)
        out.append(make_patch(3, p, K, noise_amp=amp, seed=1000 * seed + i,
                              coef_constant=float(coefs[i])))
    return out

