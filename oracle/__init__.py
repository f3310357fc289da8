"""FP64 CPU oracle for the isogeometric mass and stiffness operators.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it; the product path never imports it. It shares no code with
the CUDA library (see ``igasf_oracle.c`` for what it computes and where each
step comes from in the paper).

The C library is built with gcc on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igasf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libigasf_oracle.so")
_lib = None

MASS = 0
STIFFNESS = 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _LIB == os.path.join(_BUILD, "libigasf_oracle.so"):
            build()
        lib = ctypes.CDLL(_LIB)
        patch_args = [ctypes.c_int, _ip, _ip, _dp, _dp, ctypes.c_int, ctypes.c_double,
                      ctypes.c_double, _dp]
        lib.orc_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        lib.orc_bspline_all.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
        lib.orc_tables_1d.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.orc_quad_data.argtypes = patch_args + [_dp] * 6
        lib.orc_nnz.argtypes = patch_args
        lib.orc_nnz.restype = ctypes.c_int64
        lib.orc_assemble_csr.argtypes = patch_args + [ctypes.c_int, _lp, _lp, _dp]
        lib.orc_spmv.argtypes = [ctypes.c_int64, _lp, _lp, _dp, _dp, _dp]
        lib.orc_apply_rows.argtypes = patch_args + [ctypes.c_int, _dp, ctypes.c_int64, _lp, _dp,
                                                    _dp, ctypes.c_int]
        lib.orc_apply_elementwise.argtypes = patch_args + [ctypes.c_int, _dp, _dp]
        lib.orc_apply_qp.argtypes = patch_args + [ctypes.c_int, _dp, _dp, ctypes.c_int]
        lib.orc_assemble_rows.argtypes = patch_args + [ctypes.c_int, ctypes.c_int64, _lp, _lp, _lp,
                                                       _dp, ctypes.c_int]
        lib.orc_max_threads.argtypes = []
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_round_significand.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.orc_round_significand.restype = ctypes.c_double
        lib.orc_set_stored_factor_bits.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a, kind=_dp):
    return a.ctypes.data_as(kind) if a is not None else ctypes.cast(None, kind)


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle error %d" % rc)


class _PatchArgs:
    """Keeps the flat arrays alive while a call runs."""

    def __init__(self, patch):
        self.d = int(patch.d)
        self.orders = np.ascontiguousarray(patch.orders, dtype=np.int32)
        self.nks = np.ascontiguousarray([len(t) for t in patch.knots], dtype=np.int32)
        self.knots = np.ascontiguousarray(np.concatenate(patch.knots), dtype=np.float64)
        self.ctrl = np.ascontiguousarray(patch.ctrl, dtype=np.float64).reshape(-1)
        self.coef_values = None if patch.coef_values is None else \
            np.ascontiguousarray(patch.coef_values, dtype=np.float64)
        self.args = (self.d, _ptr(self.orders, _ip), _ptr(self.nks, _ip), _ptr(self.knots),
                     _ptr(self.ctrl), int(patch.coef_kind), float(patch.coef_constant),
                     float(patch.coef_alpha), _ptr(self.coef_values))


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_load().orc_gauss_legendre(n, _ptr(x), _ptr(w)))
    return x, w


def bspline_all(t: np.ndarray, p: int, x: float, deriv: bool = True):
    t = np.ascontiguousarray(t, dtype=np.float64)
    N = len(t) - p
    val = np.zeros(N)
    der = np.zeros(N)
    _check(_load().orc_bspline_all(_ptr(t), len(t), p, float(x), _ptr(val), _ptr(der)))
    return (val, der) if deriv else val


def tables_1d(t: np.ndarray, p: int):
    """Nodes, weights and dense (Q, N) value / derivative tables of one direction."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    K = int(np.count_nonzero(np.diff(t[p - 1:len(t) - p + 1]) > 0))
    Q = K * p
    N = len(t) - p
    xq, wq = np.zeros(Q), np.zeros(Q)
    B, dB = np.zeros((Q, N)), np.zeros((Q, N))
    _check(_load().orc_tables_1d(p, len(t), _ptr(t), _ptr(xq), _ptr(wq), _ptr(B), _ptr(dB)))
    return xq, wq, B, dB


def quad_data(patch):
    """Per quadrature point (lexicographic): w, G, detJ, a, FM, FK (unweighted)."""
    pa = _PatchArgs(patch)
    Qt = patch.num_quad_points
    d = patch.d
    w = np.zeros(Qt)
    G = np.zeros((Qt, d))
    detJ = np.zeros(Qt)
    a = np.zeros(Qt)
    FM = np.zeros(Qt)
    FK = np.zeros((Qt, d, d))
    _check(_load().orc_quad_data(*pa.args, _ptr(w), _ptr(G), _ptr(detJ), _ptr(a), _ptr(FM),
                                 _ptr(FK)))
    return dict(w=w, G=G, detJ=detJ, a=a, FM=FM, FK=FK)


def nnz(patch) -> int:
    pa = _PatchArgs(patch)
    r = _load().orc_nnz(*pa.args)
    if r < 0:
        raise RuntimeError("oracle error %d" % r)
    return int(r)


def assemble_csr(patch, op: int):
    """Assembled matrix as (rowptr, colind, val) numpy arrays."""
    pa = _PatchArgs(patch)
    N = patch.num_dofs
    rowptr = np.zeros(N + 1, dtype=np.int64)
    lib = _load()
    _check(lib.orc_assemble_csr(*pa.args, op, _ptr(rowptr, _lp), _ptr(None, _lp), _ptr(None)))
    nz = int(rowptr[-1])
    colind = np.zeros(nz, dtype=np.int64)
    val = np.zeros(nz)
    _check(lib.orc_assemble_csr(*pa.args, op, _ptr(rowptr, _lp), _ptr(colind, _lp), _ptr(val)))
    return rowptr, colind, val


def csr_to_dense(rowptr, colind, val, N):
    A = np.zeros((N, N))
    for r in range(N):
        A[r, colind[rowptr[r]:rowptr[r + 1]]] = val[rowptr[r]:rowptr[r + 1]]
    return A


def spmv(rowptr, colind, val, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(len(rowptr) - 1)
    _check(_load().orc_spmv(len(rowptr) - 1, _ptr(rowptr, _lp), _ptr(colind, _lp), _ptr(val),
                            _ptr(x), _ptr(y)))
    return y


def csr_inf_norm(rowptr, val) -> float:
    absval = np.abs(val)
    return float(np.max(np.add.reduceat(absval, rowptr[:-1]))) if len(val) else 0.0


def apply_rows(patch, op: int, u, rows: Sequence[int], threads: int = 0):
    """Rows of v = A u from the definition; returns (v_rows, row_abs_sums)."""
    pa = _PatchArgs(patch)
    u = np.ascontiguousarray(u, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    v = np.zeros(len(rows))
    ra = np.zeros(len(rows))
    _check(_load().orc_apply_rows(*pa.args, op, _ptr(u), len(rows), _ptr(rows, _lp), _ptr(v),
                                  _ptr(ra), int(threads)))
    return v, ra


def apply_elementwise(patch, op: int, u):
    pa = _PatchArgs(patch)
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.zeros(patch.num_dofs)
    _check(_load().orc_apply_elementwise(*pa.args, op, _ptr(u), _ptr(v)))
    return v


def apply_qp(patch, op: int, u, threads: int = 0):
    """Whole v = A u point by point (value or gradient of u at each quadrature
    point by direct sums, times w F, scattered to the test functions)."""
    pa = _PatchArgs(patch)
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.zeros(patch.num_dofs)
    _check(_load().orc_apply_qp(*pa.args, op, _ptr(u), _ptr(v), int(threads)))
    return v


def assemble_rows(patch, op: int, rows: Sequence[int], threads: int = 0):
    """CSR (rowptr, colind, val) of the selected rows of A, each row from the
    definition; row i of the result is row rows[i] of A."""
    pa = _PatchArgs(patch)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rowptr = np.zeros(len(rows) + 1, dtype=np.int64)
    lib = _load()
    _check(lib.orc_assemble_rows(*pa.args, op, len(rows), _ptr(rows, _lp), _ptr(rowptr, _lp),
                                 _ptr(None, _lp), _ptr(None), int(threads)))
    nz = int(rowptr[-1])
    colind = np.zeros(nz, dtype=np.int64)
    val = np.zeros(nz)
    _check(lib.orc_assemble_rows(*pa.args, op, len(rows), _ptr(rows, _lp), _ptr(rowptr, _lp),
                                 _ptr(colind, _lp), _ptr(val), int(threads)))
    return rowptr, colind, val


def set_threads(n: int):
    """Number of OpenMP threads of later oracle calls that take no `threads`
    argument (the CSR product)."""
    _check(_load().orc_set_threads(int(n)))


def max_threads() -> int:
    return int(_load().orc_max_threads())


BF16_BITS = 8   # significant bits of bfloat16


def round_significand(x: float, bits: int) -> float:
    """x rounded to `bits` significant bits, ties to even (the oracle's rule for
    factors stored in a narrower format)."""
    return float(_load().orc_round_significand(float(x), int(bits)))


class stored_factor_bits:
    """Within the block, every oracle operator uses weighted factors w F rounded
    to `bits` significant bits (8: bfloat16 storage); 0 restores FP64."""

    def __init__(self, bits: int):
        self.bits = int(bits)

    def __enter__(self):
        _check(_load().orc_set_stored_factor_bits(self.bits))
        return self

    def __exit__(self, *exc):
        _check(_load().orc_set_stored_factor_bits(0))
        return False


class use_library:
    """Context manager that points this module at another build of the oracle
    source (used by the tests that plant mistakes in a copy of it)."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib, _LIB
        self.saved = (_lib, _LIB)
        _lib = None
        _LIB = self.path
        return self

    def __exit__(self, *exc):
        global _lib, _LIB
        _lib, _LIB = self.saved
        return False
