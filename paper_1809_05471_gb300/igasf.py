"""Thin ctypes binding of libigasf (include/igasf.h).

Argument marshalling only: every step of setup and apply runs in the CUDA
library. PyTorch supplies device memory and streams. There is no fallback:
if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libigasf.so")

OK = 0
ERR_INVALID_ARG = -1
MAX_ORDER = 9   # IGASF_MAX_ORDER: the orders the kernels are built for, 2..9
MASS = 0
STIFFNESS = 1
FP64 = 0
FP32 = 1
BF16 = 2        # bfloat16-stored factors, float32 vectors and arithmetic
TF32 = 3        # FP32 factors; direction-3 contractions on tensor cores, TF32 operands
BF16_MMA = 4    # bfloat16-stored factors; direction-3 contractions on tensor cores, bf16 operands
COEF_CONSTANT = 0
COEF_EXP_SIN_COS = 1
COEF_VALUES = 2
KERNEL_DEFAULT = 0
KERNEL_REGISTERS = 1
KERNEL_RING = 2
KERNEL_ON_THE_FLY = 3
KERNEL_MMA = 4
BATCH_GRAPH = 0
BATCH_PERSISTENT = 1        # one persistent launch over a (patch, tile) work list
GEOMETRY_STORED = 0
GEOMETRY_ON_THE_FLY = 1     # FP32 applies evaluate the factors inside the tile kernel

ERRORS = {
    -1: "INVALID_ARG", -2: "KNOTS", -3: "GEOMETRY", -4: "UNSUPPORTED", -5: "CUDA",
    -6: "OOM", -7: "TIMEOUT",
}

# every symbol include/igasf.h declares
EXPORTED = [
    "igasf_setup", "igasf_apply", "igasf_apply_prec", "igasf_apply_host", "igasf_apply_host_async",
    "igasf_destroy",
    "igasf_num_dofs", "igasf_num_quad_points", "igasf_describe", "igasf_get_tables",
    "igasf_get_factors", "igasf_quad_points", "igasf_profile_begin", "igasf_profile_end", "igasf_apply_noalloc",
    "igasf_device_status", "igasf_set_test_fault", "igasf_cg_solve",
    "igasf_batch_create", "igasf_batch_create_ex", "igasf_batch_persistent_tile", "igasf_batch_apply", "igasf_batch_info", "igasf_batch_destroy",
    "igasf_autotune", "igasf_list_kernels", "igasf_assembled_nnz", "igasf_assemble_csr",
    "igasf_last_error_message", "igasf_version",
]


class IgasfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("igasf error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class Coef(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("constant", ctypes.c_double),
                ("alpha", ctypes.c_double), ("values", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("precisions", ctypes.c_uint), ("default_prec", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("kernel_variant", ctypes.c_int),
                ("geometry", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class CgReport(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("inner_iterations", ctypes.c_int), ("final_relres", ctypes.c_double),
                ("seconds", ctypes.c_double)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("order", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("tiles", ctypes.c_int * 3), ("threads_per_block", ctypes.c_int),
                ("num_dofs", ctypes.c_int64), ("num_quad_points", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int64 * 2), ("workspace_bytes", ctypes.c_int64),
                ("smem_bytes", ctypes.c_size_t * 2), ("kernel_variant", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libigasf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libigasf.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.igasf_setup.argtypes = [ctypes.c_int, ip, ip, ctypes.POINTER(dp), dp,
                                ctypes.POINTER(Coef), ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.igasf_apply.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.igasf_apply_prec.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.igasf_apply_host.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.igasf_apply_host_async.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.igasf_destroy.argtypes = [vp]
    lib.igasf_num_dofs.argtypes = [vp]
    lib.igasf_num_dofs.restype = ctypes.c_int64
    lib.igasf_num_quad_points.argtypes = [vp]
    lib.igasf_num_quad_points.restype = ctypes.c_int64
    lib.igasf_describe.argtypes = [vp, ctypes.c_int, ctypes.POINTER(PlanDesc)]
    lib.igasf_get_tables.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp]
    lib.igasf_get_factors.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    lib.igasf_quad_points.argtypes = [vp, dp]
    lib.igasf_apply_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.igasf_cg_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.POINTER(CgReport), vp]
    lib.igasf_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(vp)]
    lib.igasf_batch_create_ex.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(vp)]
    lib.igasf_batch_persistent_tile.argtypes = [ctypes.c_int, ctypes.c_int, ip]
    lib.igasf_batch_apply.argtypes = [vp, vp, vp, vp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.igasf_batch_info.argtypes = [vp, i64p, i64p, i64p, ip]
    lib.igasf_batch_destroy.argtypes = [vp]
    lib.igasf_autotune.argtypes = [ctypes.c_int, ip, ip, ctypes.POINTER(dp), dp, ctypes.POINTER(Coef),
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, dp]
    lib.igasf_list_kernels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip,
                                       ctypes.c_int]
    lib.igasf_assembled_nnz.argtypes = [vp]
    lib.igasf_assembled_nnz.restype = ctypes.c_int64
    lib.igasf_assemble_csr.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_size_t, vp]
    lib.igasf_device_status.argtypes = [vp, ctypes.c_int]
    lib.igasf_set_test_fault.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    lib.igasf_profile_begin.argtypes = [vp, ctypes.c_int]
    lib.igasf_profile_end.argtypes = [vp, dp, ip]
    lib.igasf_last_error_message.restype = ctypes.c_char_p
    lib.igasf_version.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        msg = load_library().igasf_last_error_message().decode(errors="replace")
        raise IgasfError(rc, msg)


def _dptr(a: Optional[np.ndarray]):
    dp = ctypes.POINTER(ctypes.c_double)
    return a.ctypes.data_as(dp) if a is not None else ctypes.cast(None, dp)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A setup handle: igasf_setup on construction, igasf_destroy on close()."""

    def __init__(self, d: int, orders: Sequence[int], knots: Sequence[np.ndarray],
                 ctrl: np.ndarray, coef_kind: int = COEF_CONSTANT, coef_constant: float = 1.0,
                 coef_alpha: float = 0.0, coef_values: Optional[np.ndarray] = None,
                 precisions: Sequence[int] = (FP64,), default_prec: Optional[int] = None,
                 tile: Optional[Sequence[int]] = None, kernel_variant: int = 0,
                 geometry: int = GEOMETRY_STORED):
        lib = load_library()
        self.d = d
        self._orders = (ctypes.c_int * d)(*orders)
        self._knots = [np.ascontiguousarray(t, dtype=np.float64) for t in knots]
        self._lens = (ctypes.c_int * d)(*[len(t) for t in self._knots])
        dp = ctypes.POINTER(ctypes.c_double)
        self._kptrs = (dp * d)(*[_dptr(t) for t in self._knots])
        self._ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1)
        self._coef_values = None if coef_values is None else \
            np.ascontiguousarray(coef_values, dtype=np.float64)
        coef = Coef(coef_kind, coef_constant, coef_alpha, _dptr(self._coef_values))
        opt = Options()
        bits = 0
        for p in precisions:
            bits |= 1 << int(p)
        opt.precisions = bits
        opt.default_prec = int(precisions[0] if default_prec is None else default_prec)
        if tile is not None:
            for i, s in enumerate(tile):
                opt.tile[i] = int(s)
        opt.kernel_variant = int(kernel_variant)
        opt.geometry = int(geometry)
        h = ctypes.c_void_p()
        _check(lib.igasf_setup(d, self._orders, self._lens, self._kptrs, _dptr(self._ctrl),
                               ctypes.byref(coef), ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h
        self.precisions = tuple(int(p) for p in precisions)
        self.num_dofs = int(lib.igasf_num_dofs(h))
        self.num_quad_points = int(lib.igasf_num_quad_points(h))

    @classmethod
    def from_patch(cls, patch, **kw):
        return cls(patch.d, patch.orders, patch.knots, patch.ctrl, coef_kind=patch.coef_kind,
                   coef_constant=patch.coef_constant, coef_alpha=patch.coef_alpha,
                   coef_values=patch.coef_values, **kw)

    def _h(self):
        if self.handle is None:
            raise RuntimeError("plan is closed")
        return self.handle

    def apply(self, op: int, u, v, prec: int = FP64, stream=None):
        """v = A u on device tensors (float64 for FP64, float32 for the others)."""
        _check(load_library().igasf_apply_prec(self._h(), int(op), int(prec), u.data_ptr(),
                                               v.data_ptr(), _stream_handle(stream)))
        return v

    def apply_default(self, op: int, u, v, stream=None):
        _check(load_library().igasf_apply(self._h(), int(op), u.data_ptr(), v.data_ptr(),
                                          _stream_handle(stream)))
        return v

    def apply_noalloc(self, op: int, u, v, prec: int = FP64, stream=None):
        """v = A u with the library's static scratch instead of the plan's
        workspace (for callers that must not allocate device memory)."""
        _check(load_library().igasf_apply_noalloc(self._h(), int(op), int(prec), u.data_ptr(),
                                                  v.data_ptr(), _stream_handle(stream)))
        return v

    def apply_host(self, op: int, u, v, prec: int = FP64, stream=None):
        """v = A u with host arrays (numpy or pinned CPU tensors); synchronous."""
        up = u.ctypes.data if isinstance(u, np.ndarray) else u.data_ptr()
        vp = v.ctypes.data if isinstance(v, np.ndarray) else v.data_ptr()
        _check(load_library().igasf_apply_host(self._h(), int(op), int(prec), up, vp,
                                               _stream_handle(stream)))
        return v

    def apply_host_async(self, op: int, u, v, prec: int = FP64, stream=None):
        """Enqueue v = A u for host arrays (pinned CPU tensors or numpy arrays);
        v is valid after the stream is synchronised."""
        up = u.ctypes.data if isinstance(u, np.ndarray) else u.data_ptr()
        vp = v.ctypes.data if isinstance(v, np.ndarray) else v.data_ptr()
        _check(load_library().igasf_apply_host_async(self._h(), int(op), int(prec), up, vp,
                                                     _stream_handle(stream)))
        return v

    def describe(self, prec: int = FP64) -> dict:
        d = PlanDesc()
        _check(load_library().igasf_describe(self._h(), int(prec), ctypes.byref(d)))
        return dict(d=d.d, order=d.order, tile=list(d.tile), tiles=list(d.tiles),
                    threads_per_block=d.threads_per_block, num_dofs=d.num_dofs,
                    num_quad_points=d.num_quad_points,
                    factor_bytes=[int(x) for x in d.factor_bytes],
                    workspace_bytes=int(d.workspace_bytes),
                    smem_bytes=[int(x) for x in d.smem_bytes],
                    kernel_variant=int(d.kernel_variant))

    def tables(self, direction: int):
        """(nodes, weights, B[Q, p], dB[Q, p]) of one direction, FP64 from the device."""
        desc = self.describe(self.precisions[0])
        p = desc["order"]
        # Q of this direction from the knot vector: p points per non-empty span
        Q = int(np.count_nonzero(np.diff(np.asarray(self._knots[direction])) > 0)) * p
        nodes, weights = np.zeros(Q), np.zeros(Q)
        B, dB = np.zeros((Q, p)), np.zeros((Q, p))
        _check(load_library().igasf_get_tables(self._h(), direction, _dptr(nodes), _dptr(weights),
                                               _dptr(B), _dptr(dB)))
        return nodes, weights, B, dB

    def quad_points(self) -> np.ndarray:
        """Physical quadrature points G(x_q), (num_quad_points, d), lexicographic."""
        out = np.zeros((self.num_quad_points, self.d))
        _check(load_library().igasf_quad_points(self._h(), _dptr(out)))
        return out

    def factors(self, op: int, prec: int = FP64) -> np.ndarray:
        nf = 1 if op == MASS else self.d * (self.d + 1) // 2
        out = np.zeros(self.num_quad_points * nf)
        _check(load_library().igasf_get_factors(self._h(), int(op), int(prec), _dptr(out)))
        return out.reshape(self.num_quad_points, nf) if nf > 1 else out

    def cg_solve(self, b, x, inner_prec: int = FP32, rtol: float = 1e-10,
                 inner_rtol: float = 1e-4, max_iterations: int = 200000, stream=None) -> dict:
        """Solve K x = b (homogeneous Dirichlet) on device float64 tensors."""
        rep = CgReport()
        _check(load_library().igasf_cg_solve(self._h(), int(inner_prec), b.data_ptr(), x.data_ptr(),
                                             float(rtol), float(inner_rtol), int(max_iterations),
                                             ctypes.byref(rep), _stream_handle(stream)))
        return dict(converged=bool(rep.converged), outer_iterations=rep.outer_iterations,
                    inner_iterations=rep.inner_iterations, final_relres=rep.final_relres,
                    seconds=rep.seconds)

    def assembled_nnz(self) -> int:
        """Stored entries of the assembled matrix (Corollary on nnz)."""
        n = int(load_library().igasf_assembled_nnz(self._h()))
        if n < 0:
            _check(n)
        return n

    def assemble_csr(self, op: int, workspace_limit_bytes: int = 0, stream=None):
        """FP64 CSR of the operator, assembled on the device by sum
        factorization (Alg. 1): (rowptr, colind, values) as device tensors
        (int64, int64, float64). The plan must store FP64."""
        import torch
        nnz = self.assembled_nnz()
        dev = torch.device("cuda", torch.cuda.current_device())
        rowptr = torch.empty(self.num_dofs + 1, dtype=torch.int64, device=dev)
        colind = torch.empty(nnz, dtype=torch.int64, device=dev)
        values = torch.empty(nnz, dtype=torch.float64, device=dev)
        _check(load_library().igasf_assemble_csr(self._h(), int(op), rowptr.data_ptr(),
                                                 colind.data_ptr(), values.data_ptr(),
                                                 int(workspace_limit_bytes), _stream_handle(stream)))
        return rowptr, colind, values
    def device_status(self, clear: bool = True) -> int:
        """IGASF_OK (0) or IGASF_ERR_TIMEOUT (-7) if a bounded device wait ran out."""
        return int(load_library().igasf_device_status(self._h(), int(clear)))

    def set_test_fault(self, skip_slab: int = -1, wait_limit_cycles: int = 2000000000):
        _check(load_library().igasf_set_test_fault(self._h(), int(skip_slab),
                                                   int(wait_limit_cycles)))

    def profile_begin(self, max_applies: int):
        _check(load_library().igasf_profile_begin(self._h(), int(max_applies)))

    def profile_end(self):
        """Summed (tile kernel ms, gather ms) and the number of applies timed."""
        ms = np.zeros(2)
        n = ctypes.c_int(0)
        _check(load_library().igasf_profile_end(self._h(), _dptr(ms), ctypes.byref(n)))
        return float(ms[0]), float(ms[1]), int(n.value)

    def close(self):
        if self.handle is not None:
            _check(load_library().igasf_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def list_kernels(d: int, p: int, prec: int, geometry: int = GEOMETRY_STORED):
    """The compiled (tile, kernel variant) candidates of (d, p, prec), default first."""
    lib = load_library()
    n = lib.igasf_list_kernels(int(d), int(p), int(prec), int(geometry), None, None, 0)
    if n < 0:
        _check(n)
    tiles = (ctypes.c_int * (3 * max(n, 1)))()
    variants = (ctypes.c_int * max(n, 1))()
    lib.igasf_list_kernels(int(d), int(p), int(prec), int(geometry), tiles, variants, n)
    return [(list(tiles[3 * i:3 * i + 3]), int(variants[i])) for i in range(n)]


def autotune(patch, op: int = STIFFNESS, prec: int = FP32, repeats: int = 5):
    """Fastest compiled (tile, kernel variant) for this patch, and its ms per apply."""
    lib = load_library()
    d = patch.d
    knots = [np.ascontiguousarray(t, dtype=np.float64) for t in patch.knots]
    dp = ctypes.POINTER(ctypes.c_double)
    kptrs = (dp * d)(*[_dptr(t) for t in knots])
    lens = (ctypes.c_int * d)(*[len(t) for t in knots])
    orders = (ctypes.c_int * d)(*patch.orders)
    ctrl = np.ascontiguousarray(patch.ctrl, dtype=np.float64).reshape(-1)
    cv = None if patch.coef_values is None else np.ascontiguousarray(patch.coef_values, np.float64)
    coef = Coef(patch.coef_kind, patch.coef_constant, patch.coef_alpha, _dptr(cv))
    tile = (ctypes.c_int * 3)()
    variant = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib.igasf_autotune(d, orders, lens, kptrs, _dptr(ctrl), ctypes.byref(coef), int(op),
                              int(prec), int(repeats), tile, ctypes.byref(variant),
                              ctypes.byref(ms)))
    return list(tile), int(variant.value), float(ms.value)


def batch_persistent_tile(p: int, prec: int = FP32):
    """Tile shape the persistent batch schedule runs for order p (host-only)."""
    t = (ctypes.c_int * 3)()
    _check(load_library().igasf_batch_persistent_tile(int(p), int(prec), t))
    return [int(x) for x in t]


class Batch:
    """igasf_batch over plans (which must outlive it): one graph launch per apply."""

    def __init__(self, plans: Sequence[Plan], op: int = STIFFNESS, prec: int = FP32,
                 schedule: int = BATCH_GRAPH):
        lib = load_library()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h().value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.igasf_batch_create_ex(len(self.plans), arr, int(op), int(prec), int(schedule),
                                         ctypes.byref(h)))
        self.handle = h
        self.offsets = np.cumsum([0] + [p.num_dofs for p in self.plans])
        td, tq, fb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ng = ctypes.c_int()
        _check(lib.igasf_batch_info(h, ctypes.byref(td), ctypes.byref(tq), ctypes.byref(fb),
                                    ctypes.byref(ng)))
        self.total_dofs, self.total_quad_points = int(td.value), int(tq.value)
        self.factor_bytes, self.launch_groups = int(fb.value), int(ng.value)

    def apply(self, u, v, stream=None):
        _check(load_library().igasf_batch_apply(self.handle, u.data_ptr(), v.data_ptr(),
                                                _stream_handle(stream)))
        return v

    def close(self):
        if self.handle is not None:
            _check(load_library().igasf_batch_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

