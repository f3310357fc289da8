"""The C-ABI library builds, loads and exports what include/igasf.h declares;
host-side validation rejects bad inputs before any CUDA call (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1809_05471_gb300 import igasf as G
from paper_1809_05471_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "igasf.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(igasf_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_05471_gb300 import build
    build.build()
    return G.load_library()


def test_header_declares_the_binding_list():
    assert _declared_functions() == sorted(G.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (igasf_\w+)", out))
    for name in _declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_version(lib):
    assert lib.igasf_version() == 1


def _setup(lib, d, orders, knots, ctrl, coef=None, opt=None):
    orders_c = (ctypes.c_int * d)(*orders)
    knots = [np.ascontiguousarray(t, dtype=np.float64) for t in knots]
    lens = (ctypes.c_int * d)(*[len(t) for t in knots])
    dp = ctypes.POINTER(ctypes.c_double)
    kp = (dp * d)(*[t.ctypes.data_as(dp) for t in knots])
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = lib.igasf_setup(d, orders_c, lens, kp, ctrl.ctypes.data_as(dp),
                         ctypes.byref(coef) if coef is not None else None,
                         ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    return rc, h


def _patch(d=3, p=3, K=2):
    patch, _ = I.make_patch(d, p, K)
    return patch


def test_rejects_bad_dimension_and_orders(lib):
    pt = _patch()
    rc, h = _setup(lib, 4, [3] * 4, pt.knots + [pt.knots[0]], pt.ctrl)
    assert rc == -4 and h.value is None
    rc, _ = _setup(lib, 3, [3, 3, 4], pt.knots, pt.ctrl)
    assert rc == -4
    assert b"orders differ" in lib.igasf_last_error_message()
    rc, _ = _setup(lib, 3, [0, 0, 0], pt.knots, pt.ctrl)
    assert rc == -1
    big = I.make_patch(3, 10, 1)[0]
    rc, _ = _setup(lib, 3, [10] * 3, big.knots, big.ctrl)
    assert rc == -4


def test_rejects_bad_knots(lib):
    pt = _patch()
    t = pt.knots[0].copy()
    dec = t.copy()
    dec[3], dec[4] = dec[4], dec[3] + 0.5
    rc, _ = _setup(lib, 3, [3] * 3, [dec, t, t], pt.ctrl)
    assert rc == -2
    not_open = t.copy()
    not_open[1] = 0.01
    rc, _ = _setup(lib, 3, [3] * 3, [not_open, t, t], pt.ctrl)
    assert rc == -2
    rc, _ = _setup(lib, 3, [3] * 3, [t[:4], t, t], pt.ctrl)
    assert rc == -2
    nan = t.copy()
    nan[3] = np.nan
    rc, _ = _setup(lib, 3, [3] * 3, [nan, t, t], pt.ctrl)
    assert rc == -2
    # interior multiplicity == order: not an open knot vector of this order
    full = I.open_knots_from_breaks(3, [0, 0.5, 1], [3])
    rc, _ = _setup(lib, 3, [3] * 3, [full, t, t], pt.ctrl)
    assert rc == -2
    # repeated interior knot below the order: passes the host validation (without
    # a GPU the setup then stops at its first CUDA call)
    rep = I.open_knots_from_breaks(3, [0, 0.5, 1], [2])
    prep, _ = I.make_patch(3, 3, 2, knots=[rep, t, t])
    rc, h = _setup(lib, 3, [3] * 3, prep.knots, prep.ctrl)
    assert rc in (0, -5), rc
    if rc == 0:
        lib.igasf_destroy(h)


def test_rejects_null_and_bad_options(lib):
    pt = _patch()
    h = ctypes.c_void_p()
    assert lib.igasf_setup(3, None, None, None, None, None, None, ctypes.byref(h)) == -1
    assert lib.igasf_setup(3, None, None, None, None, None, None, None) == -1
    opt = G.Options()
    opt.reserved[0] = 1
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -1
    opt = G.Options()
    opt.default_prec = 7
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -1
    opt = G.Options()
    opt.precisions = 1 << 5
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -1
    opt = G.Options()
    opt.tile[0] = 3          # not a built tile shape
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -4
    coef = G.Coef(G.COEF_VALUES, 0.0, 0.0, ctypes.cast(None, ctypes.POINTER(ctypes.c_double)))
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, coef=coef)
    assert rc == -1
    coef = G.Coef(9, 0.0, 0.0, ctypes.cast(None, ctypes.POINTER(ctypes.c_double)))
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, coef=coef)
    assert rc == -1


def test_rejects_bad_geometry_options(lib):
    """Factors on the fly: a known mode, FP32 stored, d = 3, and a coefficient
    the kernel can evaluate; all checked on the host before any device work."""
    pt = _patch()
    opt = G.Options()
    opt.geometry = 5
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -1
    opt = G.Options()
    opt.geometry = G.GEOMETRY_ON_THE_FLY            # default precisions: FP64 only
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -1
    assert b"FP32" in lib.igasf_last_error_message()
    opt.precisions = 1 << G.FP32
    opt.default_prec = G.FP32
    vals = np.ones(8)
    coef = G.Coef(G.COEF_VALUES, 0.0, 0.0, vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, coef=coef, opt=opt)
    assert rc == -4
    p2, _ = I.make_patch(2, 3, 4, seed=0)
    rc, _ = _setup(lib, 2, [3] * 2, p2.knots, p2.ctrl, opt=opt)
    assert rc == -4
    opt = G.Options()
    opt.kernel_variant = G.KERNEL_MMA               # valid, but FP64 has no tensor-core kernel
    rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
    assert rc == -4
    for kv in (G.KERNEL_ON_THE_FLY, 5, -1):     # not selectable as kernel variants
        opt = G.Options()
        opt.kernel_variant = kv
        rc, _ = _setup(lib, 3, [3] * 3, pt.knots, pt.ctrl, opt=opt)
        assert rc == -1


def test_null_handle_calls(lib):
    assert lib.igasf_apply(None, 0, None, None, None) == -1
    assert lib.igasf_apply_prec(None, 0, 0, None, None, None) == -1
    assert lib.igasf_apply_host(None, 0, 0, None, None, None) == -1
    assert lib.igasf_apply_host_async(None, 0, 0, None, None, None) == -1
    assert lib.igasf_destroy(None) == 0
    assert lib.igasf_num_dofs(None) == -1
    assert lib.igasf_num_quad_points(None) == -1
    assert lib.igasf_describe(None, 0, None) == -1
    assert lib.igasf_get_tables(None, 0, None, None, None, None) == -1
    assert lib.igasf_get_factors(None, 0, 0, None) == -1
    assert lib.igasf_device_status(None, 0) == -1
    assert lib.igasf_set_test_fault(None, 0, 100000) == -1
    assert lib.igasf_cg_solve(None, 1, None, None, 1e-10, 1e-4, 10, None, None) == -1
    assert lib.igasf_batch_create(0, None, 1, 1, None) == -1
    assert lib.igasf_batch_apply(None, None, None, None) == -1
    assert lib.igasf_batch_info(None, None, None, None, None) == -1
    assert lib.igasf_batch_destroy(None) == 0
    assert lib.igasf_autotune(3, None, None, None, None, None, 1, 1, 1, None, None, None) == -1


def test_binding_raises_without_library(tmp_path):
    import importlib
    mod = importlib.reload(G)
    try:
        mod._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            mod.load_library(str(tmp_path / "missing.so"))
    finally:
        importlib.reload(G)


def test_rejects_patch_beyond_int32_dofs_before_reading_ctrl(lib):
    """1302^3 dofs exceed the 32-bit dof index: refused on the host, before the
    control points are read or any device memory is touched."""
    p = 3
    t = I.open_uniform_knots(p, 1300)
    ctrl = np.zeros(3)                      # far too short: must not be read
    rc, _ = _setup(lib, 3, [p] * 3, [t, t, t], ctrl)
    assert rc == -4
    assert b"too large" in lib.igasf_last_error_message()


def test_list_kernels_enumerates_selectable_candidates(lib):
    """Host-only listing: every (d, p, precision) has a default, each (tile,
    variant) appears once per list, unused directions read 1, the on-the-fly
    list exists for FP32 in 3D only, and bad arguments are rejected."""
    for d in (2, 3):
        for p in range(2, G.MAX_ORDER + 1):
            for prec in (G.FP64, G.FP32, G.BF16):
                cands = G.list_kernels(d, p, prec)
                assert len(cands) >= 1
                keys = [(tuple(t), v) for t, v in cands]
                assert len(set(keys)) == len(keys)
                for t, v in cands:
                    assert all(s >= 1 for s in t[:d]) and all(s == 1 for s in t[d:])
                    assert v in (G.KERNEL_REGISTERS, G.KERNEL_RING)
                if prec == G.FP64:
                    assert all(v == G.KERNEL_REGISTERS for _, v in cands)
            for prec in (G.TF32, G.BF16_MMA):       # tensor-core kernels: 3D only
                cands = G.list_kernels(d, p, prec)
                assert (len(cands) >= 1) == (d == 3)
                assert all(v == G.KERNEL_MMA for _, v in cands)
                assert len({tuple(t) for t, _ in cands}) == len(cands)
            geo = G.list_kernels(d, p, G.FP32, G.GEOMETRY_ON_THE_FLY)
            assert (len(geo) >= 1) == (d == 3)
            assert all(v == G.KERNEL_ON_THE_FLY for _, v in geo)
            assert G.list_kernels(d, p, G.FP64, G.GEOMETRY_ON_THE_FLY) == []
    # the documented default of the benchmark workload's order
    assert G.list_kernels(3, 4, G.FP32)[0] == ([4, 4, 4], G.KERNEL_REGISTERS)
    n = lib.igasf_list_kernels(3, 4, G.FP32, 0, None, None, 0)
    assert n == len(G.list_kernels(3, 4, G.FP32))
    for args in [(4, 3, 0, 0), (3, 1, 0, 0), (3, G.MAX_ORDER + 1, 0, 0), (3, 4, 7, 0), (3, 4, 1, 5)]:
        with pytest.raises(G.IgasfError):
            G.list_kernels(*args)
    assert lib.igasf_list_kernels(3, 4, G.FP32, 0, None, None, -1) == G.ERR_INVALID_ARG
