"""The C ABI library builds for sm_103a, loads, exports every function include/icgs.h declares,
and rejects bad arguments on the host before any device work. No GPU is needed."""
import ctypes

import numpy as np
import pytest

from paper_2604_17155_gb300 import build as B
from paper_2604_17155_gb300 import icgs


@pytest.fixture(scope="module")
def lib():
    B.build()
    return icgs.load()


def test_header_declares_the_calls():
    names = icgs.exported_names()
    for want in ["icgs_workspace_size", "icgs_colorize", "icgs_colorize_backward", "icgs_render_workspace_size",
                 "icgs_render", "icgs_last_error", "icgs_last_required_instances", "icgs_last_stats",
                 "icgs_colorize_noalloc", "icgs_noalloc_scratch_bytes", "icgs_selftest_tc", "icgs_selftest_tc_rows",
                 "icgs_refine_workspace_size", "icgs_colorize_refine", "icgs_colorize_host_workspace_size",
                 "icgs_colorize_host", "icgs_accumulate", "icgs_solve_workspace_size", "icgs_solve",
                 "icgs_normal_size", "icgs_colorize_async", "icgs_colorize_backward_async",
                 "icgs_colorize_refine_async", "icgs_render_async", "icgs_async_status", "icgs_debug_tc_wait"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in icgs.exported_names():
        assert hasattr(lib, name), name


def _structs(n=10, n_cams=2, w=40, h=30, K=3, L=3):
    sc = icgs._Scene(n, 16, 16, 16, 16)  # fake non-null device pointers: never dereferenced on the host
    intr = np.tile(np.array([50.0, 50.0, w / 2, h / 2], np.float32), (n_cams, 1))
    w2c = np.tile(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 3], np.float32), (n_cams, 1))
    cm = icgs._Cameras(n_cams, w, h, 0.2, intr.ctypes.data, w2c.ctypes.data)
    tg = icgs._Targets(icgs.F32, K, 16)
    opt = icgs._Options(sh_degree=L, lambda_=None, precision=icgs.MIXED, cond_tau=0.0, refold_tau=0.0, cam_batch=0,
                        instance_capacity=0)
    return sc, cm, tg, opt, (intr, w2c)


def test_workspace_size_grows_with_capacity(lib):
    sc, cm, tg, opt, keep = _structs()
    sizes = []
    for cap in (1000, 2000, 100000):
        opt.instance_capacity = cap
        sizes.append(lib.icgs_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt)))
    assert sizes[0] > 0 and sizes[0] < sizes[1] < sizes[2]
    assert sizes[2] - sizes[1] >= 2 * 8 * (100000 - 2000) - 512  # keys + merge buffer (256-B aligned)


def test_host_workspace_adds_the_staging_regions(lib):
    """icgs_colorize_host's workspace is the colorize (accumulate) workspace followed by the staged
    targets, the coefficients and the status bytes (each 256-byte aligned): with 16-bit targets it
    is smaller by exactly the difference in staged target bytes."""
    n, n_cams, w, h, K, L = 10, 2, 40, 30, 3, 3
    sc, cm, tg, opt, keep = _structs(n, n_cams, w, h, K, L)
    a = lambda x: (x + 255) // 256 * 256
    host32 = lib.icgs_colorize_host_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg),
                                                   ctypes.byref(opt))
    tg16 = icgs._Targets(icgs.BF16, K, 16)
    host16 = lib.icgs_colorize_host_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg16),
                                                   ctypes.byref(opt))
    assert host32 - host16 == a(n_cams * h * w * K * 4) - a(n_cams * h * w * K * 2)
    assert host32 > a(n_cams * h * w * K * 4) + a(n * 16 * K * 4) + a(n)


def test_solve_workspace_and_arguments(lib):
    """icgs_solve's workspace holds the status block, lambda and the (hi, lo) normal equations;
    bad arguments are refused before any device work."""
    sc, cm, tg, opt, keep = _structs()
    a = lambda x: (x + 255) // 256 * 256
    n, K = 1000, 3
    mixed = lib.icgs_solve_workspace_size(n, 3, K, ctypes.byref(opt))
    assert mixed >= 2 * (a(n * 256 * 4) + a(n * 16 * K * 4) + a(n * 4))
    opt.precision = icgs.PLAIN
    plain = lib.icgs_solve_workspace_size(n, 3, K, ctypes.byref(opt))
    assert plain < mixed
    opt.precision = icgs.MIXED
    assert lib.icgs_solve_workspace_size(n, 4, K, ctypes.byref(opt)) == 0  # sh_degree 4
    assert lib.icgs_solve_workspace_size(n, 3, 0, ctypes.byref(opt)) == 0  # no channels
    st = lib.icgs_solve(n, 3, K, None, ctypes.byref(opt), None, 0, None, None, None, None)
    assert st == icgs.ERR_INVALID_ARG and "required" in lib.icgs_last_error().decode()
    st = lib.icgs_solve(n, 3, K, ctypes.c_void_p(16), ctypes.byref(opt), None, 0, ctypes.c_void_p(16), None, None,
                        None)
    assert st == icgs.ERR_WORKSPACE_TOO_SMALL


def test_packed_normal_size():
    """Packed normal equations per Gaussian: the upper triangle of the B x B Gram, B K right-hand
    side entries and w (B = (L+1)^2)."""
    lib = icgs.load()
    for L, K in ((0, 1), (0, 16), (1, 3), (3, 3), (3, 64)):
        B = (L + 1) ** 2
        assert lib.icgs_normal_size(L, K) == icgs.normal_size(L, K) == B * (B + 1) // 2 + B * K + 1
    assert lib.icgs_normal_size(4, 3) == 0 and lib.icgs_normal_size(0, 0) == 0


def test_bad_arguments_rejected_on_host(lib):
    sc, cm, tg, opt, keep = _structs()
    R = lambda *a: lib.icgs_colorize(*a)
    assert R(None, ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), None, 0, None, None, None, None) == icgs.ERR_INVALID_ARG
    assert "NULL" in lib.icgs_last_error().decode()
    opt.sh_degree = 4
    assert R(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), None, 0, ctypes.c_void_p(16), None, None, None) == icgs.ERR_INVALID_ARG
    assert "sh_degree" in lib.icgs_last_error().decode()
    opt.sh_degree = 3
    # workspace too small is reported before anything is enqueued
    assert R(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), ctypes.c_void_p(256), 1024,
             ctypes.c_void_p(16), None, None, None) == icgs.ERR_WORKSPACE_TOO_SMALL
    tg.dtype = 7
    assert R(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), None, 0, ctypes.c_void_p(16), None, None, None) == icgs.ERR_INVALID_ARG
    tg.dtype = icgs.F32
    bad = np.array([[0.0, 50.0, 20.0, 15.0]] * 2, np.float32)
    cm.intrinsics = bad.ctypes.data
    assert R(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), None, 0, ctypes.c_void_p(16), None, None, None) == icgs.ERR_INVALID_ARG
    assert "focal" in lib.icgs_last_error().decode()
    lam = np.full(16, -1.0, np.float32)
    cm.intrinsics = keep[0].ctypes.data
    opt.lambda_ = lam.ctypes.data
    assert R(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), ctypes.c_void_p(256), 1 << 40,
             ctypes.c_void_p(16), None, None, None) == icgs.ERR_INVALID_ARG
    assert "lambda" in lib.icgs_last_error().decode()


def test_backward_rejects_too_many_channels(lib):
    sc, cm, tg, opt, keep = _structs(K=65)
    st = lib.icgs_colorize_backward(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt),
                                    ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None, 0, None, None, None)
    assert st == icgs.ERR_UNSUPPORTED


def test_tc_selftest_rows_rejects_bad_shapes_on_host(lib):
    """icgs_selftest_tc_rows takes M = 64 or 128 rows and N = 32 or 80 columns; anything else is
    refused on the host with a message, before any device work."""
    p = ctypes.c_void_p(256)
    st = lib.icgs_selftest_tc_rows(p, 32, p, 32, 1, p, None, p, None)
    assert st == icgs.ERR_INVALID_ARG and "M = 32" in lib.icgs_last_error().decode()
    st = lib.icgs_selftest_tc_rows(p, 64, p, 48, 1, p, None, p, None)
    assert st == icgs.ERR_INVALID_ARG and "N = 48" in lib.icgs_last_error().decode()
    st = lib.icgs_selftest_tc_rows(None, 64, p, 32, 1, p, None, p, None)
    assert st == icgs.ERR_INVALID_ARG and "required" in lib.icgs_last_error().decode()


def test_async_calls_reject_bad_arguments_on_host(lib):
    """The enqueue-only calls check their arguments on the host exactly like the synchronous ones,
    and icgs_async_status refuses a missing or misaligned workspace, all before any device work."""
    sc, cm, tg, opt, keep = _structs()
    st = lib.icgs_colorize_async(None, ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), None, 0, None, None,
                                 None, None)
    assert st == icgs.ERR_INVALID_ARG and "NULL" in lib.icgs_last_error().decode()
    st = lib.icgs_colorize_async(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt),
                                 ctypes.c_void_p(256), 1024, ctypes.c_void_p(16), None, None, None)
    assert st == icgs.ERR_WORKSPACE_TOO_SMALL
    st = lib.icgs_render_async(ctypes.byref(sc), ctypes.byref(cm), 5, 3, ctypes.c_void_p(16), 0, None, 0,
                               ctypes.c_void_p(16), None)
    assert st == icgs.ERR_INVALID_ARG and "sh_degree" in lib.icgs_last_error().decode()
    st = lib.icgs_colorize_backward_async(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt),
                                          None, None, None, None, 0, None, None, None)
    assert st == icgs.ERR_INVALID_ARG and "required" in lib.icgs_last_error().decode()
    st = lib.icgs_colorize_refine_async(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(opt), -1,
                                        None, None, 0, None, None)
    assert st == icgs.ERR_INVALID_ARG and "n_steps" in lib.icgs_last_error().decode()
    assert lib.icgs_async_status(None, None) == icgs.ERR_INVALID_ARG
    assert lib.icgs_async_status(ctypes.c_void_p(4096 + 16), None) == icgs.ERR_INVALID_ARG
    assert "aligned" in lib.icgs_last_error().decode()
