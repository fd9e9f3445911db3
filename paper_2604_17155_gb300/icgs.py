"""Thin Python binding of libicgs.so (include/icgs.h): argument marshalling only.

Every step of colorize / render / the adjoint runs in the library's CUDA kernels. PyTorch supplies
device memory (inputs, outputs and the workspace) and the current CUDA stream. There is no CPU
path: if libicgs.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libicgs.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "icgs.h")

OK, ERR_INVALID_ARG, ERR_WORKSPACE_TOO_SMALL, ERR_CUDA, ERR_CAPACITY, ERR_UNSUPPORTED, ERR_DEVICE_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
ERR_NONFINITE_INPUT = -7
F32, BF16, F16 = 0, 1, 2
PLAIN, MIXED = 0, 1
GAUSSIAN_OK, GAUSSIAN_UNSEEN, GAUSSIAN_FP64 = 0, 1, 2


def solve_record_floats(sh_degree):
    """Floats per Gaussian of the solve record colorize() returns (the `chol` tensor): the
    row-packed lower Cholesky factor of A = G + w Lambda, then A itself in float-float (hi parts,
    then lo parts), each B (B + 1) / 2 floats with B = (L + 1)^2."""
    B = (sh_degree + 1) ** 2
    return 3 * (B * (B + 1) // 2)


class IcgsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"icgs error {status}: {message}")
        self.status = status


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity", ctypes.c_void_p)]


class _Cameras(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("near_z", ctypes.c_float), ("intrinsics", ctypes.c_void_p), ("world_to_cam", ctypes.c_void_p)]


class _Targets(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("channels", ctypes.c_int32), ("data", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("sh_degree", ctypes.c_int32), ("lambda_", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("cond_tau", ctypes.c_float), ("refold_tau", ctypes.c_float), ("cam_batch", ctypes.c_int32),
                ("instance_capacity", ctypes.c_int64)]


_lib = None


def exported_names():
    """Function names declared in include/icgs.h."""
    txt = open(HEADER_PATH).read()
    return re.findall(r"ICGS_API\s+[\w\s\*]*?\b(icgs_\w+)\s*\(", txt)


def load(path: str = LIB_PATH):
    """Loads libicgs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libicgs.so not found at {path}; build it with "
                           "`python -m paper_2604_17155_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, S = ctypes.c_void_p, ctypes.c_size_t
    lib.icgs_workspace_size.argtypes = [P, P, P, P]
    lib.icgs_workspace_size.restype = S
    lib.icgs_colorize.argtypes = [P, P, P, P, P, S, P, P, P, P]
    lib.icgs_colorize.restype = ctypes.c_int
    lib.icgs_colorize_backward.argtypes = [P, P, P, P, P, P, P, P, S, P, P, P]
    lib.icgs_colorize_backward.restype = ctypes.c_int
    lib.icgs_render_workspace_size.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    lib.icgs_render_workspace_size.restype = S
    lib.icgs_render.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64, P, S, P, P]
    lib.icgs_render.restype = ctypes.c_int
    lib.icgs_last_error.argtypes = []
    lib.icgs_last_error.restype = ctypes.c_char_p
    lib.icgs_last_required_instances.argtypes = []
    lib.icgs_last_required_instances.restype = ctypes.c_int64
    lib.icgs_last_stats.argtypes = [P]
    lib.icgs_last_stats.restype = None
    lib.icgs_colorize_noalloc.argtypes = [P, P, P, P, P, P, P, P]
    lib.icgs_colorize_noalloc.restype = ctypes.c_int
    lib.icgs_noalloc_scratch_bytes.argtypes = []
    lib.icgs_noalloc_scratch_bytes.restype = S
    lib.icgs_refine_workspace_size.argtypes = [P, P, P, P]
    lib.icgs_refine_workspace_size.restype = S
    lib.icgs_colorize_refine.argtypes = [P, P, P, P, ctypes.c_int32, P, P, S, P, P]
    lib.icgs_colorize_refine.restype = ctypes.c_int
    lib.icgs_colorize_host_workspace_size.argtypes = [P, P, P, P]
    lib.icgs_colorize_host_workspace_size.restype = S
    lib.icgs_colorize_host.argtypes = [P, P, P, P, P, S, P, P, P, P]
    lib.icgs_colorize_host.restype = ctypes.c_int
    lib.icgs_normal_size.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.icgs_normal_size.restype = ctypes.c_int64
    lib.icgs_accumulate.argtypes = [P, P, P, P, P, S, P, P]
    lib.icgs_accumulate.restype = ctypes.c_int
    lib.icgs_solve_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P]
    lib.icgs_solve_workspace_size.restype = S
    lib.icgs_solve.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P, P, S, P, P, P, P]
    lib.icgs_solve.restype = ctypes.c_int
    lib.icgs_selftest_tc.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, P, P]
    lib.icgs_selftest_tc.restype = ctypes.c_int
    lib.icgs_selftest_tc_rows.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P]
    lib.icgs_selftest_tc_rows.restype = ctypes.c_int
    lib.icgs_colorize_async.argtypes = [P, P, P, P, P, S, P, P, P, P]
    lib.icgs_colorize_async.restype = ctypes.c_int
    lib.icgs_colorize_backward_async.argtypes = [P, P, P, P, P, P, P, P, S, P, P, P]
    lib.icgs_colorize_backward_async.restype = ctypes.c_int
    lib.icgs_colorize_refine_async.argtypes = [P, P, P, P, ctypes.c_int32, P, P, S, P, P]
    lib.icgs_colorize_refine_async.restype = ctypes.c_int
    lib.icgs_render_async.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64, P, S, P, P]
    lib.icgs_render_async.restype = ctypes.c_int
    lib.icgs_async_status.argtypes = [P, P]
    lib.icgs_async_status.restype = ctypes.c_int
    lib.icgs_sets_workspace_size.argtypes = [P, P, ctypes.c_int32, P, P]
    lib.icgs_sets_workspace_size.restype = S
    lib.icgs_colorize_sets.argtypes = [P, P, ctypes.c_int32, P, P, P, S, P, P, P, ctypes.c_float, P, P]
    lib.icgs_colorize_sets.restype = ctypes.c_int
    lib.icgs_debug_tc_wait.argtypes = [ctypes.c_int64, ctypes.c_int32]
    lib.icgs_debug_tc_wait.restype = None
    lib.icgs_sort_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64]
    lib.icgs_sort_workspace_size.restype = S
    lib.icgs_sort_tile_lists.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, P, S, P]
    lib.icgs_sort_tile_lists.restype = ctypes.c_int
    lib.icgs_set_stage_timing.argtypes = [ctypes.c_int]
    lib.icgs_set_stage_timing.restype = None
    lib.icgs_last_stage_ms.argtypes = [P, ctypes.c_int]
    lib.icgs_last_stage_ms.restype = ctypes.c_int
    lib.icgs_stage_name.argtypes = [ctypes.c_int]
    lib.icgs_stage_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != OK:
        raise IcgsError(status, load().icgs_last_error().decode(errors="replace"))


def last_stats():
    out = (ctypes.c_int64 * 5)()
    load().icgs_last_stats(out)
    return {"instances": int(out[0]), "contrib_pairs": int(out[1]), "fp64": int(out[2]), "launches": int(out[3]),
            "refold": int(out[4])}


def set_stage_timing(enable: bool):
    """Records CUDA events at stage boundaries of every call on this thread (benchmarks)."""
    load().icgs_set_stage_timing(1 if enable else 0)


def last_stage_ms():
    """{stage name: milliseconds} of the last call on this thread (needs set_stage_timing(True))."""
    lib = load()
    out = (ctypes.c_double * 16)()
    n = lib.icgs_last_stage_ms(out, 16)
    return {lib.icgs_stage_name(i).decode(): float(out[i]) for i in range(n)}


# ------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _dev_f32(x, device):
    torch = _torch()
    t = torch.as_tensor(x, device=device)
    if t.dtype != torch.float32:
        t = t.float()
    return t.contiguous()


class Scene:
    """Device-resident scene: means [n,3], scales [n,3], quats [n,4] (w,x,y,z), opacity [n]."""

    def __init__(self, means, scales, quats, opacity, device="cuda"):
        self.means = _dev_f32(means, device)
        self.scales = _dev_f32(scales, device)
        self.quats = _dev_f32(quats, device)
        self.opacity = _dev_f32(opacity, device)

    @classmethod
    def from_workload(cls, scene, device="cuda"):
        return cls(scene.means, scene.scales, scene.quats, scene.opacity, device)

    @property
    def n(self):
        return int(self.means.shape[0])

    def _struct(self, opacity=None):
        o = self.opacity if opacity is None else opacity
        return _Scene(self.n, self.means.data_ptr(), self.scales.data_ptr(), self.quats.data_ptr(), o.data_ptr())


class Cameras:
    """Host-side camera rig: intrinsics [C,4] (fx, fy, cx, cy) and world_to_cam [C,12]."""

    def __init__(self, width, height, intrinsics, world_to_cam, near_z=0.2):
        self.width, self.height = int(width), int(height)
        self.intrinsics = np.ascontiguousarray(intrinsics, np.float32).reshape(-1, 4)
        self.world_to_cam = np.ascontiguousarray(world_to_cam, np.float32).reshape(-1, 12)
        self.near_z = float(near_z)

    @classmethod
    def from_workload(cls, cams):
        intr = np.stack([cams.fx, cams.fy, cams.cx, cams.cy], 1)
        return cls(cams.width, cams.height, intr, cams.world_to_cam.reshape(-1, 12), cams.near_z)

    @property
    def n(self):
        return int(self.intrinsics.shape[0])

    def subset(self, idx):
        """The cameras at the given indices, in that order."""
        idx = np.asarray(idx, np.int64)
        return Cameras(self.width, self.height, self.intrinsics[idx], self.world_to_cam[idx], self.near_z)

    def _struct(self):
        return _Cameras(self.n, self.width, self.height, self.near_z,
                        self.intrinsics.ctypes.data, self.world_to_cam.ctypes.data)


def _targets_struct(targets):
    torch = _torch()
    dt = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}.get(targets.dtype)
    if dt is None:
        raise TypeError(f"targets dtype {targets.dtype} is not float32, bfloat16 or float16")
    if not targets.is_cuda or not targets.is_contiguous() or targets.dim() != 4:
        raise ValueError("targets must be a contiguous CUDA tensor [n_cams,H,W,K]")
    return _Targets(dt, int(targets.shape[-1]), targets.data_ptr())


def _options(sh_degree, lam, precision, cond_tau, cam_batch, capacity, refold_tau=0.0):
    lam_arr = None if lam is None else np.ascontiguousarray(lam, np.float32)
    o = _Options(int(sh_degree), None if lam_arr is None else lam_arr.ctypes.data,
                 {"plain": PLAIN, "mixed": MIXED}.get(precision, precision), float(cond_tau), float(refold_tau),
                 int(cam_batch), int(capacity))
    return o, lam_arr


def _stream_ptr(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class _WorkspaceCache:
    """One growing byte buffer per device; instance capacity learned from ICGS_ERR_CAPACITY."""

    def __init__(self):
        self.buf = {}
        self.capacity = {}

    def get(self, device, nbytes):
        torch = _torch()
        key = str(device)
        b = self.buf.get(key)
        if b is None or b.numel() < nbytes:
            self.buf[key] = None
            b = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
            self.buf[key] = b
        return b


_ws = _WorkspaceCache()


def _run_with_capacity(device, size_fn, call_fn, capacity):
    """Calls call_fn(ws_ptr, ws_bytes, capacity); on ICGS_ERR_CAPACITY retries once with the
    reported requirement (plus 10%)."""
    lib = load()
    cap = capacity if capacity > 0 else _ws.capacity.get(str(device), 0)
    for _ in range(2):
        nbytes = size_fn(cap)
        if nbytes == 0:
            _check(ERR_INVALID_ARG)
        ws = _ws.get(device, nbytes)
        st = call_fn(ws.data_ptr(), ws.numel(), cap)
        if st == ERR_CAPACITY:
            cap = int(lib.icgs_last_required_instances() * 1.1) + 1024
            _ws.capacity[str(device)] = cap
            continue
        _check(st)
        return
    _check(st)


# ------------------------------------------------------------------------------------------
# public calls
# ------------------------------------------------------------------------------------------
def colorize(scene: Scene, cams: Cameras, targets, sh_degree, lam=None, precision="mixed",
             cond_tau=0.0, cam_batch=0, instance_capacity=0, opacity=None, refold_tau=0.0):
    """Alg. 1 lines 1-6: per-Gaussian SH coefficients [n,(L+1)^2,K] (float32), status [n] (uint8)
    and the solve records [n, solve_record_floats(L)]: the Cholesky factor of A_i = G_i + w_i Lambda
    and A_i itself in float-float (what colorize_backward and colorize_refine take)."""
    torch = _torch()
    lib = load()
    dev = targets.device
    B = (sh_degree + 1) ** 2
    K = int(targets.shape[-1])
    coeffs = torch.empty((scene.n, B, K), dtype=torch.float32, device=dev)
    status = torch.empty((scene.n,), dtype=torch.uint8, device=dev)
    chol = torch.empty((scene.n, solve_record_floats(sh_degree)), dtype=torch.float32, device=dev)
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _targets_struct(targets)

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_colorize(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                 ctypes.c_void_p(ptr), nbytes, ctypes.c_void_p(coeffs.data_ptr()),
                                 ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(chol.data_ptr()),
                                 _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return coeffs, status, chol


def colorize_sets(scene: Scene, cams: Cameras, target_sets, sh_degree, lam=None, precision="mixed", cond_tau=0.0,
                  cam_batch=0, instance_capacity=0, refold_tau=0.0, threshold=None):
    """icgs_colorize_sets: several target stacks of the same cameras (a list of CUDA tensors
    [n_cams,H,W,K_s], each float32, bfloat16 or float16) colorized on one geometry with one shared
    factorisation. Returns coefficients [n,(L+1)^2,sum K_s] (channels in set order), status [n],
    solve records, and, with threshold given (sh_degree 0 only), keep [n, sum K_s] uint8: 1 where
    the Gaussian's colour reaches the threshold (Sec. 5 uses 0.6)."""
    torch = _torch()
    lib = load()
    if not target_sets:
        raise ValueError("at least one target set is required")
    dev = target_sets[0].device
    B = (sh_degree + 1) ** 2
    structs = [_targets_struct(t) for t in target_sets]
    arr = (_Targets * len(structs))(*structs)
    K = sum(int(t.shape[-1]) for t in target_sets)
    coeffs = torch.empty((scene.n, B, K), dtype=torch.float32, device=dev)
    status = torch.empty((scene.n,), dtype=torch.uint8, device=dev)
    chol = torch.empty((scene.n, solve_record_floats(sh_degree)), dtype=torch.float32, device=dev)
    keep = torch.empty((scene.n, K), dtype=torch.uint8, device=dev) if threshold is not None else None
    sc = scene._struct()
    cm = cams._struct()

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_sets_workspace_size(ctypes.byref(sc), ctypes.byref(cm), len(structs), arr, ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_colorize_sets(ctypes.byref(sc), ctypes.byref(cm), len(structs), arr, ctypes.byref(o),
                                      ctypes.c_void_p(ptr), nbytes, ctypes.c_void_p(coeffs.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(chol.data_ptr()),
                                      float(threshold if threshold is not None else 0.0),
                                      ctypes.c_void_p(keep.data_ptr() if keep is not None else 0), _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return coeffs, status, chol, keep


class AsyncColorize:
    """A colorize enqueued by colorize_async(): owns its workspace and outputs until wait()."""

    def __init__(self, workspace, stream, outputs):
        self.workspace = workspace
        self.stream = stream
        self.outputs = outputs

    def wait(self):
        """Joins the call (synchronises its stream) and returns (coeffs, status, chol); raises
        IcgsError with the device outcome (ERR_CAPACITY, ERR_NONFINITE_INPUT, ...) if it failed."""
        _check(load().icgs_async_status(ctypes.c_void_p(self.workspace.data_ptr()), self.stream))
        return self.outputs


def colorize_async(scene: Scene, cams: Cameras, targets, sh_degree, lam=None, precision="mixed", cond_tau=0.0,
                   cam_batch=0, instance_capacity=0, opacity=None, refold_tau=0.0):
    """colorize() through icgs_colorize_async on the current stream: returns at once, before the
    work has run, with a handle whose wait() joins it. The call has its own workspace, so several
    may run concurrently on different streams. A capacity overflow surfaces in wait() (no retry)."""
    torch = _torch()
    lib = load()
    dev = targets.device
    B = (sh_degree + 1) ** 2
    K = int(targets.shape[-1])
    coeffs = torch.empty((scene.n, B, K), dtype=torch.float32, device=dev)
    status = torch.empty((scene.n,), dtype=torch.uint8, device=dev)
    chol = torch.empty((scene.n, solve_record_floats(sh_degree)), dtype=torch.float32, device=dev)
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _targets_struct(targets)
    o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, instance_capacity, refold_tau)
    nbytes = lib.icgs_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o))
    if nbytes == 0:
        _check(ERR_INVALID_ARG)
    ws = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
    stream = _stream_ptr(dev)
    _check(lib.icgs_colorize_async(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(coeffs.data_ptr()),
                                   ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(chol.data_ptr()), stream))
    return AsyncColorize(ws, stream, (coeffs, status, chol))


def colorize_host(scene: Scene, cams: Cameras, targets, sh_degree, lam=None, precision="mixed",
                  cond_tau=0.0, cam_batch=0, instance_capacity=0, opacity=None, refold_tau=0.0,
                  coeffs_out=None, status_out=None):
    """colorize() with the targets in host memory and the results returned in host memory
    (icgs_colorize_host): targets is a contiguous CPU tensor [n_cams,H,W,K] (float32, bfloat16 or
    float16; page-locked for copies that overlap the compute). Returns CPU coefficients
    [n,(L+1)^2,K] float32 and status [n] uint8, written into coeffs_out / status_out when given."""
    torch = _torch()
    lib = load()
    dev = scene.means.device
    dt = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}.get(targets.dtype)
    if dt is None:
        raise TypeError(f"targets dtype {targets.dtype} is not float32, bfloat16 or float16")
    if targets.is_cuda or not targets.is_contiguous() or targets.dim() != 4:
        raise ValueError("targets must be a contiguous CPU tensor [n_cams,H,W,K]")
    B = (sh_degree + 1) ** 2
    K = int(targets.shape[-1])
    pin = torch.cuda.is_available()
    coeffs = coeffs_out if coeffs_out is not None else torch.empty((scene.n, B, K), dtype=torch.float32,
                                                                   pin_memory=pin)
    status = status_out if status_out is not None else torch.empty((scene.n,), dtype=torch.uint8, pin_memory=pin)
    if coeffs.shape != (scene.n, B, K) or coeffs.dtype != torch.float32 or coeffs.is_cuda or not coeffs.is_contiguous():
        raise ValueError("coeffs_out must be a contiguous CPU float32 tensor [n,(L+1)^2,K]")
    if status.shape != (scene.n,) or status.dtype != torch.uint8 or status.is_cuda:
        raise ValueError("status_out must be a CPU uint8 tensor [n]")
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _Targets(dt, K, targets.data_ptr())

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_colorize_host_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg),
                                                     ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, cap, refold_tau)
        return lib.icgs_colorize_host(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                      ctypes.c_void_p(ptr), nbytes, ctypes.c_void_p(coeffs.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()), None, _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return coeffs, status


def normal_size(sh_degree, channels):
    """Doubles per Gaussian of the packed normal equations (icgs_normal_size): the upper triangle
    of G row by row, then b [B,K], then w."""
    B = (sh_degree + 1) ** 2
    return B * (B + 1) // 2 + B * channels + 1


def accumulate(scene: Scene, cams: Cameras, targets, sh_degree, lam=None, precision="mixed", cam_batch=0,
               instance_capacity=0, opacity=None):
    """icgs_accumulate: the normal equations of these cameras (Eq. 12-14) as packed float64 device
    sums [n, normal_size(L, K)]. Sums over disjoint camera subsets add up to the sums over their
    union."""
    torch = _torch()
    lib = load()
    dev = targets.device
    K = int(targets.shape[-1])
    sums = torch.empty((scene.n, normal_size(sh_degree, K)), dtype=torch.float64, device=dev)
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _targets_struct(targets)

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_accumulate(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                   ctypes.c_void_p(ptr), nbytes, ctypes.c_void_p(sums.data_ptr()), _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return sums


def solve(sums, sh_degree, lam=None, precision="mixed", cond_tau=0.0):
    """icgs_solve: coefficients [n,B,K] float32, status [n] uint8 and solve records from packed
    float64 device sums [n, normal_size(L, K)] (as accumulate() returns them, their sum over camera
    subsets, or any contiguous range of their rows)."""
    torch = _torch()
    lib = load()
    dev = sums.device
    n = int(sums.shape[0])
    B = (sh_degree + 1) ** 2
    P = B * (B + 1) // 2
    K = (int(sums.shape[1]) - P - 1) // B
    if (sums.dtype != torch.float64 or not sums.is_cuda or not sums.is_contiguous() or sums.dim() != 2
            or K < 1 or normal_size(sh_degree, K) != sums.shape[1]):
        raise ValueError("expected contiguous float64 CUDA sums [n, normal_size(L, K)]")
    coeffs = torch.empty((n, B, K), dtype=torch.float32, device=dev)
    status = torch.empty((n,), dtype=torch.uint8, device=dev)
    chol = torch.empty((n, solve_record_floats(sh_degree)), dtype=torch.float32, device=dev)
    o, _keep = _options(sh_degree, lam, precision, cond_tau, 0, 0)
    nbytes = lib.icgs_solve_workspace_size(n, sh_degree, K, ctypes.byref(o))
    if nbytes == 0:
        _check(ERR_INVALID_ARG)
    ws = _ws.get(dev, nbytes)
    _check(lib.icgs_solve(n, sh_degree, K, ctypes.c_void_p(sums.data_ptr()), ctypes.byref(o),
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(coeffs.data_ptr()),
                          ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(chol.data_ptr()), _stream_ptr(dev)))
    return coeffs, status, chol


def shard_cameras(n_cams, rank, world):
    """The camera indices of one rank in a round-robin partition of n_cams cameras."""
    return np.arange(rank, n_cams, world)


def shard_gaussians(n, rank, world):
    """The contiguous Gaussian range [lo, hi) a rank solves: ranges of ceil(n / world) rows."""
    chunk = -(-n // world)
    return min(n, rank * chunk), min(n, (rank + 1) * chunk)


def colorize_sharded(scene, cams, targets, sh_degree, rank, world, group=None, lam=None, precision="mixed",
                     gather=True, accumulate_fn=None, solve_fn=None):
    """Camera-sharded colorize. This rank accumulates the packed normal equations of its round-robin
    share of the cameras; one torch.distributed reduce-scatter (sum; NCCL for GPU tensors) leaves it
    the totals of its contiguous Gaussian range (shard_gaussians); it solves that range; with
    gather=True one all-gather replicates the coefficients. targets holds all cameras' images;
    only this rank's slice is read.

    accumulate_fn(scene, cams_subset, targets_subset, sh_degree, lam, precision) -> sums [n, R]
    float64 and solve_fn(sums_range, sh_degree, lam, precision) -> (coeffs, status, chol) default to
    accumulate() and solve(). Returns dict(coeffs=[n,B,K] with gather else the range's rows,
    status and chol of the range, range=(lo, hi))."""
    torch = _torch()
    import torch.distributed as dist
    accumulate_fn = accumulate_fn or (lambda sc, cm, t, L, lm, pr: accumulate(sc, cm, t, L, lam=lm, precision=pr))
    solve_fn = solve_fn or (lambda s, L, lm, pr: solve(s, L, lam=lm, precision=pr))
    mine = shard_cameras(cams.n, rank, world)
    idx = torch.as_tensor(mine, device=targets.device)
    sums = accumulate_fn(scene, cams.subset(mine), targets.index_select(0, idx).contiguous(), sh_degree, lam,
                         precision)
    n, R = int(sums.shape[0]), int(sums.shape[1])
    lo, hi = shard_gaussians(n, rank, world)
    if world > 1:
        chunk = -(-n // world)
        full = sums
        if chunk * world != n:
            full = torch.zeros((chunk * world, R), dtype=sums.dtype, device=sums.device)
            full[:n] = sums
        part = torch.empty((chunk, R), dtype=sums.dtype, device=sums.device)
        dist.reduce_scatter_tensor(part, full, op=dist.ReduceOp.SUM, group=group)
        sums = part[:hi - lo].contiguous()
    coeffs, status, chol = solve_fn(sums, sh_degree, lam, precision)
    out = dict(coeffs=coeffs, status=status, chol=chol, range=(lo, hi))
    if gather and world > 1:
        chunk = -(-n // world)
        mine_c = torch.zeros((chunk,) + tuple(coeffs.shape[1:]), dtype=coeffs.dtype, device=coeffs.device)
        mine_c[:hi - lo] = coeffs
        allc = torch.empty((chunk * world,) + tuple(coeffs.shape[1:]), dtype=coeffs.dtype, device=coeffs.device)
        dist.all_gather_into_tensor(allc, mine_c, group=group)
        out["coeffs"] = allc[:n]
    return out


def colorize_noalloc(scene: Scene, cams: Cameras, targets, sh_degree, lam=None, precision="mixed",
                     cond_tau=0.0, cam_batch=0, instance_capacity=0, opacity=None, refold_tau=0.0):
    """Like colorize(), but the library works in its own built-in device scratch instead of a
    workspace, for callers that cannot allocate device memory (see icgs_colorize_noalloc in
    include/icgs.h). The outputs are still the caller's tensors; problems larger than the scratch
    raise IcgsError with ERR_WORKSPACE_TOO_SMALL or ERR_CAPACITY."""
    torch = _torch()
    lib = load()
    dev = targets.device
    B = (sh_degree + 1) ** 2
    K = int(targets.shape[-1])
    coeffs = torch.empty((scene.n, B, K), dtype=torch.float32, device=dev)
    status = torch.empty((scene.n,), dtype=torch.uint8, device=dev)
    chol = torch.empty((scene.n, solve_record_floats(sh_degree)), dtype=torch.float32, device=dev)
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _targets_struct(targets)
    o, _keep = _options(sh_degree, lam, precision, cond_tau, cam_batch, instance_capacity, refold_tau)
    _check(lib.icgs_colorize_noalloc(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                     ctypes.c_void_p(coeffs.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(chol.data_ptr()), _stream_ptr(dev)))
    return coeffs, status, chol


def colorize_refine(scene: Scene, cams: Cameras, targets, sh_degree, coeffs, chol, n_steps, lam=None,
                    precision="mixed", cam_batch=0, instance_capacity=0):
    """Alg. 1 lines 7-10: n_steps refinement steps of coeffs (updated in place and returned), with
    the Cholesky factors colorize() returned."""
    lib = load()
    dev = targets.device
    if not coeffs.is_contiguous() or coeffs.dtype != _torch().float32:
        raise ValueError("coeffs must be a contiguous float32 tensor (it is updated in place)")
    sc = scene._struct()
    cm = cams._struct()
    tg = _targets_struct(targets)
    chol = chol.contiguous()

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_refine_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_colorize_refine(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o),
                                        int(n_steps), ctypes.c_void_p(chol.data_ptr()), ctypes.c_void_p(ptr), nbytes,
                                        ctypes.c_void_p(coeffs.data_ptr()), _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return coeffs


def selftest_tc(A, B, bf16=True, lanes=False):
    """Diagnostic: A [M,256] @ B [N,256]^T (M = 64 or 128, N = 32 or 80) through the tensor-core
    path of the 16-bit accumulate walk; A and B are 16-bit CUDA tensors. Returns float32 [M, N],
    and with lanes=True also the raw contents of the 128 TMEM lanes, float32 [128, N]."""
    torch = _torch()
    lib = load()
    A = A.contiguous()
    B = B.contiguous()
    M, N = int(A.shape[0]), int(B.shape[0])
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    DL = torch.full((128, N), float("nan"), dtype=torch.float32, device=A.device) if lanes else None
    ws = _ws.get(A.device, 256)
    _check(lib.icgs_selftest_tc_rows(ctypes.c_void_p(A.data_ptr()), M, ctypes.c_void_p(B.data_ptr()), N,
                                     1 if bf16 else 0, ctypes.c_void_p(D.data_ptr()),
                                     ctypes.c_void_p(DL.data_ptr() if lanes else 0), ctypes.c_void_p(ws.data_ptr()),
                                     _stream_ptr(A.device)))
    return (D, DL) if lanes else D


def sort_tile_lists(tile_off, keys):
    """Diagnostic: the library's depth sort of tile lists, in place. tile_off: int32 CUDA tensor
    [ntiles + 1] (non-decreasing from 0); keys: int64 CUDA tensor, each (float32 depth bits << 32)
    | Gaussian index."""
    lib = load()
    if tile_off.dtype != _torch().int32 or keys.dtype != _torch().int64:
        raise ValueError("tile_off must be int32 and keys int64")
    if not (tile_off.is_contiguous() and keys.is_contiguous()):
        raise ValueError("tile_off and keys must be contiguous")
    ntiles, nkeys = int(tile_off.numel()) - 1, int(keys.numel())
    size = lib.icgs_sort_workspace_size(ntiles, nkeys)
    ws = _ws.get(keys.device, size)
    _check(lib.icgs_sort_tile_lists(ctypes.c_void_p(tile_off.data_ptr()), ctypes.c_void_p(keys.data_ptr()), ntiles,
                                    nkeys, ctypes.c_void_p(ws.data_ptr()), size,
                                    _stream_ptr(keys.device)))
    return keys


def colorize_backward(scene: Scene, cams: Cameras, targets, sh_degree, coeffs, chol, grad_coeffs, lam=None,
                      precision="mixed", cam_batch=0, instance_capacity=0, want_targets=True,
                      want_opacity=True, opacity=None):
    """dL/d(targets) [n_cams,H,W,K] and dL/d(opacity) [n] for a given dL/dc."""
    torch = _torch()
    lib = load()
    dev = targets.device
    gt = torch.empty(targets.shape, dtype=torch.float32, device=dev) if want_targets else None
    go = torch.empty((scene.n,), dtype=torch.float32, device=dev) if want_opacity else None
    sc = scene._struct(opacity)
    cm = cams._struct()
    tg = _targets_struct(targets)
    grad_coeffs = grad_coeffs.contiguous().float()
    coeffs = coeffs.contiguous()
    chol = chol.contiguous()

    def size_fn(cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_workspace_size(ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o))

    def call_fn(ptr, nbytes, cap):
        o, _keep = _options(sh_degree, lam, precision, 0.0, cam_batch, cap)
        return lib.icgs_colorize_backward(
            ctypes.byref(sc), ctypes.byref(cm), ctypes.byref(tg), ctypes.byref(o), ctypes.c_void_p(coeffs.data_ptr()),
            ctypes.c_void_p(chol.data_ptr()), ctypes.c_void_p(grad_coeffs.data_ptr()), ctypes.c_void_p(ptr), nbytes,
            ctypes.c_void_p(gt.data_ptr() if gt is not None else 0), ctypes.c_void_p(go.data_ptr() if go is not None else 0),
            _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return gt, go


def render(scene: Scene, cams: Cameras, coeffs, sh_degree, instance_capacity=0):
    """Eq. 1-3: images [n_cams,H,W,K] float32 from coefficients [n,(L+1)^2,K]."""
    torch = _torch()
    lib = load()
    coeffs = coeffs.contiguous().float()
    dev = coeffs.device
    K = int(coeffs.shape[-1])
    images = torch.empty((cams.n, cams.height, cams.width, K), dtype=torch.float32, device=dev)
    sc = scene._struct()
    cm = cams._struct()

    def size_fn(cap):
        return lib.icgs_render_workspace_size(ctypes.byref(sc), ctypes.byref(cm), int(sh_degree), K, int(cap))

    def call_fn(ptr, nbytes, cap):
        return lib.icgs_render(ctypes.byref(sc), ctypes.byref(cm), int(sh_degree), K, ctypes.c_void_p(coeffs.data_ptr()),
                               int(cap), ctypes.c_void_p(ptr), nbytes, ctypes.c_void_p(images.data_ptr()),
                               _stream_ptr(dev))

    _run_with_capacity(dev, size_fn, call_fn, instance_capacity)
    return images


def _make_autograd():
    torch = _torch()

    class ColorizeFn(torch.autograd.Function):
        """c = colorize(targets, opacity) with the hand-written adjoint in backward()."""

        @staticmethod
        def forward(ctx, targets, opacity, scene, cams, sh_degree, lam, precision):
            coeffs, status, chol = colorize(scene, cams, targets, sh_degree, lam=lam, precision=precision,
                                            opacity=opacity.detach().contiguous().float())
            ctx.save_for_backward(targets, opacity, coeffs, chol)
            ctx.cfg = (scene, cams, sh_degree, lam, precision)
            ctx.mark_non_differentiable(status)
            return coeffs, status

        @staticmethod
        def backward(ctx, grad_coeffs, _grad_status):
            targets, opacity, coeffs, chol = ctx.saved_tensors
            scene, cams, sh_degree, lam, precision = ctx.cfg
            gt, go = colorize_backward(scene, cams, targets, sh_degree, coeffs, chol, grad_coeffs, lam=lam,
                                       precision=precision, want_targets=ctx.needs_input_grad[0],
                                       want_opacity=ctx.needs_input_grad[1],
                                       opacity=opacity.detach().contiguous().float())
            if gt is not None:
                gt = gt.to(targets.dtype)
            return gt, go, None, None, None, None, None

    return ColorizeFn


_ColorizeFn = None


def colorize_differentiable(scene: Scene, cams: Cameras, targets, opacity, sh_degree, lam=None, precision="mixed"):
    """Autograd entry: returns coefficients differentiable with respect to targets and opacity."""
    global _ColorizeFn
    if _ColorizeFn is None:
        _ColorizeFn = _make_autograd()
    coeffs, _status = _ColorizeFn.apply(targets, opacity, scene, cams, sh_degree, lam, precision)
    return coeffs
