"""icgs_colorize_noalloc -- colorize for callers that cannot allocate device memory.

Some callers have no way to hand the library a workspace: a plugin inside an application that
owns all device memory through its own allocator, or a latency-critical loop that must not
allocate after start-up. For them the library carries a fixed scratch array on every GPU that
loads it. This test calls that entry point through the C ABI twice in a row and compares each
result with the regular icgs_colorize on the same inputs, at the tolerance of the other GPU
tests; it also checks that a problem too large for the scratch is refused with a clear error.

The file is named so that pytest collects it last; it works alone in a fresh process too.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import TOL_FP32, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


def _compare(c_a, c_b, st):
    ok = to_np(st) == 0
    e = O.relative_errors(to_np(c_a), to_np(c_b).astype(np.float64))
    return float(e[ok].max()) if ok.any() else 0.0


def _scene(L):
    if L == 0:
        sc = W.make_scene("tiny", 1000)
        cams = W.make_cameras("tiny")
    else:
        sc = W.cluster_scene(3000, 91, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
        cams = W.hemisphere_cameras(16, 4.0, 100, 76, 50.0)
    t = O.render(sc, cams, W.sh_coefficients(sc.n, L, 3, seed=92), L).astype(np.float32)
    return sc, cams, t


@pytest.mark.parametrize("L", [0, 3])
def test_noalloc_matches_colorize_on_two_calls(icgs, L):
    sc, cams, t = _scene(L)
    gs = icgs.Scene.from_workload(sc, "cuda")
    gc = icgs.Cameras.from_workload(cams)
    tt = torch.tensor(t, device="cuda")
    c_ref, s_ref, ch_ref = icgs.colorize(gs, gc, tt, L)
    for call in range(2):
        c, s, ch = icgs.colorize_noalloc(gs, gc, tt, L)
        torch.cuda.synchronize()
        assert torch.equal(s, s_ref), f"call {call}: status differs"
        err = _compare(c, c_ref, s_ref)
        print(f"noalloc L={L} call {call}: max rel diff to icgs_colorize {err:.2e}")
        assert err <= TOL_FP32


def test_noalloc_fits_a_problem_only_colorize_itself_fits(icgs):
    """The scratch is sized against colorize's own workspace, not the larger colorize + adjoint one
    icgs_workspace_size reports: a problem whose combined workspace exceeds the scratch by the
    adjoint's regions still runs, and matches icgs_colorize."""
    import ctypes
    lib = icgs.load()
    cams = W.hemisphere_cameras(8, 4.0, 64, 48, 50.0)
    gc = icgs.Cameras.from_workload(cams)
    scratch = lib.icgs_noalloc_scratch_bytes()
    n_pick, both = None, 0
    tg = icgs._Targets(icgs.F32, 3, 16)
    o, _keep = icgs._options(3, None, "mixed", 0.0, 0, 1, 0.0)
    for n in range(2000, 200000, 1000):  # the smallest scene whose colorize + adjoint workspace overflows
        sz = icgs._Scene(n, 16, 16, 16, 16)  # sizes only: the pointers are never dereferenced
        both = lib.icgs_workspace_size(ctypes.byref(sz), ctypes.byref(gc._struct()), ctypes.byref(tg), ctypes.byref(o))
        if both > scratch:
            n_pick = n
            break
    assert n_pick is not None
    sc = W.cluster_scene(n_pick, 94, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    gs = icgs.Scene.from_workload(sc, "cuda")
    t = O.render(sc, cams, W.sh_coefficients(sc.n, 3, 3, seed=95), 3).astype(np.float32)
    tt = torch.tensor(t, device="cuda")
    c_ref, s_ref, _ = icgs.colorize(gs, gc, tt, 3)
    c, s, _ = icgs.colorize_noalloc(gs, gc, tt, 3)
    print(f"noalloc near the limit: {n_pick} Gaussians, colorize + adjoint workspace {both} > scratch {scratch}")
    assert torch.equal(s, s_ref)
    assert _compare(c, c_ref, s_ref) <= TOL_FP32


def test_noalloc_rejects_problems_beyond_its_scratch(icgs):
    # 2,000,000 Gaussians x 8 cameras need far more than the built-in scratch for their
    # per-(camera, Gaussian) records alone; the call must refuse before touching the GPU
    n = 2_000_000
    sc = W.uniform_scene(n, 93, box=1.0)
    cams = W.make_cameras("tiny")
    gs = icgs.Scene.from_workload(sc, "cuda")
    gc = icgs.Cameras.from_workload(cams)
    tt = torch.zeros((cams.n, cams.height, cams.width, 3), device="cuda")
    with pytest.raises(icgs.IcgsError) as ei:
        icgs.colorize_noalloc(gs, gc, tt, 0)
    assert ei.value.status == icgs.ERR_WORKSPACE_TOO_SMALL
    assert "built-in scratch" in str(ei.value)
    # the library still works afterwards
    sc2, cams2, t2 = _scene(0)
    c, s, _ = icgs.colorize_noalloc(icgs.Scene.from_workload(sc2, "cuda"), icgs.Cameras.from_workload(cams2),
                                    torch.tensor(t2, device="cuda"), 0)
    assert (to_np(s) == 0).any()
