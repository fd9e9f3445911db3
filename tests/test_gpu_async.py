"""The enqueue-only C ABI (icgs_colorize_async + icgs_async_status): two colorize calls on two
streams with separate workspaces and no host synchronisation between them, each against the FP64
oracle; the call returns while its work is still running; device-side outcomes (capacity overflow,
non-finite targets) surface when the caller joins."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import TOL_BF16, TOL_FP32, coefficient_report, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


def test_two_streams_without_host_sync(icgs):
    sc = W.cluster_scene(3000, 11, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(16, 4.0, 96, 72, 50.0)
    # stream 1: L = 3 RGB on the CUDA-core walk; stream 2: 16 FP16 channels on the tensor-core walk
    t_rgb = O.render(sc, cams, W.sh_coefficients(sc.n, 3, 3, seed=13), 3).astype(np.float32)
    t_msk = W.fourier_fields(cams.n, 72, 96, 16, 14, n_modes=6)
    col_rgb = O.colorize(sc, cams, t_rgb.astype(np.float64), 3)
    tm = torch.tensor(t_msk, device=DEV).half()
    col_msk = O.colorize(sc, cams, tm.float().cpu().numpy().astype(np.float64), 0, [1e-5])
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    tr = torch.tensor(t_rgb, device=DEV)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s1):
        h1 = icgs.colorize_async(gs, gc, tr, 3)
    with torch.cuda.stream(s2):
        h2 = icgs.colorize_async(gs, gc, tm, 0, lam=[1e-5])
    c1, st1, _ = h1.wait()
    c2, st2, _ = h2.wait()
    rep1, _, _ = coefficient_report(to_np(c1), col_rgb, tol=TOL_FP32)
    rep2, _, _ = coefficient_report(to_np(c2), col_msk, tol=TOL_BF16)
    print("async rgb", rep1, "async masks", rep2)
    assert rep1["max_checked"] <= TOL_FP32 and rep1["bound_excess"] <= 0
    assert rep2["max_checked"] <= TOL_BF16 and rep2["bound_excess"] <= 0
    # the same results as the synchronous call on the same inputs (the only difference between runs
    # is the order of the FP32 atomic sums)
    c1s, _, _ = icgs.colorize(gs, gc, tr, 3)
    e = O.relative_errors(to_np(c1), to_np(c1s).astype(np.float64))
    assert np.percentile(e[to_np(st1) != icgs.GAUSSIAN_UNSEEN], 99) <= TOL_FP32


def test_async_call_returns_before_its_work_finishes(icgs):
    """20 cameras of the relighting scene (about 3 ms of GPU work): the stream is idle before the
    call and still busy when it returns, so the call did not wait for its work."""
    sc = W.make_scene("relight", 2000)
    cams = W.make_cameras("relight").subset(np.arange(20))
    t = torch.tensor(W.fourier_fields(cams.n, cams.height, cams.width, 3, seed=21, n_modes=4), device=DEV)
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    icgs.colorize_async(gs, gc, t, 3).wait()  # warm-up (module load, allocator)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert s.query()
        h = icgs.colorize_async(gs, gc, t, 3)
        busy = not s.query()
    h.wait()
    assert s.query()
    assert busy


def test_async_device_outcomes_surface_at_the_join(icgs):
    sc = W.cluster_scene(2000, 31, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(6, 4.0, 64, 48, 50.0)
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    t = torch.rand((cams.n, 48, 64, 3), device=DEV)
    # capacity overflow: reported by the join, with the count to retry with
    h = icgs.colorize_async(gs, gc, t, 0, instance_capacity=64)
    with pytest.raises(icgs.IcgsError) as ei:
        h.wait()
    assert ei.value.status == icgs.ERR_CAPACITY
    need = int(icgs.load().icgs_last_required_instances())
    assert need > 64
    c, _, _ = icgs.colorize_async(gs, gc, t, 0, instance_capacity=need).wait()
    assert torch.isfinite(c).all()
    # a NaN target inside the footprint of the scene: ERR_NONFINITE_INPUT, synchronous and enqueue-only
    t_bad = t.clone()
    t_bad[2, 24, 32, 1] = float("nan")
    t_bad[4, 20, 30, 0] = float("inf")
    with pytest.raises(icgs.IcgsError) as ei:
        icgs.colorize(gs, gc, t_bad, 0)
    assert ei.value.status == icgs.ERR_NONFINITE_INPUT
    with pytest.raises(icgs.IcgsError) as ei:
        icgs.colorize_async(gs, gc, t_bad, 3).wait()
    assert ei.value.status == icgs.ERR_NONFINITE_INPUT
    # FP16 targets on the tensor-core walk
    tb = torch.rand((cams.n, 48, 64, 16), device=DEV).half()
    tb[1, 24, 32, 5] = float("nan")
    with pytest.raises(icgs.IcgsError) as ei:
        icgs.colorize(gs, gc, tb, 0)
    assert ei.value.status == icgs.ERR_NONFINITE_INPUT
    # and the next well-formed call works
    c, _, _ = icgs.colorize(gs, gc, t, 0)
    assert torch.isfinite(c).all()
