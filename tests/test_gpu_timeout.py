"""The tensor-core walk's failure path: its bounded mbarrier waits. With the diagnostic setting that
leaves the MMAs unissued and shortens the limit to 0.2 ms (icgs_debug_tc_wait), every wait runs out
with no tensor-core work in flight; the kernel frees its TMEM and returns, the call reports
ICGS_ERR_DEVICE_TIMEOUT, and the next normal call on the same context succeeds and matches the
oracle. Nothing here faults, traps or hangs the GPU: the wait is on a barrier nothing arrives on,
bounded in time."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import TOL_BF16, coefficient_report, to_np

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


def test_tensor_core_wait_timeout_is_reported_and_recovers(icgs):
    sc = W.cluster_scene(2500, 21, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(12, 4.0, 96, 72, 50.0)
    tt = torch.tensor(W.fourier_fields(cams.n, 72, 96, 16, 24, n_modes=6), device=DEV).half()
    col = O.colorize(sc, cams, tt.float().cpu().numpy().astype(np.float64), 0, [1e-5])
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    lib = icgs.load()
    lib.icgs_debug_tc_wait(200_000, 0)
    try:
        with pytest.raises(icgs.IcgsError) as ei:
            icgs.colorize(gs, gc, tt, 0, lam=[1e-5], precision="mixed")
        assert ei.value.status == icgs.ERR_DEVICE_TIMEOUT
        assert "bounded wait" in str(ei.value)
    finally:
        lib.icgs_debug_tc_wait(0, 1)
    c, st, _ = icgs.colorize(gs, gc, tt, 0, lam=[1e-5], precision="mixed")
    rep, err, checked = coefficient_report(to_np(c), col, tol=TOL_BF16)
    print("after timeout", rep)
    assert rep["max_checked"] <= TOL_BF16 and rep["bound_excess"] <= 0
