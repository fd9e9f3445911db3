"""icgs_colorize_host: the targets come from host memory and the coefficients go back to host
memory, with the copies staged per camera chunk and overlapped with the walk. Its results must
match icgs_colorize on the same inputs (the two differ only by the order of FP32 atomic sums), for
pinned and pageable targets, one and several camera passes, the CUDA-core and the tensor-core walk,
and on repeated calls that reuse the staging region."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import TOL_FP32, TOL_BF16, coefficient_report, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


def _max_rel(c_a, c_b, ok):
    e = O.relative_errors(np.asarray(c_a, np.float64), np.asarray(c_b, np.float64))
    return float(e[ok].max()) if ok.any() else 0.0


def _rgb_scene():
    sc = W.cluster_scene(3000, 95, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(16, 4.0, 100, 76, 50.0)
    t = O.render(sc, cams, W.sh_coefficients(sc.n, 3, 3, seed=96), 3).astype(np.float32)
    return sc, cams, t


@pytest.mark.parametrize("cam_batch", [0, 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_matches_device_call(icgs, cam_batch, pinned):
    sc, cams, t = _rgb_scene()
    gs = icgs.Scene.from_workload(sc, "cuda")
    gc = icgs.Cameras.from_workload(cams)
    c_dev, s_dev, _ = icgs.colorize(gs, gc, torch.tensor(t, device="cuda"), 3, cam_batch=cam_batch)
    s_dev = to_np(s_dev)
    host_t = torch.tensor(t)
    if pinned:
        host_t = host_t.pin_memory()
    for call in range(2):  # the second call overwrites the staging region of the first
        c_h, s_h = icgs.colorize_host(gs, gc, host_t, 3, cam_batch=cam_batch)
        assert not c_h.is_cuda and not s_h.is_cuda
        s_h = s_h.numpy()
        assert np.array_equal(s_h == icgs.GAUSSIAN_UNSEEN, s_dev == icgs.GAUSSIAN_UNSEEN)
        ok = (s_h == 0) & (s_dev == 0)
        err = _max_rel(c_h.numpy(), to_np(c_dev), ok)
        print(f"host call {call} (cam_batch {cam_batch}, pinned {pinned}): max rel diff to device call {err:.2e}")
        assert ok.sum() > 0.5 * (s_h != icgs.GAUSSIAN_UNSEEN).sum()
        assert err <= TOL_FP32


def test_host_call_against_oracle(icgs):
    sc, cams, t = _rgb_scene()
    col = O.colorize(sc, cams, t.astype(np.float64), 3)
    gs = icgs.Scene.from_workload(sc, "cuda")
    gc = icgs.Cameras.from_workload(cams)
    c_h, s_h = icgs.colorize_host(gs, gc, torch.tensor(t).pin_memory(), 3)
    rep, err, checked = coefficient_report(c_h.numpy(), col, tol=TOL_FP32)
    print("host call vs oracle", rep)
    assert rep["max_checked"] <= TOL_FP32
    assert rep["bound_excess"] <= 0


def test_host_call_tensor_core_masks(icgs):
    """16-class FP16 masks at L = 0 take the tensor-core walk; chunked staging must not change it."""
    sc = W.cluster_scene(2500, 97, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(12, 4.0, 96, 72, 50.0)
    K = 16
    labels = W.voronoi_labels(sc.means, K, 98, 1.5)
    img = O.render(sc, cams, W.one_hot_dc(labels, K), 0)
    t = torch.tensor(np.eye(K, dtype=np.float32)[img.argmax(-1)]).half()
    gs = icgs.Scene.from_workload(sc, "cuda")
    gc = icgs.Cameras.from_workload(cams)
    lam = [1e-5]
    c_dev, s_dev, _ = icgs.colorize(gs, gc, t.cuda(), 0, lam=lam)
    c_h, s_h = icgs.colorize_host(gs, gc, t.pin_memory(), 0, lam=lam)
    ok = (s_h.numpy() == 0) & (to_np(s_dev) == 0)
    err = _max_rel(c_h.numpy(), to_np(c_dev), ok)
    print(f"host call, tensor-core masks: max rel diff to device call {err:.2e}")
    assert err <= TOL_BF16
