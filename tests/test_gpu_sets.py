"""Several target sets on one geometry (icgs_colorize_sets; Sec. 4: the same scene under several
lightings, Sec. 3: one inverse shared by every channel) and the segmentation threshold of Sec. 5
fused into the solve: against the FP64 oracle, and against icgs_colorize on each set alone."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import TOL_BF16, TOL_FP32, coefficient_report, flip_rel, to_np

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


def _scene():
    sc = W.cluster_scene(3000, 41, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(16, 4.0, 96, 72, 50.0)
    return sc, cams


@pytest.mark.parametrize("cam_batch", [0, 6])
def test_lighting_sets_share_one_factorisation(icgs, cam_batch):
    """Three RGB lightings (L = 3, FP32), in one call: each set's coefficients match the oracle and
    the single-set call; the one factorisation is the same as the single-set call's."""
    sc, cams = _scene()
    L = 3
    sets = [O.render(sc, cams, W.sh_coefficients(sc.n, L, 3, seed=50 + k), L).astype(np.float32) for k in range(3)]
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    tts = [torch.tensor(t, device=DEV) for t in sets]
    c, st, chol, keep = icgs.colorize_sets(gs, gc, tts, L, cam_batch=cam_batch)
    assert keep is None and c.shape == (sc.n, 16, 9)
    for k in range(3):
        col = O.colorize(sc, cams, sets[k].astype(np.float64), L)
        rep, _, _ = coefficient_report(to_np(c[..., 3 * k:3 * k + 3]), col, tol=TOL_FP32)
        print("set", k, cam_batch, rep)
        assert rep["max_checked"] <= TOL_FP32 and rep["bound_excess"] <= 0
        c1, st1, chol1 = icgs.colorize(gs, gc, tts[k], L, cam_batch=cam_batch)
        ok = to_np(st1) != icgs.GAUSSIAN_UNSEEN
        e = O.relative_errors(to_np(c[..., 3 * k:3 * k + 3]), to_np(c1).astype(np.float64))
        assert np.percentile(e[ok], 99) <= TOL_FP32
        assert np.array_equal(to_np(st) == icgs.GAUSSIAN_UNSEEN, to_np(st1) == icgs.GAUSSIAN_UNSEEN)


def test_mixed_dtype_sets_and_threshold(icgs):
    """An RGB set (FP32, CUDA-core walk) and a 16-class FP16 mask set (tensor-core walk) at L = 0,
    with the threshold 0.6 of Sec. 5: keep is 1 exactly where the oracle's colour c Y_0 >= 0.6,
    apart from Gaussians within the tolerance of the threshold (either answer is valid there)."""
    sc, cams = _scene()
    rgb = np.random.default_rng(61).uniform(0, 1, (cams.n, 72, 96, 3)).astype(np.float32)
    labels = W.voronoi_labels(sc.means, 16, 62, 1.5)
    img = O.render(sc, cams, W.one_hot_dc(labels, 16), 0)
    masks = np.eye(16, dtype=np.float32)[img.argmax(-1)]
    gs = icgs.Scene.from_workload(sc, DEV)
    gc = icgs.Cameras.from_workload(cams)
    lam = [1e-5]
    c, st, chol, keep = icgs.colorize_sets(gs, gc, [torch.tensor(rgb, device=DEV), torch.tensor(masks, device=DEV).half()],
                                           0, lam=lam, threshold=0.6)
    col_rgb = O.colorize(sc, cams, rgb.astype(np.float64), 0, lam)
    col_msk = O.colorize(sc, cams, masks.astype(np.float64), 0, lam)
    rep, _, _ = coefficient_report(to_np(c[..., :3]), col_rgb, tol=TOL_FP32)
    assert rep["max_checked"] <= TOL_FP32 and rep["bound_excess"] <= 0
    rep2, _, _ = coefficient_report(to_np(c[..., 3:]), col_msk, tol=TOL_BF16)
    print("rgb", rep, "masks", rep2)
    assert rep2["max_checked"] <= TOL_BF16 and rep2["bound_excess"] <= 0
    Y0 = 1.0 / np.sqrt(4 * np.pi)
    val = np.concatenate([col_rgb["c"][:, 0, :], col_msk["c"][:, 0, :]], axis=1) * Y0
    want = (val >= 0.6) & (col_rgb["w"] > 0)[:, None]
    got = to_np(keep).astype(bool)
    # within the tolerance plus the flip bound of the threshold, either answer is valid
    tol = np.concatenate([np.full((sc.n, 3), TOL_FP32) + flip_rel(col_rgb)[:, None],
                          np.full((sc.n, 16), TOL_BF16) + flip_rel(col_msk)[:, None]], axis=1)
    # (the relative error is per Gaussian over its channels: a channel may move by err x the norm)
    norms = np.concatenate([np.repeat(np.linalg.norm(val[:, :3], axis=1)[:, None], 3, 1),
                            np.repeat(np.linalg.norm(val[:, 3:], axis=1)[:, None], 16, 1)], axis=1)
    near = np.abs(val - 0.6) <= 2 * tol * norms + 1e-6
    bad = (got != want) & ~near
    print("threshold: kept", int(got.sum()), "of", got.size, "disagreements outside the margin", int(bad.sum()),
          "near", int(near.sum()))
    assert want.sum() > 100 and bad.sum() == 0
    # the threshold needs view-independent values
    with pytest.raises(icgs.IcgsError) as ei:
        icgs.colorize_sets(gs, gc, [torch.tensor(rgb, device=DEV)], 1, threshold=0.6)
    assert ei.value.status == icgs.ERR_UNSUPPORTED
