"""Per-pixel blend weights w = alpha T (Eq. 2, Eq. 4) of the CUDA walk against the oracle's, read
through icgs_render with one-hot colours: with L = 0 and c[g_k, 0, k] = 1/Y_0, channel k of the
render is the weight map of Gaussian g_k. This measures the float32 error of the walk's alpha and T
directly, and checks the premise of the flip bound: outside the oracle's near-decision margins
(oracle.DELTA_ALPHA, oracle.DELTA_T) no decision is taken differently, and the weight errors there
stay far below those margins."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

from _parity import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Y0 = 1.0 / math.sqrt(4.0 * math.pi)
N_SAMPLE = 64


def _weights_report(icgs, scene, cams, sample):
    dev = "cuda"
    gs = icgs.Scene.from_workload(scene, dev)
    gc = icgs.Cameras.from_workload(cams)
    K = len(sample)
    coeffs = torch.zeros((scene.n, 1, K), dtype=torch.float32, device=dev)
    coeffs[torch.as_tensor(sample, device=dev), 0, torch.arange(K, device=dev)] = 1.0 / Y0
    img = to_np(icgs.render(gs, gc, coeffs, 0))               # [C,H,W,K]
    pos = {int(g): k for k, g in enumerate(sample)}
    sub = scene.subset(sample)
    stats = dict(pairs=0, flagged_pairs=0, flips_outside=0, flips_inside=0, max_rel=0.0, max_rel_front=0.0,
                 rel=[])
    for j in range(cams.n):
        p = O.project(sub, cams, j)
        mask = np.zeros((cams.height, cams.width), bool)
        for k in range(K):
            if p["visible"][k]:
                mask[int(p["y0"][k]):int(p["y1"][k]) + 1, int(p["x0"][k]):int(p["x1"][k]) + 1] = True
        pix, gid, w, T = O.weights(scene, cams, j, mask=mask, with_T=True)
        flags = O.accumulate_stakes(scene, cams.subset([j]), np.zeros((1, cams.height, cams.width, 1)),
                                    mask=mask[None], flags=True)["pix_flag"][0].reshape(-1)
        keep = np.isin(gid, sample)
        pix, gid, w, T = pix[keep], gid[keep], w[keep], T[keep]
        kk = np.array([pos[int(g)] for g in gid], np.int64)
        g_img = img[j].reshape(-1, K)
        gw = g_img[pix, kk].astype(np.float64)
        # pairs the GPU takes and the oracle does not (inside the walked pixels)
        ora = np.zeros_like(g_img, dtype=bool)
        ora[pix, kk] = True
        mpix = np.where(mask.reshape(-1))[0]
        extra = (g_img[mpix] != 0) & ~ora[mpix]
        fl = flags.astype(bool)
        missing = gw == 0
        stats["flips_outside"] += int(extra[~fl[mpix]].sum() + missing[~fl[pix]].sum())
        stats["flips_inside"] += int(extra[fl[mpix]].sum() + missing[fl[pix]].sum())
        clean = ~fl[pix] & ~missing
        rel = np.abs(gw - w)[clean] / w[clean]
        stats["pairs"] += int(len(w))
        stats["flagged_pairs"] += int(fl[pix].sum())
        if rel.size:
            stats["max_rel"] = max(stats["max_rel"], float(rel.max()))
            front = (T[clean] == 1.0)
            if front.any():
                stats["max_rel_front"] = max(stats["max_rel_front"], float(rel[front].max()))
            stats["rel"].append(rel)
    rel = np.concatenate(stats.pop("rel")) if stats["pairs"] else np.zeros(1)
    stats["p99_rel"] = float(np.percentile(rel, 99))
    stats["p9999_rel"] = float(np.percentile(rel, 99.99))
    return stats


def _check(stats):
    # no decision differs outside the margins, and the weights there stay below a quarter of the
    # alpha margin (alpha of front pairs, T = 1) and of the stop margin (alpha T of every pair)
    assert stats["pairs"] > 1000
    assert stats["flips_outside"] == 0
    assert stats["max_rel_front"] <= O.DELTA_ALPHA / 4
    assert stats["max_rel"] <= O.DELTA_T / 4


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


def test_blend_weights_mid_scene(icgs):
    sc = W.cluster_scene(4000, 11, radius=1.5, log_scale_mean=-3.6, log_scale_std=0.4)
    cams = W.hemisphere_cameras(24, 4.0, 120, 90, 50.0)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(sc.n, N_SAMPLE, replace=False))
    st = _weights_report(icgs, sc, cams, sample)
    print("weights mid scene", st, "margins", O.DELTA_ALPHA, O.DELTA_T)
    _check(st)


def _visible_sample(sc, cams, n, seed):
    vis = np.zeros(sc.n, bool)
    for j in range(cams.n):
        vis |= O.project(sc, cams, j)["visible"] > 0
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(np.where(vis)[0], n, replace=False))


def test_blend_weights_relight_full_resolution(icgs):
    """The relighting scene (200,000 Gaussians) at its full 800x800 resolution, 8 of its cameras,
    256 Gaussians."""
    sc = W.make_scene("relight", 2000)
    cams = W.make_cameras("relight").subset(np.arange(0, 100, 13))
    st = _weights_report(icgs, sc, cams, _visible_sample(sc, cams, 4 * N_SAMPLE, 8))
    print("weights relight 800x800", st, "margins", O.DELTA_ALPHA, O.DELTA_T)
    _check(st)


def test_blend_weights_segmentation_full_resolution(icgs):
    """The large segmentation scene (3,000,000 Gaussians in a radius-10 ball) at its full 1600x1060
    resolution, 3 of its cameras, 128 Gaussians."""
    sc = W.make_scene("segmentation", 4000)
    cams = W.make_cameras("segmentation").subset([0, 99, 199])
    st = _weights_report(icgs, sc, cams, _visible_sample(sc, cams, 2 * N_SAMPLE, 9))
    print("weights segmentation 1600x1060", st, "margins", O.DELTA_ALPHA, O.DELTA_T)
    _check(st)
