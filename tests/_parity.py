"""Shared helpers of the GPU parity tests (comparison of the CUDA path with the FP64 oracle)."""
import numpy as np

from oracle import oracle as O

# Tolerances (relative, per Gaussian: ||c_gpu - c_oracle|| / ||c_oracle||).
TOL_FP32 = 1e-4      # FP32 targets / CUDA-core path
TOL_BF16 = 2e-3      # BF16 tensor-core feature path
W_MIN = 1.0          # Gaussians with less total visibility than one pixel-weight are reported only
STAKE_REL = 2e-5     # "checked": the oracle's near-threshold decisions (alpha = 1/255, T = 1e-4,
                     # within its relative margin) decide at most this fraction of the visibility
STAKE_GAIN = 20.0    # every other Gaussian with w >= W_MIN: err <= tol + STAKE_GAIN * stake / w


def coefficient_report(c_gpu, col, w_min=W_MIN, stake_rel=STAKE_REL, tol=None):
    """Per-Gaussian relative errors against the oracle.

    A threshold decision that float32 and float64 can take differently (alpha near 1/255, T near
    1e-4) legitimately moves the weight it decides; the oracle records that weight as "stake".
    "checked" Gaussians (enough visibility, negligible stake) are compared at the tolerance;
    the remaining visible ones are bounded by the tolerance plus STAKE_GAIN * stake / w
    (reported as `bound_excess` > 0 when violated)."""
    c_ref = col["c"]
    err = O.relative_errors(np.asarray(c_gpu, np.float64), c_ref)
    w = col["w"]
    stake = (col["stake_own"] + col["stake_up"]).sum(0)
    seen = w > 0
    checked = (w >= w_min) & (stake <= stake_rel * w)
    flagged = seen & ~checked
    others = (w >= w_min) & ~checked
    rel_stake = np.where(w > 0, stake / np.maximum(w, 1e-30), 0.0)
    rep = dict(n=len(w), seen=int(seen.sum()), checked=int(checked.sum()), flagged=int(flagged.sum()),
               max_checked=float(err[checked].max()) if checked.any() else 0.0,
               p99_checked=float(np.percentile(err[checked], 99)) if checked.any() else 0.0,
               p99_seen=float(np.percentile(err[seen], 99)) if seen.any() else 0.0,
               max_seen=float(err[seen].max()) if seen.any() else 0.0,
               worst=int(np.argmax(np.where(checked, err, -1))) if checked.any() else -1)
    if tol is not None:
        excess = err[others] - (tol + STAKE_GAIN * rel_stake[others])
        rep["bound_excess"] = float(excess.max()) if others.any() else -1.0
    return rep, err, checked


def to_np(t):
    return t.detach().float().cpu().numpy()


def psnr_delta(scene, cams, targets, c_gpu, c_ref, sh_degree):
    """Re-rendered image PSNR against the targets (FP64 oracle render of both coefficient sets, peak
    = the targets' largest magnitude) of the GPU's coefficients minus that of the oracle's: the
    image-space effect of the coefficient differences. Returns (delta dB, oracle's PSNR dB)."""
    targets = np.asarray(targets, np.float64)
    peak = float(np.abs(targets).max())
    p_gpu = O.psnr(O.render(scene, cams, np.asarray(c_gpu, np.float64), sh_degree), targets, peak)
    p_ref = O.psnr(O.render(scene, cams, c_ref, sh_degree), targets, peak)
    return p_gpu - p_ref, p_ref
