"""Shared helpers of the GPU parity tests (comparison of the CUDA path with the FP64 oracle)."""
import numpy as np

from oracle import oracle as O

# Tolerances (relative, per Gaussian: ||c_gpu - c_oracle|| / ||c_oracle||).
TOL_FP32 = 1e-4      # FP32 targets / CUDA-core path
TOL_BF16 = 2e-3      # BF16 tensor-core feature path
W_MIN = 1.0          # Gaussians with less total visibility than one pixel-weight are reported only
STAKE_REL = 1e-3     # Gaussians whose near-threshold decisions put more than this fraction of
                     # their visibility at stake are reported separately (threshold flips)


def coefficient_report(c_gpu, col, w_min=W_MIN, stake_rel=STAKE_REL):
    """Split Gaussians into the checked set (enough visibility, no decision within the oracle's
    margin deciding more than stake_rel of the visibility) and the rest; return error stats."""
    c_ref = col["c"]
    err = O.relative_errors(np.asarray(c_gpu, np.float64), c_ref)
    w = col["w"]
    stake = (col["stake_own"] + col["stake_up"]).sum(0)
    seen = w > 0
    checked = (w >= w_min) & (stake <= stake_rel * w)
    flagged = seen & ~checked
    rep = dict(n=len(w), seen=int(seen.sum()), checked=int(checked.sum()), flagged=int(flagged.sum()),
               max_checked=float(err[checked].max()) if checked.any() else 0.0,
               p99_checked=float(np.percentile(err[checked], 99)) if checked.any() else 0.0,
               p99_seen=float(np.percentile(err[seen], 99)) if seen.any() else 0.0,
               max_seen=float(err[seen].max()) if seen.any() else 0.0,
               worst=int(np.argmax(np.where(checked, err, -1))) if checked.any() else -1)
    return rep, err, checked


def to_np(t):
    return t.detach().float().cpu().numpy()
