"""Shared helpers of the GPU parity tests (comparison of the CUDA path with the FP64 oracle)."""
import numpy as np

from oracle import oracle as O

# Tolerances (relative, per Gaussian: ||c_gpu - c_oracle|| / ||c_oracle||).
TOL_FP32 = 1e-4      # FP32 targets / CUDA-core path
TOL_BF16 = 2e-3      # BF16 tensor-core feature path
W_MIN = 1.0          # Gaussians with less total visibility than one pixel-weight are reported only
CHECK_FRAC = 0.1     # "checked": the flip bound is at most this fraction of the tolerance


def flip_rel(col):
    """Per-Gaussian bound on the relative coefficient change that threshold flips can cause
    (oracle.flip_bound over the oracle's stakes, divided by the error metric's denominator)."""
    if "flip_rel" in col:
        return col["flip_rel"]
    stake = col["stake_own"] + col["stake_up"]
    fb, gamma = O.flip_bound(col["c"], col["A"], col["Y"], col["lam"], stake, col["stake_tw"], w=col["w"],
                             with_gamma=True)
    col["flip_gamma"] = gamma
    r = np.linalg.norm(col["c"].reshape(col["c"].shape[0], -1), axis=1)
    floor = 1e-6 * (r.max() if r.size else 1.0)
    rel = fb / np.maximum(r, floor if floor > 0 else 1e-30)
    col["flip_rel"] = rel
    return rel


def coefficient_report(c_gpu, col, w_min=W_MIN, tol=TOL_FP32):
    """Per-Gaussian relative errors against the oracle.

    A threshold decision that float32 and float64 can take differently (alpha near 1/255, T near
    1e-4) legitimately moves the weight it decides. The oracle bounds, per Gaussian, the
    coefficient change any combination of such flips can cause (flip_rel; derivation in
    oracle.flip_bound). Every Gaussian with w >= w_min and a finite bound must satisfy
    err <= tol + flip_rel (`bound_excess` = the largest err - (tol + flip_rel), <= 0 when it
    holds); the "checked" ones, whose bound is at most CHECK_FRAC * tol, are reported separately
    (`max_checked`, `p99_checked`)."""
    c_ref = col["c"]
    err = O.relative_errors(np.asarray(c_gpu, np.float64), c_ref)
    w = col["w"]
    fr = flip_rel(col)
    seen = w > 0
    eligible = w >= w_min
    bounded = eligible & np.isfinite(fr)
    checked = eligible & (fr <= CHECK_FRAC * tol)
    excess = err[bounded] - (tol + fr[bounded])
    rep = dict(n=len(w), seen=int(seen.sum()), eligible=int(eligible.sum()), checked=int(checked.sum()),
               within_2tol=int((eligible & (fr <= tol)).sum()), unbounded=int((eligible & ~bounded).sum()),
               max_checked=float(err[checked].max()) if checked.any() else 0.0,
               p99_checked=float(np.percentile(err[checked], 99)) if checked.any() else 0.0,
               max_eligible=float(err[eligible].max()) if eligible.any() else 0.0,
               p99_seen=float(np.percentile(err[seen], 99)) if seen.any() else 0.0,
               max_seen=float(err[seen].max()) if seen.any() else 0.0,
               bound_excess=float(excess.max()) if bounded.any() else -1.0,
               worst=int(np.argmax(np.where(checked, err, -1))) if checked.any() else -1)
    return rep, err, checked


# Adjoint (dL/dt, dL/do) against the oracle's FP64 adjoint, worst element over the pixels and
# Gaussians that no near threshold decision touches (on the others a flip legitimately changes the
# contributor set the gradient runs over).
ADJ_TOL_T = 1e-3     # per pixel: |d| / max(|ref|, 1e-3 max|ref|)
ADJ_TOL_O = 1e-3     # per Gaussian: |d| / max(|ref|, 1e-3 max|ref|)


GAMMA_DIRTY = 1e-5   # adjoint: a Gaussian whose A flips may move by more than this (relative) is "dirty"


def adjoint_flags(scene, cams, targets, col, threads=None):
    """The oracle's flags for the adjoint's clean sets. A Gaussian is "dirty" when flips of its near
    decisions may move its A enough to matter: the solve u = A^-1 dL/dc then moves by up to
    gamma / (1 - gamma) relative (oracle.flip_bound), and GAMMA_DIRTY keeps that far below the
    adjoint tolerance. Flagged pixels: a near decision, or a dirty contributor."""
    flip_rel(col)
    dirty = col["flip_gamma"] > GAMMA_DIRTY
    f = O.accumulate_stakes(scene, cams, targets, flags=True, dirty=dirty, threads=threads)
    f["dirty"] = dirty
    return f


def adjoint_report(gt, go, gt_ref, go_ref, col, flags, w_min=W_MIN):
    """Worst relative errors of the adjoint over the clean sets: pixels that no near decision and
    no dirty Gaussian touches (flags["pix_flag"] == 0, see adjoint_flags) for dL/dt; Gaussians with
    w >= w_min, not dirty, and with no weight in a flagged pixel for dL/do."""
    clean_px = flags["pix_flag"] == 0
    ft = np.abs(gt_ref).max() * 1e-3
    et = np.abs(gt - gt_ref) / np.maximum(np.abs(gt_ref), ft)
    clean_g = (col["w"] >= w_min) & (flags["flag_w"].sum(0) == 0)
    if "dirty" in flags:
        clean_g &= ~flags["dirty"]
    fo = np.abs(go_ref).max() * 1e-3
    eo = np.abs(go - go_ref) / np.maximum(np.abs(go_ref), fo)
    return dict(pixels=int(clean_px.size), clean_pixels=int(clean_px.sum()),
                dt_max_clean=float(et[clean_px].max()) if clean_px.any() else 0.0,
                dt_p999_all=float(np.percentile(et, 99.9)), dt_max_all=float(et.max()),
                gaussians=int((col["w"] >= w_min).sum()), clean_gaussians=int(clean_g.sum()),
                do_max_clean=float(eo[clean_g].max()) if clean_g.any() else 0.0,
                do_p99_all=float(np.percentile(eo[col["w"] >= w_min], 99)), do_max_all=float(eo[col["w"] >= w_min].max()))


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
