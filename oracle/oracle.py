"""FP64 CPU oracle for instant colorization of Gaussian splats (arXiv 2604.17155).

TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
may import this module. It shares no code with the CUDA library (paper_2604_17155_gb300) and
never imports it; both take their inputs from paper_2604_17155_gb300.workloads, which holds no
colorization arithmetic.

Layers:
  * icgs_oracle.c (loaded with ctypes): projection, depth ordering, per-pixel front-to-back walk
    (Eq. 2, Eq. 4), the per-image sums V and S (Eq. 5, Eq. 6), render, adjoint walk, and the
    real spherical-harmonic basis (Eq. 3).
  * this file: the fold into the normal equations G_i = sum_j V_i^j Y_ij Y_ij^T,
    b_i = sum_j Y_ij S_ij^T, w_i = sum_j V_i^j (Eq. 12-13) and the regularised solve
    c_i = (G_i + w_i Lambda)^-1 b_i (Eq. 14), written as their plain definitions; dense least
    squares by Householder QR on tiny scenes (the objective of Eq. 15 itself); the adjoint of
    the solve.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icgs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libicgs_oracle.so")
_lib = None

STATUS_OK, STATUS_UNSEEN = 0, 1


def build(force=False) -> str:
    """Compile icgs_oracle.c with gcc. -ffp-contract=off keeps the depth key identical on every
    host (no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _OCam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("w2c", ctypes.c_double * 12), ("near_z", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.icgso_project.argtypes = [i64, P, P, P, P, P, P]
        lib.icgso_project.restype = ctypes.c_int
        lib.icgso_accumulate.argtypes = [i64, P, P, P, P, P, i32, P, P, i32, dbl, dbl, P, P, P, P, P, P, P, P]
        lib.icgso_accumulate.restype = i64
        lib.icgso_render.argtypes = [i64, P, P, P, P, P, i32, P, P, i32, P]
        lib.icgso_render.restype = i64
        lib.icgso_weights.argtypes = [i64, P, P, P, P, P, P, i32, i64, P, P, P, P]
        lib.icgso_weights.restype = i64
        lib.icgso_adjoint.argtypes = [i64, P, P, P, P, P, i32, P, P, P, P, P]
        lib.icgso_adjoint.restype = i64
        lib.icgso_sh_basis.argtypes = [i32, i64, P, P]
        lib.icgso_sh_basis.restype = ctypes.c_int
        lib.icgso_set_threshold_scale.argtypes = [dbl, dbl]
        lib.icgso_set_threshold_scale.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ocam(cams, j):
    c = _OCam()
    c.width, c.height = int(cams.width), int(cams.height)
    c.fx, c.fy = float(cams.fx[j]), float(cams.fy[j])
    c.cx, c.cy = float(cams.cx[j]), float(cams.cy[j])
    w = np.asarray(cams.world_to_cam[j], np.float32).astype(np.float64).reshape(-1)
    for k in range(12):
        c.w2c[k] = float(w[k])
    c.near_z = float(np.float32(cams.near_z))  # the library receives near_z as float32
    return c


def _scene_arrays(scene):
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return f(scene.means), f(scene.scales), f(scene.quats), f(scene.opacity)


def _threads(threads):
    return threads if threads else max(1, min(16, os.cpu_count() or 1))


# ------------------------------------------------------------------------------------------
# Regularisation and basis
# ------------------------------------------------------------------------------------------
def paper_lambda(sh_degree):
    """Per-coefficient Tikhonov weights of Sec. 4 (Implementation details): 1e-5 for the DC
    term, 1e-4 for degree 1, 1e-3 for degree 2, 1e-2 for degree 3."""
    per_band = [1e-5, 1e-4, 1e-3, 1e-2]
    lam = []
    for l in range(sh_degree + 1):
        lam += [per_band[min(l, 3)]] * (2 * l + 1)
    return np.array(lam, np.float64)


def sh_basis(sh_degree, dirs):
    """[M,(L+1)^2] real orthonormal SH (Eq. 3) of the directions [M,3] (any length)."""
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    B = (sh_degree + 1) ** 2
    out = np.empty((dirs.shape[0], B), np.float64)
    if _load().icgso_sh_basis(sh_degree, dirs.shape[0], _ptr(dirs), _ptr(out)) != 0:
        raise ValueError("sh_degree out of range")
    return out


def camera_centres(cams):
    """[C,3] camera centres o_j = -R^T t in double."""
    w = cams.world_to_cam.astype(np.float64)
    R, t = w[:, :, :3], w[:, :, 3]
    return -np.einsum("cji,cj->ci", R, t)


def view_basis(scene, cams, sh_degree):
    """Y_ij = Y(mu_i - o_j) for every camera j and Gaussian i: [C,N,(L+1)^2]. The view direction
    points from the camera centre to the Gaussian mean (Sec. 3, below Eq. 9)."""
    mu = scene.means.astype(np.float64)
    o = camera_centres(cams)
    d = mu[None, :, :] - o[:, None, :]
    return sh_basis(sh_degree, d.reshape(-1, 3)).reshape(cams.n, scene.n, -1)


# ------------------------------------------------------------------------------------------
# Per-camera passes (C)
# ------------------------------------------------------------------------------------------
def project(scene, cams, j):
    """Projection records of camera j: dict of [N] arrays (see icgso_project)."""
    m, s, q, o = _scene_arrays(scene)
    out = np.zeros((scene.n, 16), np.float64)
    c = _ocam(cams, j)
    _load().icgso_project(scene.n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), ctypes.byref(c), _ptr(out))
    names = ["visible", "mx", "my", "cov_xx", "cov_xy", "cov_yy", "conic_a", "conic_b", "conic_c",
             "depth", "key", "qthr", "x0", "x1", "y0", "y1"]
    return {k: out[:, i] for i, k in enumerate(names)}


# Relative margins within which a threshold decision counts as "near" (icgs_oracle.c, walk_pixel):
# alpha against 1/255 and T (1 - alpha) against 1e-4. A near decision may be taken the other way
# by a renderer whose alpha and T carry float32 rounding; the oracle records what it could move.
# Each margin is at least ten times the largest relative error of the float32 walk's alpha (front
# pairs, T = 1) and of its weights alpha T measured against this oracle on the GB300
# (tests/test_gpu_weights.py, which also checks that no decision outside the margins differs).
DELTA_ALPHA = 4e-5
DELTA_T = 2e-4


def accumulate_stakes(scene, cams, targets, mask=None, brute=False, delta=(DELTA_ALPHA, DELTA_T), threads=None,
                      flags=False, dirty=None):
    """Per-camera visibility sums (Eq. 5) and weighted target sums (Eq. 6 numerator), with the
    stake of the near threshold decisions (walk_pixel in icgs_oracle.c).

    targets: [C,H,W,K]; mask: optional [C,H,W] bool of the pixels to walk; delta: (margin of the
    alpha decision, margin of the stop decision), relative. Returns a dict of V [C,N], S [C,N,K],
    stake_own, stake_up [C,N] (bounds on |dV| from a Gaussian's own near decisions and from those in
    front of it), stake_tw [C,N] (the same weighted by the pixels' target norms), pairs [C]; with
    flags=True also pix_flag [C,H,W] (pixels whose walk has a near decision) and flag_w [C,N]
    (each Gaussian's weight in those pixels); dirty [N] bool (optional) also flags every pixel that
    one of those Gaussians contributes to."""
    lib = _load()
    m, s, q, o = _scene_arrays(scene)
    C, N = cams.n, scene.n
    K = targets.shape[-1]
    da, dt = (float(delta), float(delta)) if np.isscalar(delta) else (float(delta[0]), float(delta[1]))
    V = np.zeros((C, N)); S = np.zeros((C, N, K))
    so = np.zeros((C, N)); su = np.zeros((C, N)); stw = np.zeros((C, N))
    pf = np.zeros((C, cams.height, cams.width), np.uint8) if flags else None
    fw = np.zeros((C, N)) if flags else None
    pairs = np.zeros(C, np.int64)
    dm = None if dirty is None else np.ascontiguousarray(dirty, np.uint8)

    def one(j):
        t = np.ascontiguousarray(targets[j], np.float64)
        mk = None if mask is None else np.ascontiguousarray(mask[j], np.uint8)
        c = _ocam(cams, j)
        r = lib.icgso_accumulate(N, _ptr(m), _ptr(s), _ptr(q), _ptr(o), ctypes.byref(c), K, _ptr(t),
                                 _ptr(mk), int(brute), da, dt, _ptr(V[j]), _ptr(S[j]),
                                 _ptr(so[j]), _ptr(su[j]), _ptr(stw[j]),
                                 None if pf is None else _ptr(pf[j]), None if fw is None else _ptr(fw[j]), _ptr(dm))
        if r < 0:
            raise MemoryError("oracle accumulate failed")
        pairs[j] = r

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(C)))
    out = dict(V=V, S=S, stake_own=so, stake_up=su, stake_tw=stw, pairs=pairs)
    if flags:
        out.update(pix_flag=pf, flag_w=fw)
    return out


def accumulate(scene, cams, targets, mask=None, brute=False, delta=(DELTA_ALPHA, DELTA_T), threads=None):
    """accumulate_stakes() as a tuple: V [C,N], S [C,N,K], stake_own [C,N], stake_up [C,N], pairs [C]."""
    a = accumulate_stakes(scene, cams, targets, mask=mask, brute=brute, delta=delta, threads=threads)
    return a["V"], a["S"], a["stake_own"], a["stake_up"], a["pairs"]


class threshold_scale:
    """Test-only context: the alpha threshold 1/255 and the stop threshold 1e-4 scaled by the given
    factors inside the block (icgso_set_threshold_scale). Flips, on purpose, every decision that
    close to a threshold."""

    def __init__(self, alpha_scale=1.0, t_scale=1.0):
        self.a, self.t = float(alpha_scale), float(t_scale)

    def __enter__(self):
        _load().icgso_set_threshold_scale(self.a, self.t)
        return self

    def __exit__(self, *exc):
        _load().icgso_set_threshold_scale(1.0, 1.0)
        return False


def camera_colors(scene, cams, coeffs, sh_degree):
    """C_i(d_ij) = sum_m c_i^m Y_m(d_ij) (Eq. 3): [C,N,K]."""
    Y = view_basis(scene, cams, sh_degree)
    return np.einsum("cnb,nbk->cnk", Y, coeffs.astype(np.float64))


def render(scene, cams, coeffs, sh_degree, mask=None, brute=False, threads=None):
    """Images [C,H,W,K] of Eq. 1-3 (background 0)."""
    lib = _load()
    m, s, q, o = _scene_arrays(scene)
    cols = camera_colors(scene, cams, coeffs, sh_degree)
    K = cols.shape[-1]
    img = np.zeros((cams.n, cams.height, cams.width, K))

    def one(j):
        cj = np.ascontiguousarray(cols[j])
        mk = None if mask is None else np.ascontiguousarray(mask[j], np.uint8)
        c = _ocam(cams, j)
        if lib.icgso_render(scene.n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), ctypes.byref(c), K, _ptr(cj),
                            _ptr(mk), int(brute), _ptr(img[j])) < 0:
            raise MemoryError("oracle render failed")

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(cams.n)))
    return img


def weights(scene, cams, j, brute=False, mask=None, with_T=False):
    """Every nonzero per-pixel visibility V_{i,x,y} (Eq. 4) of camera j:
    (pixel index y*W+x, Gaussian index, weight), and with with_T the transmittance in front of the
    Gaussian. mask: optional [H,W] bool of the pixels to walk."""
    lib = _load()
    m, s, q, o = _scene_arrays(scene)
    c = _ocam(cams, j)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    cap = 1 << 16
    while True:
        pix = np.empty(cap, np.int32); gid = np.empty(cap, np.int32); w = np.empty(cap, np.float64)
        T = np.empty(cap, np.float64) if with_T else None
        cnt = lib.icgso_weights(scene.n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), ctypes.byref(c), _ptr(mk),
                                int(brute), cap, _ptr(pix), _ptr(gid), _ptr(w), _ptr(T))
        if cnt < 0:
            raise MemoryError("oracle weights failed")
        if cnt <= cap:
            return (pix[:cnt], gid[:cnt], w[:cnt], T[:cnt]) if with_T else (pix[:cnt], gid[:cnt], w[:cnt])
        cap = int(cnt)


# ------------------------------------------------------------------------------------------
# Normal equations and the regularised solve (numpy)
# ------------------------------------------------------------------------------------------
def fold(V, S, Y):
    """G_i = sum_j V_i^j Y_ij Y_ij^T, b_i = sum_j Y_ij S_ij^T, w_i = sum_j V_i^j (Eq. 12-14).
    V [C,N], S [C,N,K], Y [C,N,B] -> G [N,B,B], b [N,B,K], w [N]."""
    G = np.einsum("cn,cnb,cnd->nbd", V, Y, Y)
    b = np.einsum("cnb,cnk->nbk", Y, S)
    w = V.sum(0)
    return G, b, w


def solve(G, b, w, lam):
    """c_i = (G_i + w_i Lambda)^-1 b_i (Eq. 14, Alg. 1 line 6). Gaussians that no camera sees
    (w_i = 0) get c_i = 0 and status UNSEEN."""
    N, B, _ = G.shape
    A = G + w[:, None, None] * np.diag(np.asarray(lam, np.float64))[None]
    c = np.zeros_like(b)
    seen = w > 0
    if seen.any():
        c[seen] = np.linalg.solve(A[seen], b[seen])
    status = np.where(seen, STATUS_OK, STATUS_UNSEEN).astype(np.uint8)
    return c, status, A


def colorize(scene, cams, targets, sh_degree, lam=None, mask=None, delta=(DELTA_ALPHA, DELTA_T), threads=None,
             flags=False):
    """The single-shot colorization of Alg. 1 (lines 1-6). Returns a dict with the coefficients
    c [N,(L+1)^2,K], status [N], and the intermediate V, S, G, b, w, stakes and pair count."""
    lam = paper_lambda(sh_degree) if lam is None else np.asarray(lam, np.float64)
    a = accumulate_stakes(scene, cams, targets, mask=mask, delta=delta, threads=threads, flags=flags)
    Y = view_basis(scene, cams, sh_degree)
    G, b, w = fold(a["V"], a["S"], Y)
    c, status, A = solve(G, b, w, lam)
    out = dict(a, c=c, status=status, Y=Y, G=G, b=b, w=w, A=A, lam=lam)
    return out


def flip_bound(c, A, Y, lam, stake, stake_tw, w=None, chunk=4096, with_gamma=False):
    """Per-Gaussian upper bound on ||c'_i - c_i||_F when the near threshold decisions that produced
    the sums are taken the other way in any combination (the walk's stake, icgs_oracle.c).

    Each flipped (pixel, Gaussian) pair moves V_ij by some dV with sum |dV| <= stake_ij, and S_ij
    by dV t_p (t_p the pixel's target), so A_i = G_i + w_i Lambda and b_i move by
      dA = sum dV (Y_ij Y_ij^T + Lambda),   db = sum dV Y_ij t_p^T   (Eq. 12-14).
    Exactly, c' - c = (A + dA)^-1 (db - dA c) = (I + M dA)^-1 M (db - dA c) with M = A^-1, so
      ||c' - c|| <= beta / (1 - gamma),
      beta  = sum_j [ ||M Y_ij|| (stake_tw_ij + ||c^T Y_ij|| stake_ij) + ||M Lambda c||_F stake_ij ],
      gamma = sum_j stake_ij (||M Y_ij|| ||Y_ij|| + ||M Lambda||_2)  (a bound on ||M dA||_2),
    using ||t_p - c^T Y|| <= ||t_p|| + ||c^T Y||. Infinite where gamma >= 1.
    c [N,B,K], A [N,B,B], Y [C,N,B], lam [B], stake and stake_tw [C,N] (own + up). Returns [N]
    (and gamma [N] with with_gamma: any solve with A moves by at most gamma / (1 - gamma) relative)."""
    N = c.shape[0]
    lam = np.asarray(lam, np.float64)
    out = np.zeros(N)
    gam = np.zeros(N)
    live = (stake > 0).any(0)
    if w is not None:
        live &= w > 0
    idx = np.where(live)[0]
    Lam = np.diag(lam)
    for k0 in range(0, len(idx), chunk):
        ii = idx[k0:k0 + chunk]
        Ai = A[ii]
        Yi = Y[:, ii, :]                                            # [C,n,B]
        MY = np.linalg.solve(Ai, Yi.transpose(1, 2, 0))             # [n,B,C]
        nMY = np.linalg.norm(MY, axis=1)                            # [n,C]
        nY = np.linalg.norm(Yi, axis=2).T                           # [n,C]
        ncol = np.linalg.norm(np.einsum("cnb,nbk->nck", Yi, c[ii]), axis=2)   # [n,C]
        nMLc = np.linalg.norm(np.linalg.solve(Ai, lam[None, :, None] * c[ii]).reshape(len(ii), -1), axis=1)
        nML = np.linalg.norm(np.linalg.solve(Ai, np.broadcast_to(Lam, Ai.shape)), ord=2, axis=(1, 2))
        s = stake[:, ii].T
        st = stake_tw[:, ii].T
        beta = (nMY * (st + ncol * s)).sum(1) + nMLc * s.sum(1)
        gamma = (s * nMY * nY).sum(1) + nML * s.sum(1)
        out[ii] = np.where(gamma < 1.0, beta / np.maximum(1.0 - gamma, 1e-300), np.inf)
        gam[ii] = gamma
    return (out, gam) if with_gamma else out


def refine(scene, cams, targets, sh_degree, lam, col, n_steps, threads=None):
    """Iterative refinement (Alg. 1 lines 7-10), starting from colorize()'s result col: each step
    renders the current coefficients (line 8), accumulates the visibility-weighted residual
    targets t - img (line 9; V, Y, w and A stay those of the geometry) and updates
    c <- c + A^-1 (sum_j Y_ij S_res_ij^T - w_i Lambda c_i) (line 10)."""
    lam = paper_lambda(sh_degree) if lam is None else np.asarray(lam, np.float64)
    c = col["c"].copy()
    A, Y, w = col["A"], col["Y"], col["w"]
    seen = w > 0
    for _ in range(n_steps):
        img = render(scene, cams, c, sh_degree, threads=threads)
        _, S_res, _, _, _ = accumulate(scene, cams, targets - img, threads=threads)
        b = np.einsum("cnb,cnk->nbk", Y, S_res)
        rhs = b - w[:, None, None] * lam[None, :, None] * c
        dc = np.zeros_like(c)
        if seen.any():
            dc[seen] = np.linalg.solve(A[seen], rhs[seen])
        c = c + dc
    return c


def dense_lstsq(scene, cams, targets, sh_degree, lam=None):
    """Per-Gaussian minimiser of the regularised objective (Eq. 15 with Eq. 10-11's per-pixel
    form): rows sqrt(V_{i,x,y}) Y_ij against sqrt(V_{i,x,y}) t_{x,y}, plus rows
    sqrt(w_i lambda_m) e_m against 0, solved by Householder QR. Tiny scenes only."""
    lam = paper_lambda(sh_degree) if lam is None else np.asarray(lam, np.float64)
    Y = view_basis(scene, cams, sh_degree)
    N, B = scene.n, Y.shape[-1]
    K = targets.shape[-1]
    rows = [[] for _ in range(N)]
    for j in range(cams.n):
        pix, gid, w = weights(scene, cams, j)
        t = targets[j].reshape(-1, K).astype(np.float64)
        for p, i, wt in zip(pix, gid, w):
            rows[i].append((math.sqrt(wt), Y[j, i], t[p], wt))
    c = np.zeros((N, B, K))
    for i in range(N):
        if not rows[i]:
            continue
        wi = sum(r[3] for r in rows[i])
        A = np.array([r[0] * r[1] for r in rows[i]] + list(np.diag(np.sqrt(wi * lam))))
        rhs = np.array([r[0] * r[2] for r in rows[i]] + [np.zeros(K)] * B)
        Q, R = np.linalg.qr(A)
        c[i] = np.linalg.solve(R, Q.T @ rhs)
    return c


# ------------------------------------------------------------------------------------------
# Adjoint
# ------------------------------------------------------------------------------------------
def adjoint(scene, cams, targets, sh_degree, lam, grad_c, col=None, threads=None):
    """Gradients of a loss L(c) through c = A^-1 b (Eq. 14) with respect to the target images and
    the opacities, given dL/dc [N,B,K]. With u_i = A_i^-1 dL/dc_i:
      dL/dS_ijk = Y_ij . u_ik = a_ijk,
      dL/dV_ij  = -sum_k u_ik^T (Y_ij Y_ij^T + Lambda) c_ik = beta_ij   (w_i = sum_j V_ij),
    and the per-pixel adjoint walk in C turns these into dL/dt and dL/dopacity.
    Returns grad_t [C,H,W,K], grad_o [N]."""
    lam = paper_lambda(sh_degree) if lam is None else np.asarray(lam, np.float64)
    if col is None:
        col = colorize(scene, cams, targets, sh_degree, lam, threads=threads)
    c, A, Y, w = col["c"], col["A"], col["Y"], col["w"]
    u = np.zeros_like(c)
    seen = w > 0
    u[seen] = np.linalg.solve(A[seen], grad_c.astype(np.float64)[seen])
    a = np.einsum("cnb,nbk->cnk", Y, u)                                   # [C,N,K]
    uy = a
    cy = np.einsum("cnb,nbk->cnk", Y, c)
    reg = np.einsum("b,nbk,nbk->n", lam, u, c)
    beta = -(np.einsum("cnk,cnk->cn", uy, cy) + reg[None, :])          # [C,N]
    lib = _load()
    m, s, q, o = _scene_arrays(scene)
    K = targets.shape[-1]
    grad_t = np.zeros((cams.n, cams.height, cams.width, K))
    grad_o = np.zeros((cams.n, scene.n))

    def one(j):
        t = np.ascontiguousarray(targets[j], np.float64)
        aj = np.ascontiguousarray(a[j]); bj = np.ascontiguousarray(beta[j])
        cam = _ocam(cams, j)
        if lib.icgso_adjoint(scene.n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), ctypes.byref(cam), K, _ptr(t),
                             _ptr(aj), _ptr(bj), _ptr(grad_t[j]), _ptr(grad_o[j])) < 0:
            raise MemoryError("oracle adjoint failed")

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(cams.n)))
    return grad_t, grad_o.sum(0)


# ------------------------------------------------------------------------------------------
# Error metrics used by the parity tests
# ------------------------------------------------------------------------------------------
def relative_errors(c_test, c_ref):
    """Per-Gaussian ||c_test - c_ref||_2 / max(||c_ref||_2, 1e-6 * max_i ||c_ref,i||_2)."""
    d = np.linalg.norm((c_test.astype(np.float64) - c_ref).reshape(c_ref.shape[0], -1), axis=1)
    r = np.linalg.norm(c_ref.reshape(c_ref.shape[0], -1), axis=1)
    floor = 1e-6 * (r.max() if r.size else 1.0)
    return d / np.maximum(r, floor if floor > 0 else 1e-30)


def psnr(img, ref, peak=1.0):
    mse = float(np.mean((np.asarray(img, np.float64) - ref) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)
