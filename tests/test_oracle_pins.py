"""Pins of the FP64 oracle against facts that do not come from the oracle itself: library
routines (scipy's spherical harmonics and rotations), closed forms, Monte Carlo and finite
differences of the pinhole projection, brute force, dense QR least squares, and invariants of
the least-squares problem (Sec. 3, Eq. 2-15). These run on the CPU only."""
import math

from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W

Y0 = 1.0 / math.sqrt(4.0 * math.pi)


# ------------------------------------------------------------------------------------------
# helpers: hand-placed scenes in front of an identity camera
# ------------------------------------------------------------------------------------------
def one_camera(width=32, height=32, f=40.0, cx=None, cy=None, w2c=None):
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    w2c = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if w2c is None else w2c
    return W.Cameras(width, height, np.array([f], np.float32), np.array([f], np.float32),
                     np.array([cx], np.float32), np.array([cy], np.float32),
                     np.asarray(w2c, np.float32)[None])


def scene_of(means, scales, opacity, quats=None):
    n = len(means)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quats is None else quats
    return W.Scene(np.asarray(means, np.float32).reshape(n, 3), np.asarray(scales, np.float32).reshape(n, 3),
                   np.asarray(q, np.float32).reshape(n, 4), np.asarray(opacity, np.float32).reshape(n))


def weight_map(scene, cams, j=0):
    pix, gid, w = O.weights(scene, cams, j)
    out = {}
    for p, i, x in zip(pix, gid, w):
        out.setdefault(int(p), []).append((int(i), float(x)))
    return out


# ------------------------------------------------------------------------------------------
# Spherical harmonics (Eq. 3)
# ------------------------------------------------------------------------------------------
def _scipy_real_sh(l, m, theta, phi):
    sp = pytest.importorskip("scipy.special")
    am = abs(m)
    if hasattr(sp, "sph_harm_y"):
        Yc = sp.sph_harm_y(l, am, theta, phi)
    else:  # older scipy: sph_harm(m, n, azimuth, polar)
        Yc = sp.sph_harm(am, l, phi, theta)
    sgn = (-1.0) ** am
    if m > 0:
        return math.sqrt(2.0) * sgn * Yc.real
    if m < 0:
        return math.sqrt(2.0) * sgn * Yc.imag
    return Yc.real


def test_sh_matches_scipy_real_harmonics():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = O.sh_basis(4, d * 3.7)  # length must not matter
    for l in range(5):
        for m in range(-l, l + 1):
            ref = _scipy_real_sh(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, rtol=1e-12, atol=1e-12)


def test_sh_degree1_is_plus_y_z_x():
    d = np.array([[0.3, -0.5, 0.81]])
    d = d / np.linalg.norm(d)
    Y = O.sh_basis(1, d)[0]
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    np.testing.assert_allclose(Y, [Y0, c1 * d[0, 1], c1 * d[0, 2], c1 * d[0, 0]], rtol=1e-14)


def test_sh_orthonormal_by_quadrature():
    x, wx = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wq = (wx[:, None] * np.full(nphi, 2 * math.pi / nphi)[None]).reshape(-1)
    Y = O.sh_basis(3, d)
    gram = (Y * wq[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    rng = np.random.default_rng(1)
    Y = O.sh_basis(3, rng.standard_normal((100, 3)))
    for l in range(4):
        s = (Y[:, l * l:(l + 1) ** 2] ** 2).sum(1)
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * math.pi), rtol=1e-13)


def test_paper_lambda_matches_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_lambda.txt")
    vals = [float(t) for line in open(path) if not line.startswith("#") for t in line.split()]
    np.testing.assert_array_equal(O.paper_lambda(3), vals)
    np.testing.assert_array_equal(O.paper_lambda(0), vals[:1])


# ------------------------------------------------------------------------------------------
# Projection (Eq. 1 with the 3DGS EWA model)
# ------------------------------------------------------------------------------------------
def test_projection_on_axis_isotropic_closed_form():
    f, Z, s = 40.0, 3.0, float(np.float32(0.05))  # inputs are float32
    cams = one_camera(f=f)
    sc = scene_of([[0, 0, Z]], [[s, s, s]], [0.5], quats=[[0.3, 0.2, -0.7, 0.1]])
    p = O.project(sc, cams, 0)
    var = (f * s / Z) ** 2 + 0.3
    assert p["visible"][0] == 1
    np.testing.assert_allclose([p["mx"][0], p["my"][0]], [16.0, 16.0], atol=1e-12)
    np.testing.assert_allclose([p["cov_xx"][0], p["cov_xy"][0], p["cov_yy"][0]], [var, 0, var], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose([p["conic_a"][0], p["conic_b"][0], p["conic_c"][0]], [1 / var, 0, 1 / var], rtol=1e-12, atol=1e-15)
    assert p["depth"][0] == Z


def _camera_pose(rng):
    from scipy.spatial.transform import Rotation
    R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
    t = rng.normal(0, 0.3, 3)
    return np.concatenate([R, t[:, None]], 1)


def _pinhole(X, w2c, f, c):
    Xc = X @ w2c[:, :3].T + w2c[:, 3]
    return np.stack([f * Xc[:, 0] / Xc[:, 2] + c[0], f * Xc[:, 1] / Xc[:, 2] + c[1]], 1)


def _sigma3(scale, quat_wxyz):
    from scipy.spatial.transform import Rotation
    w, x, y, z = quat_wxyz
    R = Rotation.from_quat([x, y, z, w]).as_matrix()  # scipy is scalar-last
    M = R @ np.diag(scale)
    return M @ M.T


def test_projection_matches_monte_carlo_and_finite_difference():
    """Sigma' - 0.3 I equals the covariance of projected samples (linearisation of the pinhole
    map) and J W Sigma W^T J^T with J from central differences of the pinhole map."""
    rng = np.random.default_rng(7)
    f, c = 50.0, (20.0, 15.0)
    for trial in range(4):
        w2c = _camera_pose(rng).astype(np.float32).astype(np.float64)
        o_cam = -w2c[:, :3].T @ w2c[:, 3]
        fwd = w2c[2, :3]
        mean = o_cam + 4.0 * fwd + w2c[0, :3] * rng.uniform(-1, 1) + w2c[1, :3] * rng.uniform(-0.8, 0.8)
        scale = rng.uniform(0.005, 0.04, 3)
        quat = rng.standard_normal(4)
        sc = scene_of([mean], [scale], [0.7], quats=[quat])
        cams = one_camera(40, 30, f=f, cx=c[0], cy=c[1], w2c=w2c)
        p = O.project(sc, cams, 0)
        cov = np.array([[p["cov_xx"][0], p["cov_xy"][0]], [p["cov_xy"][0], p["cov_yy"][0]]]) - 0.3 * np.eye(2)
        m32 = sc.means[0].astype(np.float64)
        S3 = _sigma3(sc.scales[0].astype(np.float64), sc.quats[0].astype(np.float64))
        # finite-difference Jacobian of the pinhole map at the mean
        J = np.zeros((2, 3))
        h = 1e-6
        for a in range(3):
            e = np.zeros(3); e[a] = h
            J[:, a] = (_pinhole((m32 + e)[None], w2c, f, c)[0] - _pinhole((m32 - e)[None], w2c, f, c)[0]) / (2 * h)
        np.testing.assert_allclose(cov, J @ S3 @ J.T, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose([p["mx"][0], p["my"][0]], _pinhole(m32[None], w2c, f, c)[0], rtol=1e-12)
        # Monte Carlo
        L = np.linalg.cholesky(S3)
        X = m32 + rng.standard_normal((200_000, 3)) @ L.T
        U = _pinhole(X, w2c, f, c)
        mc = np.cov(U.T)
        np.testing.assert_allclose(cov, mc, rtol=0.03, atol=0.03 * np.abs(mc).max())


def test_projection_clamps_jacobian_outside_guard_band():
    f, Z = 40.0, 2.0
    cams = one_camera(32, 32, f=f)
    lim = 1.3 * 16 / f
    x = 2.5 * lim * Z  # far outside the clamp, still in front
    sc = scene_of([[x, 0, Z]], [[0.05, 0.02, 0.03]], [0.9])
    p = O.project(sc, cams, 0)
    # cov equals the one of the same Gaussian placed at the clamped position (same depth)
    sc2 = scene_of([[lim * Z, 0, Z]], [[0.05, 0.02, 0.03]], [0.9])
    p2 = O.project(sc2, cams, 0)
    for k in ("cov_xx", "cov_xy", "cov_yy"):  # equal up to the float32 rounding of the position
        np.testing.assert_allclose(p[k][0], p2[k][0], rtol=1e-6)
    np.testing.assert_allclose(p["mx"][0], f * float(np.float32(x)) / Z + 16.0, rtol=1e-12)


def _round_f32(q):
    """The float32 nearest to the rational q (ties to even), by exact comparison of neighbours."""
    if q == 0:
        return 0.0
    a = np.float32(float(q))
    cands = [np.nextafter(a, np.float32(-np.inf)), a, np.nextafter(a, np.float32(np.inf))]
    return float(min(cands, key=lambda f: (abs(Fraction(float(f)) - q), int(np.float32(f).view(np.uint32)) & 1)))


def test_depth_key_is_the_float32_fma_chain():
    """The ordering key is fma(W22, z, fma(W21, y, fma(W20, x, W23))) in float32, each fused
    multiply-add rounded once: checked against exact rational arithmetic, on rotated cameras."""
    rng = np.random.default_rng(11)
    for trial in range(4):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        t = rng.uniform(-1, 1, 3) + [0, 0, 6.0]
        w2c = np.concatenate([R, t[:, None]], 1).astype(np.float32)[None]
        cams = W.Cameras(64, 64, np.array([60.0], np.float32), np.array([60.0], np.float32),
                         np.array([32.0], np.float32), np.array([32.0], np.float32), w2c)
        sc = W.uniform_scene(200, 12 + trial, box=1.5)
        key = O.project(sc, cams, 0)["key"]
        Wf = [float(v) for v in w2c[0].reshape(-1)]
        for i in range(sc.n):
            mx, my, mz = (float(v) for v in sc.means[i])
            k = _round_f32(Fraction(Wf[8]) * Fraction(mx) + Fraction(Wf[11]))
            k = _round_f32(Fraction(Wf[9]) * Fraction(my) + Fraction(k))
            k = _round_f32(Fraction(Wf[10]) * Fraction(mz) + Fraction(k))
            assert key[i] == k, (trial, i, key[i], k)


def test_near_plane_and_opacity_culling():
    cams = one_camera()
    sc = scene_of([[0, 0, 0.19], [0, 0, 0.21], [0, 0, 3.0], [0, 0, 3.0]],
                  [[0.01] * 3] * 4, [0.5, 0.5, 0.5 / 255.0, 1.01 / 255.0])
    vis = O.project(sc, cams, 0)["visible"]
    np.testing.assert_array_equal(vis, [0, 1, 0, 1])


# ------------------------------------------------------------------------------------------
# Per-pixel visibility (Eq. 2, Eq. 4)
# ------------------------------------------------------------------------------------------
def test_single_gaussian_weights_closed_form():
    """One isotropic on-axis Gaussian: every pixel's weight is o exp(-r^2/(2 var)) where it is at
    least 1/255 (pixel centres at x+0.5), and nothing elsewhere; centred on a pixel centre."""
    f, Z, s, o = 40.0, 3.0, float(np.float32(0.3)), float(np.float32(0.6))  # inputs are float32
    cams = one_camera(48, 48, f=f, cx=24.5, cy=24.5)
    sc = scene_of([[0, 0, Z]], [[s, s, s]], [o])
    var = (f * s / Z) ** 2 + 0.3
    wm = weight_map(sc, cams)
    n_expect = 0
    for y in range(48):
        for x in range(48):
            r2 = (x + 0.5 - 24.5) ** 2 + (y + 0.5 - 24.5) ** 2
            a = o * math.exp(-0.5 * r2 / var)
            got = wm.get(y * 48 + x)
            if a >= 1 / 255:
                n_expect += 1
                assert got is not None and len(got) == 1
                assert abs(got[0][1] - a) <= 1e-14
            else:
                assert got is None
    assert len(wm) == n_expect
    assert wm[24 * 48 + 24][0][1] == pytest.approx(o, rel=0, abs=1e-15)
    # total visibility ~ the truncated Gaussian integral 2 pi var (o - 1/255)
    total = sum(v[0][1] for v in wm.values())
    assert total == pytest.approx(2 * math.pi * var * (o - 1 / 255), rel=2e-3)


def test_two_gaussians_front_to_back():
    cams = one_camera(33, 33, cx=16.5, cy=16.5)
    near, far = [0, 0, 2.0], [0, 0, 4.0]
    for order in ([near, far], [far, near]):
        sc = scene_of(order, [[0.05] * 3, [0.1] * 3], [0.7, 0.5])
        centre = weight_map(sc, cams)[16 * 33 + 16]
        front = 0 if order[0] is near else 1
        a_front = 0.7 if front == 0 else 0.5
        wf = dict(centre)
        a_back = float(np.float32(1.2 - a_front))
        a_front = float(np.float32(a_front))
        assert wf[front] == pytest.approx(a_front, abs=1e-15)
        assert wf[1 - front] == pytest.approx(a_back * (1 - a_front), abs=1e-15)


def test_equal_depth_tie_broken_by_index():
    cams = one_camera(33, 33, cx=16.5, cy=16.5)
    sc = scene_of([[0, 0, 3.0], [0, 0, 3.0]], [[0.05] * 3, [0.07] * 3], [0.3, 0.8])
    wf = dict(weight_map(sc, cams)[16 * 33 + 16])
    o0, o1 = float(np.float32(0.3)), float(np.float32(0.8))
    assert wf[0] == pytest.approx(o0, abs=1e-15)
    assert wf[1] == pytest.approx(o1 * (1 - o0), abs=1e-15)


def test_transmittance_stop_and_alpha_cap():
    cams = one_camera(33, 33, cx=16.5, cy=16.5)
    k = 8
    sc = scene_of([[0, 0, 2.0 + 0.1 * i] for i in range(k)], [[0.05] * 3] * k, [0.8] * k)
    wf = dict(weight_map(sc, cams)[16 * 33 + 16])
    # T: 1, .2, .04, .008, .0016, then .00032*(1-.8) < 1e-4 stops before the 6th
    o = float(np.float32(0.8))
    expect = [o * (1 - o) ** i for i in range(5)]
    assert sorted(wf) == list(range(5))
    np.testing.assert_allclose([wf[i] for i in range(5)], expect, rtol=1e-13)
    sc = scene_of([[0, 0, 2.0]], [[0.05] * 3], [0.999])
    assert dict(weight_map(sc, cams)[16 * 33 + 16])[0] == pytest.approx(0.99, abs=1e-15)


def _tiny_random(seed, n=20, n_cams=4, size=32):
    sc = W.uniform_scene(n, seed, box=0.6, log_scale_mean=-2.5, log_scale_std=0.4)
    cams = W.hemisphere_cameras(n_cams, 3.0, size, size, 50.0)
    return sc, cams


def test_bruteforce_equals_scatter_bitwise():
    sc, cams = _tiny_random(3)
    rng = np.random.default_rng(3)
    t = rng.uniform(0, 1, (cams.n, 32, 32, 3))
    a = O.accumulate(sc, cams, t)
    lib = O._load()
    # brute force: every visible Gaussian is a candidate of every pixel
    V = np.zeros((cams.n, sc.n)); S = np.zeros((cams.n, sc.n, 3))
    m, s, q, o = O._scene_arrays(sc)
    for j in range(cams.n):
        c = O._ocam(cams, j)
        tj = np.ascontiguousarray(t[j])
        lib.icgso_accumulate(sc.n, O._ptr(m), O._ptr(s), O._ptr(q), O._ptr(o), O.ctypes.byref(c), 3, O._ptr(tj),
                             None, 1, 0.0, 0.0, O._ptr(V[j]), O._ptr(S[j]), None, None, None, None, None, None)
    np.testing.assert_array_equal(a[0], V)
    np.testing.assert_array_equal(a[1], S)
    coeffs = W.sh_coefficients(sc.n, 2, 3, seed=4)
    np.testing.assert_array_equal(O.render(sc, cams, coeffs, 2), O.render(sc, cams, coeffs, 2, brute=True))


def test_render_is_sum_of_weighted_colors():
    """Eq. 1-3: the rendered pixel equals sum_i V_{i,x,y} C_i(d_ij) over the listed weights."""
    sc, cams = _tiny_random(5, n=30)
    coeffs = W.sh_coefficients(sc.n, 3, 2, seed=6)
    img = O.render(sc, cams, coeffs, 3)
    cols = O.camera_colors(sc, cams, coeffs, 3)
    for j in range(cams.n):
        pix, gid, w = O.weights(sc, cams, j)
        ref = np.zeros((32 * 32, 2))
        np.add.at(ref, pix, w[:, None] * cols[j, gid])
        np.testing.assert_allclose(img[j].reshape(-1, 2), ref, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------------------------------
# Normal equations and the regularised solve (Eq. 12-15)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L,lam", [(0, [1e-6]), (3, None), (2, [0.3] * 9)])
def test_normal_equations_match_dense_qr(L, lam):
    sc, cams = _tiny_random(11, n=25, n_cams=20, size=40)
    rng = np.random.default_rng(12)
    t = rng.uniform(0, 1, (cams.n, 40, 40, 2))
    col = O.colorize(sc, cams, t, L, lam)
    ref = O.dense_lstsq(sc, cams, t, L, lam)
    seen = col["w"] > 0
    assert seen.sum() > 15
    err = O.relative_errors(col["c"][seen], ref[seen])
    assert err.max() < 1e-8, err.max()


def test_l0_closed_form_with_ridge():
    sc, cams = _tiny_random(13, n=40, n_cams=6)
    t = np.random.default_rng(14).uniform(0, 1, (cams.n, 32, 32, 3))
    lam = 1e-2
    col = O.colorize(sc, cams, t, 0, [lam])
    V, S = col["V"].sum(0), col["S"].sum(0)
    seen = V > 0
    ref = Y0 * S[seen] / ((Y0 * Y0 + lam) * V[seen, None])
    np.testing.assert_allclose(col["c"][seen, 0, :], ref, rtol=1e-12)
    assert (col["status"][~seen] == O.STATUS_UNSEEN).all() and (col["c"][~seen] == 0).all()


def test_gram_invariants_addition_theorem():
    sc, cams = _tiny_random(15, n=40, n_cams=10)
    t = np.zeros((cams.n, 32, 32, 1))
    col = O.colorize(sc, cams, t, 3)
    G, w = col["G"], col["w"]
    np.testing.assert_allclose(G[:, 0, 0], w / (4 * math.pi), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(np.trace(G, axis1=1, axis2=2), w * 16 / (4 * math.pi), rtol=1e-12, atol=1e-15)


def test_condition_bound():
    """lambda_min(A_i) >= w_i min(lambda) and lambda_max(A_i) <= w_i ((L+1)^2/(4 pi) + max(lambda))."""
    sc, cams = _tiny_random(16, n=40, n_cams=10)
    col = O.colorize(sc, cams, np.zeros((cams.n, 32, 32, 1)), 3)
    seen = col["w"] > 0
    ev = np.linalg.eigvalsh(col["A"][seen])
    w = col["w"][seen]
    lam = O.paper_lambda(3)
    assert (ev[:, 0] >= w * lam.min() * (1 - 1e-9)).all()
    assert (ev[:, -1] <= w * (16 / (4 * math.pi) + lam.max()) * (1 + 1e-9)).all()


def test_constant_target_gives_constant():
    sc, cams = _tiny_random(17, n=40, n_cams=6)
    tval = np.array([0.25, 0.5, 0.75])
    t = np.broadcast_to(tval, (cams.n, 32, 32, 3)).copy()
    lam = 1e-5
    col = O.colorize(sc, cams, t, 0, [lam])
    seen = col["w"] > 0
    np.testing.assert_allclose(col["c"][seen, 0, :], np.broadcast_to(tval * Y0 / (Y0 ** 2 + lam), (seen.sum(), 3)), rtol=1e-12)
    # L=3, Lambda=0, many views: the unique minimiser is t*sqrt(4 pi) e_1
    sc, cams = _tiny_random(18, n=15, n_cams=40, size=48)
    t = np.broadcast_to(tval, (cams.n, 48, 48, 3)).copy()
    col = O.colorize(sc, cams, t, 3, np.zeros(16))
    ok = col["w"] > 0
    ev = np.linalg.eigvalsh(col["G"][ok])
    ok_idx = np.where(ok)[0][ev[:, 0] > 1e-6 * col["w"][ok]]
    assert len(ok_idx) >= 5
    ref = np.zeros((16, 3)); ref[0] = tval / Y0
    for i in ok_idx:
        np.testing.assert_allclose(col["c"][i], ref, atol=1e-7)


def test_exact_recovery_single_layer():
    """Gaussians whose supports are disjoint in every kept view, each target pixel carrying the
    view-dependent colour of its one contributor: Lambda = 0 recovers c exactly (Eq. 13)."""
    rng = np.random.default_rng(21)
    n = 10
    pts = []
    while len(pts) < n:
        p = rng.uniform(-0.8, 0.8, 3)
        if all(np.linalg.norm(p - q) > 0.5 for q in pts):
            pts.append(p)
    sc = scene_of(pts, [[0.008, 0.005, 0.004]] * n, rng.uniform(0.3, 0.95, n), quats=rng.standard_normal((n, 4)))
    cams = W.hemisphere_cameras(60, 4.0, 192, 192, 60.0)
    keep = []
    for j in range(cams.n):
        pix, gid, w = O.weights(sc, cams, j)
        if len(np.unique(pix)) == len(pix):
            keep.append(j)
    assert len(keep) >= 30
    cams = cams.subset(keep)
    c_true = W.sh_coefficients(n, 3, 3, seed=22)
    cols = O.camera_colors(sc, cams, c_true, 3)
    t = np.zeros((cams.n, 192, 192, 3))
    for j in range(cams.n):
        pix, gid, w = O.weights(sc, cams, j)
        t[j].reshape(-1, 3)[pix] = cols[j, gid]
    col = O.colorize(sc, cams, t, 3, np.zeros(16))
    assert (col["w"] > 0).all()
    err = O.relative_errors(col["c"], c_true.astype(np.float64))
    assert err.max() < 1e-9, err.max()


def test_linear_in_targets_and_invariant_to_camera_and_channel_order():
    sc, cams = _tiny_random(23, n=40, n_cams=8)
    rng = np.random.default_rng(24)
    t1 = rng.uniform(0, 1, (cams.n, 32, 32, 3)); t2 = rng.uniform(0, 1, (cams.n, 32, 32, 3))
    c1 = O.colorize(sc, cams, t1, 3)["c"]; c2 = O.colorize(sc, cams, t2, 3)["c"]
    c12 = O.colorize(sc, cams, 0.3 * t1 - 1.7 * t2, 3)["c"]
    np.testing.assert_allclose(c12, 0.3 * c1 - 1.7 * c2, rtol=1e-9, atol=1e-9 * np.abs(c1).max())
    perm = rng.permutation(cams.n)
    cp = O.colorize(sc, cams.subset(perm), t1[perm], 3)["c"]
    np.testing.assert_allclose(cp, c1, rtol=1e-9, atol=1e-10 * np.abs(c1).max())
    ch = [2, 0, 1]
    cc = O.colorize(sc, cams, t1[..., ch], 3)["c"]
    np.testing.assert_array_equal(cc, c1[..., ch])


# ------------------------------------------------------------------------------------------
# Adjoint
# ------------------------------------------------------------------------------------------
def _loss(c, r):
    return float((r * c * c).sum())


def test_adjoint_targets_exact_central_difference():
    """L = sum r c^2 is quadratic in the targets, so a central difference (h = 1e-3) is exact up to
    rounding; 64 random pixels of the targets."""
    sc, cams = _tiny_random(31, n=30, n_cams=6, size=24)
    rng = np.random.default_rng(32)
    t = rng.uniform(0, 1, (cams.n, 24, 24, 3))
    L = 3
    r = rng.standard_normal((sc.n, 16, 3))
    col = O.colorize(sc, cams, t, L)
    gt, go = O.adjoint(sc, cams, t, L, None, 2 * r * col["c"], col=col)
    idx = np.argwhere(np.abs(gt) > 0)
    pick = idx[rng.choice(len(idx), 64, replace=False)]
    h = 1e-3
    for (j, y, x, k) in pick:
        tp = t.copy(); tp[j, y, x, k] += h
        tm = t.copy(); tm[j, y, x, k] -= h
        fd = (_loss(O.colorize(sc, cams, tp, L)["c"], r) - _loss(O.colorize(sc, cams, tm, L)["c"], r)) / (2 * h)
        assert fd == pytest.approx(gt[j, y, x, k], rel=1e-6, abs=1e-9 * np.abs(gt).max())


def test_adjoint_opacity_central_difference():
    """Central differences (h = 1e-3) of L = sum r c^2 in 64 random opacities against the analytic
    adjoint. A sample whose +-h evaluations change any contributor set (the alpha >= 1/255 or stop
    decision of any pair) is redrawn and counted; opacities within h of the 0.99 cap are not drawn,
    so no clamp changes either."""
    sc, cams = _tiny_random(33, n=200, n_cams=6, size=32)
    rng = np.random.default_rng(34)
    t = rng.uniform(0, 1, (cams.n, 32, 32, 3))
    L = 3
    r = rng.standard_normal((sc.n, 16, 3))
    col = O.colorize(sc, cams, t, L)
    gt, go = O.adjoint(sc, cams, t, L, None, 2 * r * col["c"], col=col)
    h = 1e-3

    def contributors(scene):
        return [tuple(map(np.ndarray.tobytes, O.weights(scene, cams, j)[:2])) for j in range(cams.n)]

    base = contributors(sc)
    checked = redrawn = 0
    for i in rng.permutation(sc.n):
        if col["w"][i] == 0 or sc.opacity[i] + 2 * h >= 0.99:
            continue
        res, same = [], True
        for sgn in (1, -1):
            s2 = sc.subset(np.arange(sc.n)); s2.opacity[i] = np.float32(sc.opacity[i] + sgn * h)
            res.append(O.colorize(s2, cams, t, L))
            same = same and contributors(s2) == base
        if not same:
            redrawn += 1
            continue
        # the step in float32 opacity is what the oracle sees
        dh = float(np.float32(sc.opacity[i] + h)) - float(np.float32(sc.opacity[i] - h))
        fd = (_loss(res[0]["c"], r) - _loss(res[1]["c"], r)) / dh
        assert fd == pytest.approx(go[i], rel=2e-3, abs=1e-6 * np.abs(go).max())
        checked += 1
        if checked == 64:
            break
    print(f"opacity FD: {checked} checked, {redrawn} redrawn")
    assert checked == 64


# ------------------------------------------------------------------------------------------
# Iterative refinement (Alg. 1 lines 7-10)
# ------------------------------------------------------------------------------------------
def test_refinement_single_gaussian_fixed_point():
    """One translucent Gaussian, L = 0: the refinement converges to the stationary point of the
    regularised render loss, c* = Y0 sum a t / (Y0^2 sum a^2 + lam sum a) with a the per-pixel
    alpha (T = 1), reached geometrically."""
    cams = one_camera(33, 33, cx=16.5, cy=16.5)
    sc = scene_of([[0, 0, 3.0]], [[0.15] * 3], [0.8])
    rng = np.random.default_rng(81)
    t = rng.uniform(0, 1, (1, 33, 33, 2))
    lam = 1e-3
    col = O.colorize(sc, cams, t, 0, [lam])
    pix, gid, a = O.weights(sc, cams, 0)
    tp = t[0].reshape(-1, 2)[pix]
    c_star = Y0 * (a[:, None] * tp).sum(0) / (Y0 ** 2 * (a * a).sum() + lam * a.sum())
    c = O.refine(sc, cams, t, 0, [lam], col, 60)
    np.testing.assert_allclose(c[0, 0], c_star, rtol=1e-9)


def test_refinement_step_is_preconditioned_render_gradient():
    """The update of Alg. 1 line 10 is A^-1 times minus the gradient of
    E(c) = 1/2 sum_pixels |t - render(c)|^2 + 1/2 sum_i w_i c_i^T Lambda c_i; the render is linear in
    c, so central differences of E through the oracle's render are exact up to rounding."""
    sc, cams = _tiny_random(91, n=12, n_cams=6, size=24)
    rng = np.random.default_rng(92)
    t = rng.uniform(0, 1, (cams.n, 24, 24, 1))
    L = 1
    lam = O.paper_lambda(L)
    col = O.colorize(sc, cams, t, L, lam)
    c0 = col["c"] + rng.normal(0, 0.05, col["c"].shape) * (col["w"] > 0)[:, None, None]
    col0 = dict(col, c=c0)
    step = O.refine(sc, cams, t, L, lam, col0, 1) - c0
    w = col["w"]

    def energy(c):
        img = O.render(sc, cams, c, L)
        return 0.5 * ((t - img) ** 2).sum() + 0.5 * np.einsum("n,b,nbk,nbk->", w, lam, c, c)

    h = 1e-3
    grad = np.zeros_like(c0)
    for i in np.where(w > 0)[0][:6]:
        for m in range(4):
            cp = c0.copy(); cp[i, m, 0] += h
            cm = c0.copy(); cm[i, m, 0] -= h
            grad[i, m, 0] = (energy(cp) - energy(cm)) / (2 * h)
        np.testing.assert_allclose(col["A"][i] @ step[i, :, 0], -grad[i, :, 0], rtol=1e-6, atol=1e-9)


# ------------------------------------------------------------------------------------------
# Near-threshold stake (walk_pixel): what a flip of an alpha or stop decision can move
# ------------------------------------------------------------------------------------------
DA, DT = O.DELTA_ALPHA, O.DELTA_T


def _centre_stack(opacities, depths=None, t=(0.3, 0.4, 0.5), px=16, scales=None):
    """Gaussians centred on pixel (16, 16) of a 33x33 camera (projected mean = that pixel's
    centre, so alpha there = opacity), front to back; walk pixel (px, 16) only. Returns the
    accumulate_stakes dict and the scene."""
    k = len(opacities)
    depths = [2.0 + 0.25 * i for i in range(k)] if depths is None else depths
    cams = one_camera(33, 33, cx=16.5, cy=16.5)
    sc = scene_of([[0, 0, d] for d in depths], [[0.05] * 3] * k if scales is None else scales, opacities)
    tgt = np.zeros((1, 33, 33, 3))
    tgt[0, 16, px] = t
    mask = np.zeros((1, 33, 33), bool)
    mask[0, 16, px] = True
    return O.accumulate_stakes(sc, cams, tgt, mask=mask, flags=True), sc


def test_stake_alpha_near_threshold_taken():
    """alpha = (1 + DA/2)/255 in front of an opaque-ish Gaussian: the oracle takes it (weight alpha),
    and a renderer that skips it moves that weight and scales the T behind by 1/(1 - alpha). The
    stake bounds both with alpha_hi = (1 + DA)/255: own = alpha_hi, up(back) = w_back alpha_hi/(1 - alpha_hi)."""
    o_f = float(np.float32((1 + 0.5 * DA) / 255))
    o_b = float(np.float32(0.5))
    a, _ = _centre_stack([o_f, o_b])
    a_hi = (1 + DA) / 255
    w_b = o_b * (1 - o_f)
    assert a["V"][0, 0] == pytest.approx(o_f, rel=1e-15)
    assert a["V"][0, 1] == pytest.approx(w_b, rel=1e-15)
    assert a["stake_own"][0, 0] == pytest.approx(a_hi, rel=1e-14)
    assert a["stake_up"][0, 0] == 0.0 and a["stake_own"][0, 1] == 0.0
    assert a["stake_up"][0, 1] == pytest.approx(w_b * a_hi / (1 - a_hi), rel=1e-14)
    tn = math.sqrt(0.3 ** 2 + 0.4 ** 2 + 0.5 ** 2)
    np.testing.assert_allclose(a["stake_tw"][0], (a["stake_own"][0] + a["stake_up"][0]) * tn, rtol=1e-14)
    assert a["pix_flag"][0, 16, 16] == 1 and a["pix_flag"].sum() == 1
    np.testing.assert_allclose(a["flag_w"][0], a["V"][0], rtol=1e-15)


def test_stake_alpha_near_threshold_skipped():
    """alpha = (1 - DA/2)/255 two pixels off the mean of the front Gaussian (isotropic, projected
    variance (f s / Z)^2 + 0.3): skipped by the oracle (no weight), at stake all the same. (An opacity
    below 1/255 would not do: both sides cull such a Gaussian exactly, on its float32 opacity.)"""
    f, Z, s_f = 40.0, 2.0, float(np.float32(0.05))
    var = (f * s_f / Z) ** 2 + 0.3
    o_f = float(np.float32((1 - 0.5 * DA) / 255 * math.exp(4.0 / (2 * var))))
    o_b = float(np.float32(0.5))
    a, _ = _centre_stack([o_f, o_b], px=18, scales=[[s_f] * 3, [1.0] * 3])
    alpha = o_f * math.exp(-4.0 / (2 * var))
    assert abs(alpha * 255 - 1) <= DA and alpha < 1 / 255
    a_hi = (1 + DA) / 255
    w_b = a["V"][0, 1]
    assert a["V"][0, 0] == 0.0 and w_b == pytest.approx(o_b, rel=1e-2)
    assert a["stake_own"][0, 0] == pytest.approx(a_hi, rel=1e-14)
    assert a["stake_up"][0, 1] == pytest.approx(w_b * a_hi / (1 - a_hi), rel=1e-14)
    assert a["stake_up"][0, 0] == 0.0 and a["stake_own"][0, 1] == 0.0


def test_no_stake_outside_the_margins():
    o_f = float(np.float32((1 + 3 * DA) / 255))
    a, _ = _centre_stack([o_f, 0.5, 0.5])
    assert a["stake_own"].sum() == 0 and a["stake_up"].sum() == 0 and a["stake_tw"].sum() == 0
    assert a["pix_flag"].sum() == 0 and a["flag_w"].sum() == 0


def _stop_stack(rel_offset):
    """Two Gaussians of opacity 0.95, then a third whose test T (1 - alpha) lands at
    1e-4 (1 + rel_offset), then a fourth of opacity 0.3."""
    o = float(np.float32(0.95))
    T2 = (1 - o) ** 2
    o3 = float(np.float32(1 - 1e-4 * (1 + rel_offset) / T2))
    return [o, o, o3, float(np.float32(0.3))], T2


def test_stake_stop_near_threshold_continued():
    """test T = 1e-4 (1 + DT/2): the oracle takes the third Gaussian (weight alpha3 T2) and then
    stops before the fourth, whose own stop decision is then also at stake (the T in front of it
    may be the other side's)."""
    ops, T2 = _stop_stack(0.5 * DT)
    a, _ = _centre_stack(ops)
    o3 = ops[2]
    w3 = o3 * T2
    tt = T2 * (1 - o3)
    assert tt >= 1e-4 and abs(tt - 1e-4) <= DT * 1e-4
    assert a["V"][0, 2] == pytest.approx(w3, rel=1e-13)
    assert a["stake_own"][0, 2] == pytest.approx(w3, rel=1e-13)   # the weight a stop there would drop
    # the fourth: T in front = tt, perturbation bound rel = 1; its own stop (tt * 0.7 < 1e-4) is
    # decided within (DT + 1) of 1e-4, so its weight alpha4 tt (1 + 1) is at stake and the oracle stops
    assert a["V"][0, 3] == 0.0
    assert a["stake_own"][0, 3] == pytest.approx(ops[3] * tt * 2.0, rel=1e-13)
    assert a["stake_own"][0, :2].sum() == 0 and a["stake_up"].sum() == 0


def test_stake_stop_near_threshold_stopped():
    """test T = 1e-4 (1 - DT/2): the oracle stops before the third Gaussian; a renderer that goes on
    takes alpha3 T2 and could still take the fourth (bounded by T2 alpha4)."""
    ops, T2 = _stop_stack(-0.5 * DT)
    a, _ = _centre_stack(ops)
    o3 = ops[2]
    assert a["V"][0, 2] == 0.0 and a["V"][0, 3] == 0.0
    assert a["stake_own"][0, 2] == pytest.approx(o3 * T2, rel=1e-13)
    assert a["stake_up"][0, 3] == pytest.approx(T2 * ops[3], rel=1e-13)
    assert a["stake_own"][0, 3] == 0.0


def test_stake_bounds_every_planted_flip():
    """Brute force: moving a threshold by 0.9 of its margin flips every decision that close to it.
    Every change of V (and of S, through the target norms) on random scenes stays within the stake,
    and every coefficient change within oracle.flip_bound."""
    da, dt = 1e-3, 1e-3  # wider than the defaults, so that these small scenes have near decisions
    for seed in (5, 6):
        sc, cams = _tiny_random(seed, n=60, n_cams=6, size=32)
        rng = np.random.default_rng(seed)
        t = rng.uniform(0, 1, (cams.n, 32, 32, 3))
        L = 2
        col = O.colorize(sc, cams, t, L, delta=(da, dt))
        stake = col["stake_own"] + col["stake_up"]
        fb = O.flip_bound(col["c"], col["A"], col["Y"], col["lam"], stake, col["stake_tw"], w=col["w"])
        moved = 0
        for sa, st in ((1 + 0.9 * da, 1), (1 - 0.9 * da, 1), (1, 1 + 0.9 * dt), (1, 1 - 0.9 * dt),
                       (1 - 0.9 * da, 1 + 0.9 * dt)):
            with O.threshold_scale(sa, st):
                c2 = O.colorize(sc, cams, t, L, delta=(da, dt))
            dV = np.abs(c2["V"] - col["V"])
            dS = np.linalg.norm(c2["S"] - col["S"], axis=-1)
            assert (dV <= stake * (1 + 1e-12) + 1e-300).all()
            assert (dS <= col["stake_tw"] * (1 + 1e-12) + 1e-300).all()
            seen = (col["w"] > 0) & (c2["w"] > 0)
            d = np.linalg.norm((c2["c"] - col["c"]).reshape(sc.n, -1), axis=1)
            assert (d[seen] <= fb[seen] * (1 + 1e-9)).all()
            moved += int((dV > 0).sum())
        assert moved > 0
