"""Seeded synthetic inputs: scenes, camera rigs and target fields.

This module only draws random numbers and lays out camera poses. It holds none
of the colorization arithmetic (no projection, blending, basis evaluation or
solve), so both the CUDA path and the CPU oracle can take their inputs from it.

The shapes follow the workloads of the paper's experiments (Sec. 4): a scene of
~1e5-1e6 Gaussians seen by 100-200 calibrated cameras, with RGB, feature or
mask targets. The paper's own captures, the Mip-NeRF 360 / LLFF scenes and the
DINOv2 / SAM2 outputs are not available, so every field here is a synthetic
stand-in with the stated distribution.

Conventions shared with the C ABI:
  * Gaussian i: mean [3], linear scale [3] (>0), rotation quaternion (w,x,y,z)
    [4] (normalised by the consumer), opacity in (0,1).
  * Camera: pinhole, looks down +z, image y axis down; world_to_cam is the
    row-major 3x4 matrix [R|t]; fx = fy = (W/2)/tan(fov_x/2); cx = W/2,
    cy = H/2; pixel (x, y) has its centre at (x+0.5, y+0.5); near plane 0.2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NEAR_Z = 0.2


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # [N,3] float32
    scales: np.ndarray     # [N,3] float32, linear
    quats: np.ndarray      # [N,4] float32, (w,x,y,z), not necessarily unit
    opacity: np.ndarray    # [N]   float32

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity[idx].copy())


@dataclasses.dataclass
class Cameras:
    width: int
    height: int
    fx: np.ndarray         # [C] float32
    fy: np.ndarray         # [C] float32
    cx: np.ndarray         # [C] float32
    cy: np.ndarray         # [C] float32
    world_to_cam: np.ndarray  # [C,3,4] float32
    near_z: float = NEAR_Z

    @property
    def n(self) -> int:
        return int(self.world_to_cam.shape[0])

    def subset(self, idx) -> "Cameras":
        idx = np.atleast_1d(np.asarray(idx))
        return Cameras(self.width, self.height, self.fx[idx].copy(), self.fy[idx].copy(),
                       self.cx[idx].copy(), self.cy[idx].copy(),
                       self.world_to_cam[idx].copy(), self.near_z)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _random_quats(rng, n):
    return rng.standard_normal((n, 4))


def _random_rotation(rng):
    # Haar-distributed rotation from the QR factorisation of a Gaussian matrix.
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _uniform_ball(rng, n, radius):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


def uniform_scene(n, seed, box=1.0, log_scale_mean=-3.5, log_scale_std=0.3,
                  logit_mean=0.0, logit_std=1.5) -> Scene:
    """Means ~ U[-box,box]^3, log-scales ~ N(mean,std) per axis, quaternions =
    N(0,I4) (normalised by the consumer), opacity = sigmoid(N(logit_mean,logit_std))."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, (n, 3))
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, (n, 3)))
    quats = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(logit_mean, logit_std, n))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 quats.astype(np.float32), opacity.astype(np.float32))


def cluster_scene(n, seed, radius=4.0, n_clusters=40, log_scale_mean=-4.5, log_scale_std=0.5,
                  logit_mean=0.5, logit_std=2.0) -> Scene:
    """Mixture of anisotropic 3D Gaussian clusters, rejected to |x| <= radius.

    For radius 4 the cluster centres are uniform in the radius-3 ball and the
    per-cluster axis standard deviations are U(0.1, 0.8); for other radii both
    scale by radius/4.
    """
    rng = np.random.default_rng(seed)
    s = radius / 4.0
    centres = _uniform_ball(rng, n_clusters, 3.0 * s)
    stds = rng.uniform(0.1, 0.8, (n_clusters, 3)) * s
    rots = np.stack([_random_rotation(rng) for _ in range(n_clusters)])
    means = np.empty((n, 3))
    filled = 0
    while filled < n:
        m = n - filled
        cid = rng.integers(0, n_clusters, m)
        local = rng.standard_normal((m, 3)) * stds[cid]
        pts = centres[cid] + np.einsum("nij,nj->ni", rots[cid], local)
        pts = pts[np.linalg.norm(pts, axis=1) <= radius]
        means[filled:filled + len(pts)] = pts
        filled += len(pts)
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, (n, 3)))
    quats = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(logit_mean, logit_std, n))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 quats.astype(np.float32), opacity.astype(np.float32))


def _look_at(position, target=(0.0, 0.0, 0.0)):
    """world_to_cam [R|t] of a camera at `position` looking at `target`; world up +z
    (or +y when the view direction is within ~2.6 deg of the z axis)."""
    p = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - p
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(f @ up) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ p
    return np.concatenate([R, t[:, None]], axis=1)


def _intrinsics(n, width, height, fov_x_deg):
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return (np.full(n, fx, np.float32), np.full(n, fx, np.float32),
            np.full(n, width / 2.0, np.float32), np.full(n, height / 2.0, np.float32))


def ring_cameras(n, radius, elevation_deg, width, height, fov_x_deg) -> Cameras:
    """n cameras on a horizontal ring at the given elevation, azimuth 360/n * k."""
    el = math.radians(elevation_deg)
    poses = []
    for k in range(n):
        az = 2.0 * math.pi * k / n
        pos = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        poses.append(_look_at(pos))
    fx, fy, cx, cy = _intrinsics(n, width, height, fov_x_deg)
    return Cameras(width, height, fx, fy, cx, cy, np.stack(poses).astype(np.float32))


def hemisphere_cameras(n, radius, width, height, fov_x_deg) -> Cameras:
    """n cameras at Fibonacci points of the upper hemisphere: z_k = 1-(k+0.5)/n,
    azimuth k * golden angle, all looking at the origin."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    poses = []
    for k in range(n):
        z = 1.0 - (k + 0.5) / n
        rxy = math.sqrt(max(0.0, 1.0 - z * z))
        az = k * golden
        poses.append(_look_at(radius * np.array([rxy * math.cos(az), rxy * math.sin(az), z])))
    fx, fy, cx, cy = _intrinsics(n, width, height, fov_x_deg)
    return Cameras(width, height, fx, fy, cx, cy, np.stack(poses).astype(np.float32))


def sh_coefficients(n, sh_degree, channels, seed, dc_low=0.0, dc_high=1.0, rest_std=0.1):
    """[N,(L+1)^2,K] float32: the DC coefficient ~ U(dc_low, dc_high), every higher
    coefficient ~ N(0, rest_std)."""
    rng = np.random.default_rng(seed)
    B = (sh_degree + 1) ** 2
    c = rng.normal(0.0, rest_std, (n, B, channels))
    c[:, 0, :] = rng.uniform(dc_low, dc_high, (n, channels))
    return c.astype(np.float32)


def dc_coefficients_from_colors(colors):
    """Degree-0 coefficients whose rendered colour equals `colors` [N,K]: the DC
    basis function is the constant 1/sqrt(4 pi), so c = colour * sqrt(4 pi)."""
    return (np.asarray(colors, np.float64) * math.sqrt(4.0 * math.pi))[:, None, :].astype(np.float32)


def fourier_fields(n_views, height, width, channels, seed, n_modes=32, max_freq=4.0):
    """[V,H,W,K] float32 smooth unit-variance fields: per view and channel,
    sqrt(2/n_modes) * sum_q cos(2 pi (a_q x/W + b_q y/H) + phi_q) with
    a, b ~ U(-max_freq, max_freq) and phi ~ U(0, 2 pi), evaluated at pixel centres."""
    rng = np.random.default_rng(seed)
    xs = (np.arange(width) + 0.5) / width
    ys = (np.arange(height) + 0.5) / height
    out = np.empty((n_views, height, width, channels), np.float32)
    amp = math.sqrt(2.0 / n_modes)
    for v in range(n_views):
        a = rng.uniform(-max_freq, max_freq, (channels, n_modes))
        b = rng.uniform(-max_freq, max_freq, (channels, n_modes))
        ph = rng.uniform(0.0, 2.0 * math.pi, (channels, n_modes))
        for k in range(channels):
            acc = np.zeros((height, width))
            for q in range(n_modes):
                # separable: cos(u+v) = cos u cos v - sin u sin v
                u = 2.0 * math.pi * a[k, q] * xs + ph[k, q]
                w = 2.0 * math.pi * b[k, q] * ys
                acc += np.cos(w)[:, None] * np.cos(u)[None, :] - np.sin(w)[:, None] * np.sin(u)[None, :]
            out[v, :, :, k] = amp * acc
    return out


def voronoi_labels(means, n_classes, seed, radius):
    """Label of each Gaussian = index of its nearest of n_classes seeds drawn
    uniformly in the ball of the given radius."""
    rng = np.random.default_rng(seed)
    seeds = _uniform_ball(rng, n_classes, radius)
    d = ((means[:, None, :].astype(np.float64) - seeds[None]) ** 2).sum(-1)
    return d.argmin(1).astype(np.int32)


def one_hot_dc(labels, n_classes):
    """Degree-0 coefficients whose rendered colour is the one-hot label."""
    colors = np.zeros((labels.shape[0], n_classes))
    colors[np.arange(labels.shape[0]), labels] = 1.0
    return dc_coefficients_from_colors(colors)


def gaussian_noise(shape, std, seed):
    return np.random.default_rng(seed).normal(0.0, std, shape).astype(np.float32)


# --------------------------------------------------------------------------------------
# The five synthetic workloads. Seeds follow 1000*workload + trial.
# --------------------------------------------------------------------------------------
WORKLOADS = {
    # tiny scene, plain FP32 method: L=0, ridge 1e-6
    "tiny": dict(kind="uniform", n=1000, box=1.0, cams="ring", n_cams=8, cam_radius=3.0,
                 elevation=20.0, width=128, height=128, fov=50.0, sh_degree=0, channels=3,
                 target="render_dc", ridge=1e-6),
    # relighting-shaped scene: L=3 RGB, paper's lambda
    "relight": dict(kind="cluster", n=200_000, radius=4.0, cams="hemisphere", n_cams=100,
                    cam_radius=6.0, width=800, height=800, fov=45.0, sh_degree=3, channels=3,
                    target="render_sh3"),
    # feature enrichment: 64 BF16 channels, L=0
    "features": dict(kind="cluster", n=1_000_000, radius=6.0, cams="hemisphere", n_cams=150,
                     cam_radius=9.0, width=1000, height=750, fov=60.0, sh_degree=0, channels=64,
                     target="fourier"),
    # large segmentation: 16-class masks (FP16), L=0; also an RGB L=3 pass
    "segmentation": dict(kind="cluster", n=3_000_000, radius=10.0, cams="hemisphere", n_cams=200,
                         cam_radius=15.0, width=1600, height=1060, fov=55.0, sh_degree=0,
                         channels=16, target="masks"),
}


def make_scene(name, seed, n=None) -> Scene:
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    if w["kind"] == "uniform":
        return uniform_scene(n, seed, box=w["box"])
    return cluster_scene(n, seed, radius=w["radius"])


def make_cameras(name, n_cams=None, width=None, height=None) -> Cameras:
    w = WORKLOADS[name]
    n_cams = w["n_cams"] if n_cams is None else n_cams
    width = w["width"] if width is None else width
    height = w["height"] if height is None else height
    if w["cams"] == "ring":
        return ring_cameras(n_cams, w["cam_radius"], w["elevation"], width, height, w["fov"])
    return hemisphere_cameras(n_cams, w["cam_radius"], width, height, w["fov"])
