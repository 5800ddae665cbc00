"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module draws random numbers and builds camera poses; it holds none of the
method's arithmetic (no projection, no compositing, no loss). Every array is
drawn with ``numpy.random.default_rng(seed)`` in float64 and cast to float32.

Workload shapes follow the streaming set-up of DASS (Sec. 3.1: each timestep
reconstructs a scene from C synchronised views) at the resolutions of the
multi-view videos the paper evaluates on (Sec. 4.1: 1352x1014 for N3DV,
1280x720 for MeetRoom). The datasets themselves are not available; these
seeded scenes stand in for them.

Conventions (shared with the C ABI in include/dass.h):
  * Gaussian parameters are structure-of-arrays, float32, N-major:
    means[N,3], log_scales[N,3], quats[N,4] (w,x,y,z, not normalised),
    opacity_logit[N], sh[N,K,3] with K=(deg+1)^2 real-SH coefficients.
  * Cameras: viewmat is a row-major 4x4 world->camera matrix in the OpenCV
    convention (x right, y down, z forward); pixel centres sit at integer
    coordinates, so the principal point of a centred camera is ((W-1)/2, (H-1)/2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Half-width of the uniform range for the SH DC coefficient so that a degree-0
# colour (dc * 1/(2 sqrt(pi)) + 0.5) is uniform in [0, 1]: the bound is sqrt(pi).
_DC_HALF_RANGE = math.sqrt(math.pi)


@dataclass
class Camera:
    viewmat: np.ndarray  # [4,4] float64 world->camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_record(self) -> np.ndarray:
        """Pack into the 22-word dass_camera layout (16 viewmat floats, fx fy cx cy, W H)."""
        rec = np.zeros(22, dtype=np.float32)
        rec[:16] = self.viewmat.astype(np.float32).reshape(-1)
        rec[16:20] = (self.fx, self.fy, self.cx, self.cy)
        ints = rec.view(np.int32)
        ints[20] = self.width
        ints[21] = self.height
        return rec


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self) -> dict:
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logit=self.opacity_logit, sh=self.sh)

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opacity_logit.copy(), self.sh.copy(), self.sh_degree, dict(self.extra))


def look_at(position, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera 4x4 for an OpenCV camera at `position` looking at `target`."""
    c = np.asarray(position, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - c
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(down, dtype=np.float64), z)
    if np.linalg.norm(x) < 1e-9:  # looking straight along the down axis
        x = np.cross(np.array([0.0, 0.0, 1.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = x, y, z
    m[:3, 3] = -m[:3, :3] @ c
    return m


def pinhole(viewmat, width, height, fovx_deg=60.0) -> Camera:
    fx = (width / 2.0) / math.tan(math.radians(fovx_deg) / 2.0)
    return Camera(viewmat, fx, fx, (width - 1) / 2.0, (height - 1) / 2.0, width, height)


def random_scene(n, sh_degree, seed, box=((-1, 1), (-1, 1), (-1, 1)),
                 log_scale_mean=-4.0, log_scale_std=0.5, sh_rest_std=0.05) -> Scene:
    """Means uniform in `box`, log-scales N(mean, std), quats N(0, I4), opacity
    logits N(0,1) (so opacity = sigmoid(N(0,1))), SH DC uniform (degree-0 colour
    uniform in [0,1]) and higher-order SH N(0, sh_rest_std)."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box], dtype=np.float64)
    hi = np.array([b[1] for b in box], dtype=np.float64)
    means = rng.uniform(lo, hi, size=(n, 3))
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    quats = rng.normal(0.0, 1.0, size=(n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    opacity_logit = rng.normal(0.0, 1.0, size=(n,))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_rest_std, size=(n, k - 1, 3))
    f = np.float32
    return Scene(means.astype(f), log_scales.astype(f), quats.astype(f),
                 opacity_logit.astype(f), sh.astype(f), sh_degree)


def perturbed(scene: Scene, seed, mean_std=0.01, dc_std=0.05) -> Scene:
    """Seed-perturbed copy used to render targets: means + N(0, mean_std), SH DC + N(0, dc_std)."""
    rng = np.random.default_rng(seed)
    out = scene.copy()
    out.means = (scene.means + rng.normal(0, mean_std, size=scene.means.shape)).astype(np.float32)
    out.sh = scene.sh.copy()
    out.sh[:, 0, :] = (scene.sh[:, 0, :] + rng.normal(0, dc_std, size=scene.sh[:, 0, :].shape)).astype(np.float32)
    return out


def dynamic_split(n, frac, seed, dmu_std=1e-3, dq_std=1e-3):
    """Random dynamic subset (sorted indices) and per-dynamic-Gaussian offsets.

    Offsets are packed [N_dyn, 7] = (dmu_x, dmu_y, dmu_z, sigma_w, sigma_x, sigma_y, sigma_z);
    dmu ~ N(0, dmu_std), sigma = (1,0,0,0) + N(0, dq_std) (a near-identity rotation offset)."""
    rng = np.random.default_rng(seed)
    n_dyn = int(round(n * frac))
    idx = np.sort(rng.choice(n, size=n_dyn, replace=False)).astype(np.int32)
    off = np.zeros((n_dyn, 7))
    off[:, :3] = rng.normal(0, dmu_std, size=(n_dyn, 3))
    off[:, 3:] = rng.normal(0, dq_std, size=(n_dyn, 4))
    off[:, 3] += 1.0
    return idx, off.astype(np.float32)


def standard_normal(shape, seed) -> np.ndarray:
    """Plain N(0, I) draws (e.g. the spawn offsets z of densification), float32."""
    return np.random.default_rng(seed).normal(0.0, 1.0, size=shape).astype(np.float32)


def uniform(shape, seed, lo=0.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


# ----------------------------------------------------------------- workloads

def config_a(seed=1001):
    """Smallest case: 2,000 Gaussians, SH degree 0, one 128x128 camera (fov 60 deg)
    at distance 4 on the -z axis looking at the origin (R = I)."""
    scene = random_scene(2000, 0, seed)
    vm = np.eye(4)
    vm[2, 3] = 4.0
    cams = [pinhole(vm, 128, 128, 60.0)]
    return scene, cams


def ring_cameras(n_cams, radius, width, height, fovx_deg=60.0):
    cams = []
    for i in range(n_cams):
        th = 2.0 * math.pi * i / n_cams
        pos = (radius * math.sin(th), 0.0, -radius * math.cos(th))
        cams.append(pinhole(look_at(pos), width, height, fovx_deg))
    return cams


def arc_cameras(n_cams, radius, width, height, yaw_deg=30.0, fovx_deg=60.0):
    cams = []
    for i in range(n_cams):
        yaw = math.radians(-yaw_deg + 2.0 * yaw_deg * i / max(1, n_cams - 1))
        pos = (radius * math.sin(yaw), 0.0, -radius * math.cos(yaw))
        cams.append(pinhole(look_at(pos), width, height, fovx_deg))
    return cams


def sphere_cameras(n_cams, seed, r_lo, r_hi, sizes, fovx_deg=60.0):
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n_cams):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = rng.uniform(r_lo, r_hi)
        w, h = sizes[rng.integers(len(sizes))]
        cams.append(pinhole(look_at(d * r), int(w), int(h), fovx_deg))
    return cams


def config_b(seed=1002, n=100_000, n_cams=4, width=960, height=540):
    """Single timestep, one launch per camera: 100k Gaussians, SH 3, 4 cameras 960x540
    on a ring of radius 4, 10% dynamic with offsets ~ N(0, 1e-3)."""
    scene = random_scene(n, 3, seed)
    cams = ring_cameras(n_cams, 4.0, width, height)
    dyn_idx, offsets = dynamic_split(n, 0.10, seed + 7)
    return scene, cams, dyn_idx, offsets


# Scene box of the forward-facing arc workload: fills the frame at depth 3..5.
ARC_BOX = ((-1.7, 1.7), (-1.3, 1.3), (-1.0, 1.0))


def config_c(seed=1003, n=300_000, n_cams=20, width=1352, height=1014):
    """Batched multi-view timestep: 300k Gaussians, SH 3, 20 cameras 1352x1014 on a
    forward-facing arc (yaw -30..+30 deg, radius 4), 10% dynamic."""
    scene = random_scene(n, 3, seed, box=ARC_BOX)
    cams = arc_cameras(n_cams, 4.0, width, height)
    dyn_idx, offsets = dynamic_split(n, 0.10, seed + 7)
    return scene, cams, dyn_idx, offsets


# ----------------------------------------------------------------- streaming scene

@dataclass
class MovingScene:
    """A scene whose dynamic Gaussians move on seeded sinusoids and rotate, and whose `new`
    Gaussians appear (opacity from ~0 to drawn values) at `t_appear` (the streaming workload).

    means_dyn(t) = means0[dyn] + amplitude * sin(2 pi t / period + phase) * axis; orientation turned
    by rate_deg * t degrees about a per-Gaussian world axis (composed with SciPy's Rotation).
    """
    base: Scene                 # every Gaussian at t = 0 (new ones with opacity logit -20)
    dyn_idx: np.ndarray
    axis: np.ndarray
    phase: np.ndarray
    rot_axis: np.ndarray
    new_idx: np.ndarray
    new_logit: np.ndarray
    amplitude: float = 0.05
    period: float = 40.0
    rate_deg: float = 2.0
    t_appear: int = 15

    def at(self, t) -> Scene:
        sc = self.base.copy()
        d = self.dyn_idx
        s = np.sin(2 * np.pi * t / self.period + self.phase)[:, None]
        sc.means[d] = (self.base.means[d] + self.amplitude * s * self.axis).astype(np.float32)
        # ground-truth rotation of the dynamic Gaussians, composed with SciPy (scalar-last quaternions)
        from scipy.spatial.transform import Rotation
        q0 = self.base.quats[d].astype(np.float64)[:, [1, 2, 3, 0]]
        turn = Rotation.from_rotvec(np.deg2rad(self.rate_deg * t) * self.rot_axis)
        q = (turn * Rotation.from_quat(q0)).as_quat()
        sc.quats[d] = q[:, [3, 0, 1, 2]].astype(np.float32)
        if t >= self.t_appear:
            sc.opacity_logit[self.new_idx] = self.new_logit
        return sc

    def initial(self) -> Scene:
        """G_0 as the reconstruction starts from it: every Gaussian except the ones not yet there."""
        keep = np.setdiff1d(np.arange(self.base.n), self.new_idx)
        b = self.base
        return Scene(b.means[keep].copy(), b.log_scales[keep].copy(), b.quats[keep].copy(),
                     b.opacity_logit[keep].copy(), b.sh[keep].copy(), b.sh_degree)


def moving_scene(n_static, n_dyn, n_new, sh_degree, seed, box=ARC_BOX, log_scale_mean=-4.0, **kw) -> MovingScene:
    """Streaming workload: n_static static + n_dyn dynamic Gaussians (dynamic ones first after the
    static ones), plus n_new Gaussians that appear at t_appear (last rows)."""
    n = n_static + n_dyn + n_new
    sc = random_scene(n, sh_degree, seed, box=box, log_scale_mean=log_scale_mean)
    rng = np.random.default_rng(seed + 1)
    dyn = np.arange(n_static, n_static + n_dyn, dtype=np.int32)
    new = np.arange(n_static + n_dyn, n, dtype=np.int64)
    axis = rng.normal(size=(n_dyn, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    rax = rng.normal(size=(n_dyn, 3))
    rax /= np.linalg.norm(rax, axis=1, keepdims=True)
    new_logit = sc.opacity_logit[new].copy()
    sc.opacity_logit[new] = -20.0
    return MovingScene(sc, dyn, axis, rng.uniform(0, 2 * np.pi, n_dyn), rax, new, new_logit, **kw)
