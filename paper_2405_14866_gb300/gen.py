"""Seeded synthetic scenes for the latent-Gaussian splatting path.

This module only *draws inputs*: per-view depth, foreground mask, scale,
rotation, opacity and feature maps plus pinhole cameras.  It contains none
of the method's arithmetic (no lifting, projection, binning or blending), so
that both the FP64 oracle and the CUDA library can be fed the very same
arrays.

The maps stand in for the outputs of the paper's depth estimator and image
encoder (Sec. 4.1, Sec. 4.2 Eq. 4: M_f in R^{HxWxd}, M_s in R^{HxWx3},
M_alpha in R^{HxWx1}); neither network nor its data is available, so the
values are drawn from the distributions listed with each workload below.

Conventions shared by everything in this repository:
  * camera frame is OpenCV-like: x right, y down, z forward;
  * a camera is (fx, fy, cx, cy, width, height, R, t, z_near, z_far) with
    R, t the world->camera transform, p_cam = R @ x_world + t;
  * pixel (u, v) = (column, row) is centred at image coordinate (u, v).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

FEAT_F32 = 0
FEAT_BF16 = 1


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray  # (3,3) float32, world -> camera
    t: np.ndarray  # (3,) float32
    z_near: float = 0.2
    z_far: float = 1.0e4

    def copy(self) -> "Camera":
        return Camera(self.fx, self.fy, self.cx, self.cy, self.width, self.height,
                      self.R.copy(), self.t.copy(), self.z_near, self.z_far)


@dataclass
class SourceView:
    depth: np.ndarray    # (H,W) f32, camera-space z in metres
    mask: np.ndarray     # (H,W) u8, 1 = foreground
    scale: np.ndarray    # (H,W,3) f32, Gaussian std-devs in metres (M_s)
    quat: np.ndarray     # (H,W,4) f32, (w,x,y,z) rotation in the source camera frame
    opacity: np.ndarray  # (H,W) f32 (M_alpha)
    feat: np.ndarray     # (H,W,C) f32 (M_f)
    cam: Camera


@dataclass
class Scene:
    name: str
    views: List[SourceView]
    targets: List[Camera]
    C: int
    feat_dtype: int           # storage dtype of the lifted features
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_foreground(self) -> int:
        return int(sum(int(v.mask.sum()) for v in self.views))


# --------------------------------------------------------------------------
# small geometry helpers for *placing* cameras (input construction only)
# --------------------------------------------------------------------------

def rot_x(deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def rot_y(deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def look_at_c2w(center, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """Camera->world rotation whose +z axis points from `center` to `target`
    (OpenCV frame: +y of the camera is 'down', so world up is -y)."""
    c = np.asarray(center, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    upv = np.asarray(up, np.float64)
    x = np.cross(z, upv)           # right = forward x up (y down, z forward)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def make_camera(f: float, width: int, height: int, center, R_c2w,
                cx: Optional[float] = None, cy: Optional[float] = None,
                z_near: float = 0.2, z_far: float = 1.0e4) -> Camera:
    """Pinhole camera at `center` with camera->world rotation `R_c2w`."""
    R_c2w = np.asarray(R_c2w, np.float64)
    R = R_c2w.T
    t = -R @ np.asarray(center, np.float64)
    return Camera(float(f), float(f),
                  float((width - 1) / 2.0 if cx is None else cx),
                  float((height - 1) / 2.0 if cy is None else cy),
                  int(width), int(height),
                  R.astype(np.float32), t.astype(np.float32), float(z_near), float(z_far))


# --------------------------------------------------------------------------
# map generators
# --------------------------------------------------------------------------

def value_noise(rng: np.random.Generator, height: int, width: int, lattice: int = 9) -> np.ndarray:
    """Cosine-interpolated value noise on a lattice x lattice grid of U[0,1]
    samples, min-max normalised to [0, 1]."""
    g = rng.random((lattice, lattice))
    def axis(n):
        pos = np.arange(n, dtype=np.float64) * (lattice - 1) / max(n - 1, 1)
        i0 = np.minimum(np.floor(pos).astype(np.int64), lattice - 2)
        fr = pos - i0
        w = 0.5 - 0.5 * np.cos(math.pi * fr)
        return i0, w
    iy, wy = axis(height)
    ix, wx = axis(width)
    g00 = g[iy][:, ix]
    g01 = g[iy][:, ix + 1]
    g10 = g[iy + 1][:, ix]
    g11 = g[iy + 1][:, ix + 1]
    wx2 = wx[None, :]
    wy2 = wy[:, None]
    n = (g00 * (1 - wx2) + g01 * wx2) * (1 - wy2) + (g10 * (1 - wx2) + g11 * wx2) * wy2
    lo, hi = n.min(), n.max()
    return (n - lo) / max(hi - lo, 1e-12)


def ellipse_mask(height: int, width: int, ax: float, ay: float) -> np.ndarray:
    """Centred ellipse with semi-axes ax*W, ay*H (fractions of the image)."""
    v, u = np.mgrid[0:height, 0:width].astype(np.float64)
    cu, cv = (width - 1) / 2.0, (height - 1) / 2.0
    r = ((u - cu) / (ax * width)) ** 2 + ((v - cv) / (ay * height)) ** 2
    return (r <= 1.0).astype(np.uint8)


def jitter_quats(rng: np.random.Generator, n: int, max_deg: float) -> np.ndarray:
    """Unit quaternions (w,x,y,z) of a rotation by U[0,max_deg] about a
    uniformly random axis."""
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.radians(rng.uniform(0.0, max_deg, size=n))
    q = np.empty((n, 4))
    q[:, 0] = np.cos(ang / 2)
    q[:, 1:] = axis * np.sin(ang / 2)[:, None]
    return q


def _view_maps(rng, cam: Camera, depth: np.ndarray, mask: np.ndarray, C: int,
               isotropic: bool, quat_deg: float) -> SourceView:
    H, W = depth.shape
    if isotropic:
        k = rng.uniform(0.8, 1.5, size=(H, W))
        s = (depth / cam.fx * k)[..., None].repeat(3, axis=2)
    else:
        k = rng.uniform(0.8, 1.5, size=(H, W, 3))
        foot = np.stack([depth / cam.fx, depth / cam.fy,
                         depth / math.sqrt(cam.fx * cam.fy)], axis=2)
        s = foot * k
    if quat_deg > 0:
        q = jitter_quats(rng, H * W, quat_deg).reshape(H, W, 4)
    else:
        q = np.zeros((H, W, 4))
        q[..., 0] = 1.0
    opac = rng.uniform(0.3, 0.95, size=(H, W))
    feat = rng.standard_normal(size=(H, W, C), dtype=np.float32)
    return SourceView(depth.astype(np.float32), mask.astype(np.uint8), s.astype(np.float32),
                      q.astype(np.float32), opac.astype(np.float32), feat, cam)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def scene_tiny(seed: int = 0, res: int = 64, C: int = 8) -> Scene:
    """Tiny plain render, FP32: one 64x64 source view at the origin,
    depth 1.0 + 0.1 sin(u/9) cos(v/7) m, fx=fy=64, cx=cy=32, every pixel a
    Gaussian, isotropic scale depth/fx*U[0.8,1.5], opacity U[0.3,0.95],
    8-channel N(0,1) features; target rotated 5 deg about y and shifted
    5 cm in x."""
    rng = np.random.default_rng(seed)
    f = float(res)
    src = make_camera(f, res, res, (0, 0, 0), np.eye(3), cx=res / 2.0, cy=res / 2.0)
    v, u = np.mgrid[0:res, 0:res].astype(np.float64)
    depth = 1.0 + 0.1 * np.sin(u / 9.0) * np.cos(v / 7.0)
    mask = np.ones((res, res), np.uint8)
    view = _view_maps(rng, src, depth, mask, C, isotropic=True, quat_deg=0.0)
    tgt = make_camera(f, res, res, (0.05, 0, 0), rot_y(5.0), cx=res / 2.0, cy=res / 2.0)
    return Scene("tiny-64x64-c8-f32", [view], [tgt], C, FEAT_F32, seed)


def _rig_two(res: int, f: float, baseline: float = 0.30, verge_deg: float = 10.0):
    half = baseline / 2
    yaw = verge_deg / 2
    return [make_camera(f, res, res, (-half, 0, 0), rot_y(+yaw)),
            make_camera(f, res, res, (+half, 0, 0), rot_y(-yaw))]


def _rig_four(res: int, f: float):
    """Narrow upper pair (15 cm, 0.2 m above, pitched 5 deg down) and a wide
    lower pair (60 cm, yawed to look at (0, 0, 1.2 m))."""
    up = [make_camera(f, res, res, (-0.075, -0.2, 0), rot_x(-5.0)),
          make_camera(f, res, res, (+0.075, -0.2, 0), rot_x(-5.0))]
    yaw = math.degrees(math.atan2(0.30, 1.2))
    low = [make_camera(f, res, res, (-0.30, 0, 0), rot_y(+yaw)),
           make_camera(f, res, res, (+0.30, 0, 0), rot_y(-yaw))]
    return up + low


def _scene_from_rig(name, cams, rng, C, feat_dtype, mask_axes, quat_deg, targets, seed) -> Scene:
    views = []
    for cam in cams:
        H, W = cam.height, cam.width
        depth = 0.8 + 0.8 * value_noise(rng, H, W)
        mask = ellipse_mask(H, W, *mask_axes)
        views.append(_view_maps(rng, cam, depth, mask, C, isotropic=False, quat_deg=quat_deg))
    return Scene(name, views, targets, C, feat_dtype, seed)


def scene_paper(seed: int = 1, res: int = 1024, C: int = 32) -> Scene:
    """Paper-shaped plain render, FP32: two verging views (30 cm baseline,
    10 deg vergence), upper-body ellipse mask (~60%), depth 0.8-1.6 m from
    seeded smooth noise, anisotropic footprint scales x U[0.8,1.5], rotation
    jitter <= 10 deg, 32-channel features; target at the midpoint."""
    rng = np.random.default_rng(seed)
    f = float(res)
    cams = _rig_two(res, f)
    tgt = make_camera(f, res, res, (0, 0, 0), np.eye(3))
    return _scene_from_rig(f"paper-2x{res}-c{C}-f32", cams, rng, C, FEAT_F32,
                           (0.45, 0.425), 10.0, [tgt], seed)


def scene_precision(seed: int = 2, res: int = 1024, C: int = 32) -> Scene:
    """Precision / headline workload: four 1024^2 views (~2.1M foreground
    Gaussians at the 50% ellipse), 32-channel features stored as BF16 and
    composited in FP32, 1024^2 target at the rig centre."""
    rng = np.random.default_rng(seed)
    f = float(res)
    cams = _rig_four(res, f)
    tgt = make_camera(f, res, res, (0, 0, 0), np.eye(3))
    return _scene_from_rig(f"precision-4x{res}-c{C}-bf16", cams, rng, C, FEAT_BF16,
                           (0.42, 0.379), 10.0, [tgt], seed)


def scene_diff_sample(seed: int, res: int = 512, C: int = 16) -> Scene:
    """One sample of the differentiation workload: the two-view rig at
    512^2 (f = 512), 60% mask (~315K Gaussians), 16-channel FP32 features."""
    rng = np.random.default_rng(seed)
    f = float(res)
    cams = _rig_two(res, f)
    tgt = make_camera(f, res, res, (0, 0, 0), np.eye(3))
    sc = _scene_from_rig(f"diff-2x{res}-c{C}-f32", cams, rng, C, FEAT_F32,
                         (0.45, 0.425), 10.0, [tgt], seed)
    sc.extra["target_map"] = rng.standard_normal(size=(C, res, res), dtype=np.float32)
    return sc


def eye_cameras(rng: np.random.Generator, res: int, n_viewers: int,
                focus=(0.0, 0.0, 1.2), ipd: float = 0.064) -> List[Camera]:
    """Left+right eye cameras for each viewer: head within +-0.4 m laterally
    and +-0.15 m in depth of the rig centre, eyes 6.4 cm apart, both looking
    at `focus`."""
    cams = []
    for _ in range(n_viewers):
        head = np.array([rng.uniform(-0.4, 0.4), 0.0, rng.uniform(-0.15, 0.15)])
        for side in (-0.5, 0.5):
            eye = head + np.array([side * ipd, 0.0, 0.0])
            cams.append(make_camera(float(res), res, res, eye, look_at_c2w(eye, focus)))
    return cams


# --------------------------------------------------------------------------
# the paper's display geometry (Sec. 3.1) and its three-view lifting rig
# (Sec. 4.1: Gaussians from the depth maps of cam0, cam2 and cam3)
# --------------------------------------------------------------------------

DISPLAY_DISTANCE = 1.25     # nominal eye-to-display distance (m)
DISPLAY_SCALE = 0.5         # scale of the rendered upper body
PANEL_HALF_HEIGHT = 0.1681  # 27-inch 16:9 panel: 0.598 m x 0.336 m
VIEWER_LATERAL = 0.4        # left-right range 0.8 m (about 40 deg of view)
VIEWER_DEPTH = 0.15         # forward-backward range 0.3 m
REMOTE_EYE_DEPTH = 1.2      # remote eye centre on the rig axis, 1.2 m out


def display_transform(remote_eye_depth: float = REMOTE_EYE_DEPTH, scale: float = DISPLAY_SCALE):
    """Similarity x_local = s * Rm @ x_remote + tm that places the remote
    user in front of the local display (Sec. 3.1).

    Both sites use the frame of their own display: display centre at the
    origin, x right, y down, user on the +z side.  The remote scene is
    turned 180 deg about the vertical axis through the midpoint
    M = (0, 0, d/2) of the remote eye-to-display segment (d = depth of the
    remote eye centre E = (0, 0, d)), which puts E on the display plane,
    then scaled by s about that image of E (the display centre)."""
    d = float(remote_eye_depth)
    Rm = np.diag([-1.0, 1.0, -1.0])
    M = np.array([0.0, 0.0, 0.5 * d])
    e_img = Rm @ (np.array([0.0, 0.0, d]) - M) + M      # = 0: the display centre
    tm = scale * (M - Rm @ M - e_img) + e_img
    return float(scale), Rm, tm


def display_eye_camera(eye_local, res: int, remote_eye_depth: float = REMOTE_EYE_DEPTH,
                       scale: float = DISPLAY_SCALE) -> Camera:
    """Camera in the remote capture frame that sees the remote Gaussians as
    a local eye at `eye_local` (display frame) sees them on the display.

    The local eye looks at the display centre; its image spans the panel
    height at the nominal 1.25 m (f = res * 1.25 / (2 * half height)).  A
    perspective image is unchanged when the scene and the camera centre are
    scaled together about a point, so the eye camera is carried back through
    the inverse similarity: centre s^-1 Rm^T (e - tm), rotation Rm^T R_eye,
    same intrinsics."""
    s, Rm, tm = display_transform(remote_eye_depth, scale)
    e = np.asarray(eye_local, np.float64)
    R_eye = look_at_c2w(e, (0.0, 0.0, 0.0))
    centre = Rm.T @ (e - tm) / s
    f = res * DISPLAY_DISTANCE / (2.0 * PANEL_HALF_HEIGHT)
    return make_camera(f, res, res, centre, Rm.T @ R_eye)


def display_eye_cameras(rng: np.random.Generator, res: int, n_viewers: int, ipd: float = 0.064,
                        heads=None) -> List[Camera]:
    """Left+right eye cameras of `n_viewers` local viewers, each head drawn
    uniformly over the paper's viewing range (lateral +-0.4 m, depth
    1.25 +- 0.15 m from the display, eyes level with the display centre,
    6.4 cm apart), mapped into the remote capture frame.  `heads` (n, 3)
    overrides the draw."""
    if heads is None:
        heads = np.stack([rng.uniform(-VIEWER_LATERAL, VIEWER_LATERAL, n_viewers), np.zeros(n_viewers),
                          DISPLAY_DISTANCE + rng.uniform(-VIEWER_DEPTH, VIEWER_DEPTH, n_viewers)], 1)
    cams = []
    for h in np.asarray(heads, np.float64):
        for side in (-0.5, 0.5):
            cams.append(display_eye_camera(h + np.array([side * ipd, 0.0, 0.0]), res))
    return cams


def scene_paper_rig(seed: int = 3, res: int = 1024, C: int = 32, n_viewers: int = 1,
                    target_res: Optional[int] = None) -> Scene:
    """The paper's lifting setup: Gaussians from three of the four capture
    views only -- the upper-left camera of the narrow pair (cam0) and both
    cameras of the wide pair (cam2, cam3) -- with the precision scene's map
    generators (50% ellipse, ~1.58M Gaussians at 1024^2, BF16 features);
    targets are display-mapped eye pairs of `n_viewers` viewers."""
    rng = np.random.default_rng(seed)
    f = float(res)
    four = _rig_four(res, f)
    cams = [four[0], four[2], four[3]]
    targets = display_eye_cameras(np.random.default_rng([seed, 1]), target_res or res, n_viewers)
    return _scene_from_rig(f"rig3-3x{res}-c{C}-bf16", cams, rng, C, FEAT_BF16,
                           (0.42, 0.379), 10.0, targets, seed)


def scene_frame(frame_id: int, res: int = 1024, C: int = 32) -> Scene:
    """Serving frame: the four-view precision scene regenerated with
    seed = frame id."""
    sc = scene_precision(seed=1000 + frame_id, res=res, C=C)
    sc.name = f"frame{frame_id}-4x{res}-c{C}-bf16"
    return sc


# --------------------------------------------------------------------------
# direct Gaussian sets (for tests of the render path on its own)
# --------------------------------------------------------------------------

@dataclass
class GaussianSet:
    mean: np.ndarray   # (N,3) f32
    cov: np.ndarray    # (N,6) f32: s00 s01 s02 s11 s12 s22
    opac: np.ndarray   # (N,)  f32
    feat: np.ndarray   # (N,C) f32


def random_gaussians(seed: int, n: int, C: int, center=(0, 0, 1.5), spread=0.5,
                     sigma_range=(0.002, 0.02)) -> GaussianSet:
    """Isotropic-ish random Gaussians in a box in front of the origin."""
    rng = np.random.default_rng(seed)
    mean = np.asarray(center) + rng.uniform(-spread, spread, size=(n, 3))
    sig = rng.uniform(*sigma_range, size=(n, 3))
    A = rng.normal(size=(n, 3, 3)) * 0.3 + np.eye(3)[None]
    M = A * sig[:, None, :]
    S = M @ np.transpose(M, (0, 2, 1))
    cov = np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)
    opac = rng.uniform(0.3, 0.95, size=n)
    feat = rng.standard_normal(size=(n, C))
    return GaussianSet(mean.astype(np.float32), cov.astype(np.float32),
                       opac.astype(np.float32), feat.astype(np.float32))


WORKLOADS = {
    "tiny": scene_tiny,
    "paper": scene_paper,
    "precision": scene_precision,
    "rig3": scene_paper_rig,
}
