"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these retype the oracle's own formulas: each checks it against an
independent fact -- a closed form, an invariant, a library routine doing a
different computation (eigen-decomposition, quaternion rotation, stable
argsort, BF16 conversion), numerical differentiation, or brute force.

Paper passages: Sec. 4.2 (lifting of foreground pixels with the camera;
Gaussian record = position, latent feature, scale, opacity; render
F = R_G({G}, Pi_novel) with the cited differentiable 3DGS rasterizer).
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2405_14866_gb300 import gen

PAR = O.params_array()


def _cam(f=64.0, W=64, H=64, cx=None, cy=None, center=(0, 0, 0), Rc2w=np.eye(3)):
    return gen.make_camera(f, W, H, center, Rc2w, cx=cx, cy=cy)


def _gset(mean, cov, opac, feat):
    return O.Gaussians(np.asarray(mean, np.float32).reshape(-1, 3), np.asarray(cov, np.float32).reshape(-1, 6),
                       np.asarray(opac, np.float32).reshape(-1), np.asarray(feat, np.float32).reshape(len(opac), -1))


def _bins_single_tile(order, n_tiles_total=1):
    """Bins with every listed Gaussian in tile 0, in the given order."""
    order = np.asarray(order, np.uint32)
    ranges = np.zeros((n_tiles_total, 2), np.uint32)
    ranges[0] = [0, len(order)]
    return O.Bins(np.zeros(len(order), np.int64), len(order), np.zeros(len(order), np.uint64), order, ranges, 1, 1)


# ---------------------------------------------------------------------------
# BF16 storage
# ---------------------------------------------------------------------------

def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, -0.0, 1e-30, 3e38], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = O.round_bf16(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


# ---------------------------------------------------------------------------
# lifting (Sec. 4.2: unproject foreground pixels with Pi)
# ---------------------------------------------------------------------------

def _small_rig_view(seed=3, res=32, quat_deg=10.0):
    rng = np.random.default_rng(seed)
    cam = gen.make_camera(40.0, res, res, (0.13, -0.07, 0.02), Rotation.from_euler("xyz", [7, -11, 4], degrees=True).as_matrix())
    depth = 0.8 + 0.8 * gen.value_noise(rng, res, res)
    mask = gen.ellipse_mask(res, res, 0.45, 0.425)
    return gen._view_maps(rng, cam, depth, mask, 5, isotropic=False, quat_deg=quat_deg)


def test_lift_reprojects_to_source_pixel():
    """Re-projecting each lifted mean with its own source camera returns the
    pixel centre and the depth (the inverse of the unprojection).  The
    camera's rotation is stored in FP32, so it is orthonormal only to
    ~1e-7: that bounds the tolerance."""
    v = _small_rig_view()
    g = O.lift_view(v, "f64")
    vv, uu = np.nonzero(v.mask)
    R = v.cam.R.astype(np.float64)
    t = v.cam.t.astype(np.float64)
    p = g.mean @ R.T + t
    u = v.cam.fx * p[:, 0] / p[:, 2] + v.cam.cx
    w = v.cam.fy * p[:, 1] / p[:, 2] + v.cam.cy
    assert np.allclose(u, uu, atol=1e-5)
    assert np.allclose(w, vv, atol=1e-5)
    assert np.allclose(p[:, 2], v.depth[vv, uu], rtol=1e-6)
    assert np.array_equal(g.opac, v.opacity[vv, uu].astype(np.float64))
    assert np.array_equal(g.feat, v.feat[vv, uu].astype(np.float64))


def test_lift_anisotropic_intrinsics_and_unnormalised_quaternion():
    """With fx != fy and cx != cy, both precisions re-project every lifted
    mean to its pixel centre.  The Gaussian's rotation is that of the
    normalised quaternion: scaling q by 2.5 leaves Sigma3D unchanged."""
    v = _small_rig_view(quat_deg=25.0)
    v.cam = gen.Camera(44.0, 37.0, 14.2, 17.9, v.cam.width, v.cam.height, v.cam.R, v.cam.t)
    vv, uu = np.nonzero(v.mask)
    R = v.cam.R.astype(np.float64)
    t = v.cam.t.astype(np.float64)
    for prec, tol in (("f64", 1e-5), ("f32", 2e-4)):
        g = O.lift_view(v, prec)
        p = g.mean.astype(np.float64) @ R.T + t
        assert np.allclose(v.cam.fx * p[:, 0] / p[:, 2] + v.cam.cx, uu, atol=tol), prec
        assert np.allclose(v.cam.fy * p[:, 1] / p[:, 2] + v.cam.cy, vv, atol=tol), prec
        v2 = gen.SourceView(v.depth, v.mask, v.scale, (v.quat * 2.5).astype(np.float32), v.opacity, v.feat, v.cam)
        g2 = O.lift_view(v2, prec)
        scale = np.abs(g.cov[:, [0, 3, 5]]).max()
        assert np.abs(g2.cov.astype(np.float64) - g.cov).max() <= 2e-6 * scale, prec


def test_lift_covariance_axes_and_scales():
    """Sigma3D has eigenvalues s_i^2 along the world axes R_src^T R(q) e_i
    (quaternion rotation evaluated by scipy, an independent routine)."""
    v = _small_rig_view(quat_deg=40.0)
    g = O.lift_view(v, "f64")
    vv, uu = np.nonzero(v.mask)
    q = v.quat[vv, uu].astype(np.float64)
    s = v.scale[vv, uu].astype(np.float64)
    Rq = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()     # scipy order x,y,z,w
    axes = np.einsum("ji,njk->nik", v.cam.R.astype(np.float64), Rq)  # R_src^T R(q)
    c = g.cov
    S = np.stack([np.stack([c[:, 0], c[:, 1], c[:, 2]], 1), np.stack([c[:, 1], c[:, 3], c[:, 4]], 1),
                  np.stack([c[:, 2], c[:, 4], c[:, 5]], 1)], 1)
    for i in range(3):
        a = axes[:, :, i]
        Sa = np.einsum("nij,nj->ni", S, a)
        err = np.abs(Sa - (s[:, i] ** 2)[:, None] * a).max(1)
        assert (err <= 1e-6 * (s ** 2).max(1)).all()     # FP32 camera rotation: ~1e-7
    ev = np.sort(np.linalg.eigvalsh(S), axis=1)
    assert (np.abs(ev - np.sort(s ** 2, axis=1)).max(1) <= 1e-6 * (s ** 2).max(1)).all()


def test_lift_identity_rotation_isotropic_scale():
    """With q = identity (the paper's setting), an axis-aligned source camera
    and isotropic scale, Sigma3D = s^2 I exactly (also in single precision)."""
    sc = gen.scene_tiny()
    v = sc.views[0]
    for prec in ("f64", "f32"):
        g = O.lift_view(v, prec)
        s = v.scale.reshape(-1, 3)[:, 0].astype(np.float64 if prec == "f64" else np.float32)
        assert np.array_equal(g.cov[:, 0], s * s)
        assert np.array_equal(g.cov[:, 3], s * s)
        assert np.array_equal(g.cov[:, 5], s * s)
        assert not g.cov[:, [1, 2, 4]].any()


def test_lift_single_precision_close_to_double():
    v = _small_rig_view()
    g64 = O.lift_view(v, "f64")
    g32 = O.lift_view(v, "f32")
    assert np.allclose(g32.mean, g64.mean, rtol=2e-6, atol=1e-7)
    scale = np.abs(g64.cov[:, [0, 3, 5]]).max(1, keepdims=True)
    assert np.abs(g32.cov - g64.cov).max() <= 1e-5 * scale.max()


def test_key_mode_has_no_fused_multiply_add():
    """Compile-flag check of the key mode (not a pin of the method): an
    input where a fused multiply-add changes the projected mean.
    p_x = R00 x + R01 y with R00 x = 1 + 2^-11 + 2^-24 (inexact in FP32) and
    R01 y = -(1 + 2^-11): two roundings give p_x = 0, a fused one 2^-24."""
    e12, e11 = np.float32(1 + 2 ** -12), np.float32(1 + 2 ** -11)
    cam = _cam(f=64.0, cx=0.0, cy=32.0)
    cam.R = np.array([[e12, -1, 0], [0, 0, 0], [0, 0, 1]], np.float32)
    cam.t = np.zeros(3, np.float32)
    g = _gset([[e12, e11, 1.0]], [[1e-4, 0, 0, 1e-4, 0, 1e-4]], [0.5], [[1.0]])
    pr = O.project_f32(g, cam, PAR)
    two = np.float32(np.float32(e12 * e12) - e11)
    fused = np.float32(np.float64(e12) * np.float64(e12) - np.float64(e11))
    assert two == 0.0 and fused != 0.0
    assert pr.ntiles[0] > 0
    assert pr.mu[0, 0] == 0.0


# ---------------------------------------------------------------------------
# EWA projection
# ---------------------------------------------------------------------------

def test_projection_on_axis_isotropic_closed_form():
    """On the optical axis J = diag(f/z, f/z): Sigma2D = ((f s / z)^2 + lowpass) I."""
    f, z, s = 64.0, 1.7, 0.013
    cam = _cam(f=f, cx=32.0, cy=32.0)
    g = _gset([[0, 0, z]], [[s * s, 0, 0, s * s, 0, s * s]], [0.5], [[1.0]]).astype(np.float64)
    mu, conic, depth, vis = O.project_f64(g, cam, PAR)
    sig2 = (f * s / z) ** 2 + O.LOWPASS
    assert vis[0]
    assert np.allclose(mu[0], [32.0, 32.0], atol=1e-12)
    assert np.allclose(conic[0], [1 / sig2, 0, 1 / sig2], rtol=1e-6, atol=1e-12)
    assert depth[0] == pytest.approx(z, rel=1e-7)


def _proj_map(cam, x):
    p = cam.R.astype(np.float64) @ x + cam.t.astype(np.float64)
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def test_projection_matches_numerical_jacobian():
    """Sigma2D = (dg/dx) Sigma3D (dg/dx)^T + lowpass I with g the pinhole
    map world -> pixels, differentiated numerically (inside the clamp)."""
    rng = np.random.default_rng(5)
    cam = _cam(f=500.0, W=640, H=480, center=(0.1, -0.05, -0.2),
               Rc2w=Rotation.from_euler("xyz", [6, -9, 3], degrees=True).as_matrix())
    gs = gen.random_gaussians(11, 40, 2, center=(0.0, 0.0, 1.5), spread=0.3)
    g = O.Gaussians(gs.mean.astype(np.float64), gs.cov.astype(np.float64), gs.opac.astype(np.float64), gs.feat.astype(np.float64))
    mu, conic, depth, vis = O.project_f64(g, cam, PAR)
    for i in range(g.n):
        x = g.mean[i]
        J = np.zeros((2, 3))
        for k in range(3):
            h = 1e-5
            e = np.zeros(3); e[k] = h
            J[:, k] = (_proj_map(cam, x + e) - _proj_map(cam, x - e)) / (2 * h)
        c = g.cov[i]
        S3 = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        S2 = J @ S3 @ J.T + O.LOWPASS * np.eye(2)
        a, b, cc = conic[i]
        inv = np.linalg.inv(np.array([[a, b], [b, cc]]))
        assert vis[i]
        assert np.allclose(inv, S2, rtol=1e-6, atol=1e-9)
        assert np.allclose(mu[i], _proj_map(cam, x), rtol=0, atol=1e-9)


def test_key_mode_projection_matches_numerical_jacobian():
    """The single-precision key mode against the same numerical Jacobian,
    at single-precision tolerance (principal point with cx != cy)."""
    cam = _cam(f=500.0, W=640, H=480, center=(-0.08, 0.04, -0.1),
               Rc2w=Rotation.from_euler("xyz", [-4, 8, 12], degrees=True).as_matrix())
    gs = gen.random_gaussians(12, 60, 1, center=(0.0, 0.0, 1.4), spread=0.3)
    g32 = O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat)
    pr = O.project_f32(g32, cam, PAR)
    assert (pr.ntiles > 0).all()
    for i in range(g32.n):
        x = g32.mean[i].astype(np.float64)
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-5
            J[:, k] = (_proj_map(cam, x + e) - _proj_map(cam, x - e)) / 2e-5
        c = g32.cov[i].astype(np.float64)
        S3 = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        S2 = J @ S3 @ J.T + O.LOWPASS * np.eye(2)
        a, b, cc = pr.conic[i].astype(np.float64)
        assert np.allclose(np.linalg.inv([[a, b], [b, cc]]), S2, rtol=2e-5, atol=1e-6)
        assert np.allclose(pr.mu[i], _proj_map(cam, x), rtol=0, atol=2e-4)
        p = cam.R.astype(np.float64) @ x + cam.t
        assert abs(float(pr.dkey[i].view(np.float32)) - p[2]) <= 1e-6 * p[2]


def test_key_mode_projection_anisotropic_intrinsics():
    """Key mode with fx != fy, W != H and the principal point off centre,
    against the numerical Jacobian of the pinhole map (inside the clamp) and
    the projected mean, at single-precision tolerance."""
    base = _cam(f=500.0, W=640, H=360, center=(0.05, -0.03, -0.1),
                Rc2w=Rotation.from_euler("xyz", [5, -7, 10], degrees=True).as_matrix())
    cam = gen.Camera(520.0, 410.0, 300.0, 170.0, 640, 360, base.R, base.t)
    gs = gen.random_gaussians(13, 60, 1, center=(0.0, 0.0, 1.4), spread=0.25)
    g32 = O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat)
    pr = O.project_f32(g32, cam, PAR)
    assert (pr.ntiles > 0).all()
    for i in range(g32.n):
        x = g32.mean[i].astype(np.float64)
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-5
            J[:, k] = (_proj_map(cam, x + e) - _proj_map(cam, x - e)) / 2e-5
        c = g32.cov[i].astype(np.float64)
        S3 = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        S2 = J @ S3 @ J.T + O.LOWPASS * np.eye(2)
        a, b, cc = pr.conic[i].astype(np.float64)
        assert np.allclose(np.linalg.inv([[a, b], [b, cc]]), S2, rtol=2e-5, atol=1e-6)
        assert np.allclose(pr.mu[i], _proj_map(cam, x), rtol=0, atol=2e-4)


def test_key_mode_clamped_jacobian_on_every_side():
    """Key mode, fx != fy, W != H: beyond +-1.3 tan(fov/2) on either side
    of either axis (1.3 * 0.5 W / fx in x, 1.3 * 0.5 H / fy in y) the
    Jacobian is the pinhole map's at the clamped direction.  Large
    footprints keep the Gaussians' rects inside the image."""
    fx, fy, W, H = 90.0, 130.0, 200, 120
    cam = gen.Camera(fx, fy, 100.0, 60.0, W, H, np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    limx, limy = 1.3 * 0.5 * W / fx, 1.3 * 0.5 * H / fy
    z = 2.0
    cov = np.array([0.6, 0.05, -0.03, 0.5, 0.02, 0.4])
    S3 = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])

    def pin(p):
        return np.array([fx * p[0] / p[2], fy * p[1] / p[2]])

    for sx, sy in [(1.6, 0.1), (-1.6, 0.1), (0.1, 1.6), (0.1, -1.6), (-1.5, -1.5), (1.5, 1.5)]:
        x = np.array([sx * limx * z, sy * limy * z, z], np.float32)
        g = _gset([x], [cov], [0.5], [[1.0]])
        pr = O.project_f32(g, cam, PAR)
        assert pr.ntiles[0] > 0
        p = x.astype(np.float64)
        pc = np.array([np.clip(p[0] / z, -limx, limx) * z, np.clip(p[1] / z, -limy, limy) * z, z])
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            J[:, k] = (pin(pc + e) - pin(pc - e)) / 2e-6
        S2 = J @ S3 @ J.T + O.LOWPASS * np.eye(2)
        a, b, c = pr.conic[0].astype(np.float64)
        assert np.allclose(np.linalg.inv([[a, b], [b, c]]), S2, rtol=5e-5), (sx, sy)
        assert np.allclose(pr.mu[0], pin(p) + [100.0, 60.0], rtol=1e-6), (sx, sy)


def test_projection_clamped_jacobian_far_off_axis():
    """Outside +-1.3 tan(fov/2) the Jacobian is evaluated at the clamped
    direction: compare with a numerical Jacobian of the pinhole map taken at
    the clamped camera-space point."""
    f, W = 100.0, 200
    cam = _cam(f=f, W=W, H=W)
    lim = 1.3 * (0.5 * W / f)
    z = 2.0
    x = np.array([3.0 * lim * z, -2.0 * lim * z, z])        # far outside in x and y
    cov = np.array([4e-4, 1e-4, -5e-5, 3e-4, 2e-5, 5e-4])
    g = O.Gaussians(x[None], cov[None], np.array([0.5]), np.ones((1, 1)))
    mu, conic, depth, vis = O.project_f64(g, cam, PAR)
    pc = np.array([lim * z, -lim * z, z])
    def pin(p):
        return np.array([f * p[0] / p[2], f * p[1] / p[2]])
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-6
        J[:, k] = (pin(pc + e) - pin(pc - e)) / 2e-6
    S3 = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])
    S2 = J @ S3 @ J.T + O.LOWPASS * np.eye(2)
    a, b, c = conic[0]
    assert np.allclose(np.linalg.inv([[a, b], [b, c]]), S2, rtol=1e-6)


def test_radius_is_three_sigma_of_major_axis():
    """r = ceil(3 sqrt(lambda_max)); lambda_max from numpy's eigvalsh of the
    inverse conic, where the 0.1 floor of the discriminant is inactive."""
    cam = _cam(f=500.0, W=640, H=480)
    gs = gen.random_gaussians(2, 400, 1, center=(0, 0, 1.2), spread=0.2, sigma_range=(0.001, 0.03))
    g32 = O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat)
    pr = O.project_f32(g32, cam, PAR)
    checked = 0
    for i in np.nonzero(pr.ntiles)[0]:
        a, b, c = pr.conic[i].astype(np.float64)
        S = np.linalg.inv([[a, b], [b, c]])
        ev = np.linalg.eigvalsh(S)
        if (ev[1] - ev[0]) ** 2 / 4 < 0.2:        # discriminant floor may be active
            continue
        r = 3 * math.sqrt(ev[1])
        if abs(r - round(r)) < 1e-3:              # too close to an integer to decide
            continue
        assert pr.radius[i] == math.ceil(r), (i, r, pr.radius[i])
        checked += 1
    assert checked > 100


def test_rect_hand_examples():
    """Tile rect = [floor((mu - r)/16), floor((mu + r + 15)/16)) clamped to
    the grid, on hand-worked cases.  A vanishing 3D footprint leaves
    Sigma2D = lowpass I = 0.3 I, so lambda_max = 0.3 + sqrt(0.1) (the floor
    of the discriminant) and r = ceil(3 * 0.7850) = 3."""
    f, z = 100.0, 2.0
    cam = _cam(f=f, W=160, H=160, cx=0.0, cy=0.0)   # principal point at the corner
    s = 1e-6 * z / f
    cov = [s * s, 0, 0, s * s, 0, s * s]
    cases = [  # (mu_x, mu_y) -> rect (x0, y0, x1, y1)
        ((40.25, 40.25), (2, 2, 3, 3)),     # 37.25/16 -> 2 ; 58.25/16 -> 3
        ((40.25, 2.5), (2, 0, 3, 1)),       # y: -0.5/16 -> -1 -> 0 ; 20.5/16 -> 1
        ((79.0, 150.0), (4, 9, 6, 10)),     # x: 76/16 -> 4, 97/16 -> 6 ; y: 147/16 -> 9, 168/16 -> 10
        ((47.0, 15.9), (2, 0, 4, 2)),       # x: 44/16 -> 2, 65/16 -> 4 ; y: 12.9/16 -> 0, 33.9/16 -> 2
        ((77.5, 40.25), (4, 2, 5, 3)),      # x: 74.5/16 -> 4, 95.5/16 -> 5 (just below a boundary)
        ((40.25, 51.0), (2, 3, 3, 4)),      # y: 48/16 = 3 exactly -> 3 ; 69/16 -> 4
        ((51.0, 40.25), (3, 2, 4, 3)),      # x: 48/16 = 3 exactly -> 3 ; 69/16 -> 4
    ]
    # a non-square grid (13 x 6 tiles), rects clamped at the right and bottom
    cam2 = _cam(f=f, W=200, H=96, cx=0.0, cy=0.0)
    cases2 = [
        ((198.0, 94.0), (12, 5, 13, 6)),    # x: 195/16 -> 12, 216/16 -> 13 ; y: 91/16 -> 5, 112/16 -> 7 -> 6
        ((150.0, 94.0), (9, 5, 10, 6)),     # x: 147/16 -> 9, 168/16 -> 10
    ]
    for c_, cs in ((cam, cases), (cam2, cases2)):
        for (mx, my), rect in cs:
            g = _gset([[mx * z / f, my * z / f, z]], [cov], [0.5], [[1.0]])
            pr = O.project_f32(g, c_, PAR)
            assert pr.radius[0] == 3
            assert tuple(pr.rect[0]) == rect, ((mx, my), pr.rect[0], pr.mu[0])
            assert pr.ntiles[0] == (rect[2] - rect[0]) * (rect[3] - rect[1])


def test_depth_key_orders_like_depth_and_culling():
    cam = _cam(f=64.0, cx=32, cy=32)
    # visible iff z_near < z < z_far (open interval): 8 sits on z_near, 9 on
    # z_far, 10 just above z_near
    z_near, z_far = np.float32(cam.z_near), np.float32(cam.z_far)
    zs = np.array([0.5, 3.0, 1.0, 0.15, 1.0, 2.0, np.nan, 0.9, z_near, z_far,
                   np.nextafter(z_near, np.float32(1))], np.float32)
    xs = np.zeros_like(zs); xs[5] = 100.0            # index 5 projects far off screen
    mean = np.stack([xs, np.zeros_like(zs), zs], 1)
    cov = np.tile([1e-4, 0, 0, 1e-4, 0, 1e-4], (len(zs), 1))
    cov[7] = 0.0                                      # degenerate: with lowpass 0 det = 0
    g = _gset(mean, cov, np.full(len(zs), 0.5), np.ones((len(zs), 1)))
    par0 = O.params_array(lowpass=0.0)
    pr = O.project_f32(g, cam, par0)
    culled = {3, 5, 6, 7, 8, 9}
    for i in range(len(zs)):
        if i in culled:
            assert pr.ntiles[i] == 0 and pr.dkey[i] == 0xFFFFFFFF
        else:
            assert pr.ntiles[i] > 0 and pr.dkey[i] == np.float32(zs[i]).view(np.uint32)
    vis = [i for i in range(len(zs)) if i not in culled]
    by_key = sorted(vis, key=lambda i: (pr.dkey[i], i))
    by_depth = sorted(vis, key=lambda i: (float(zs[i]), i))
    assert by_key == by_depth


# ---------------------------------------------------------------------------
# binning: count, scan, emit, sort, ranges
# ---------------------------------------------------------------------------

def _tiny_projected():
    sc = gen.scene_tiny()
    g32 = O.lift_scene(sc, "f32")
    cam = sc.targets[0]
    return g32, cam, O.project_f32(g32, cam, PAR)


def test_sort_matches_numpy_stable_argsort():
    g32, cam, pr = _tiny_projected()
    keys, vals = O.emit_unsorted(pr, cam.width, cam.height)
    b = O.bin_gaussians(pr, cam.width, cam.height)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(b.keys, keys[order])
    assert np.array_equal(b.ids, vals[order])
    assert b.P == int(pr.ntiles.sum())


def test_tile_lists_match_bruteforce():
    g32, cam, pr = _tiny_projected()
    b = O.bin_gaussians(pr, cam.width, cam.height)
    for t in range(b.tiles_x * b.tiles_y):
        s, e = b.ranges[t]
        bf = O.tile_list_bruteforce(pr, t % b.tiles_x, t // b.tiles_x)
        assert np.array_equal(b.ids[s:e], bf), t
    assert int((b.ranges[:, 1] - b.ranges[:, 0]).sum()) == b.P


def test_tile_lists_match_bruteforce_rotated_subcase():
    """A 256x256 render of a two-view rig (4 x 4 ... 16 x 16 tiles)."""
    sc = gen.scene_paper(seed=7, res=96, C=2)
    g32 = O.lift_scene(sc, "f32")
    cam = gen.make_camera(240.0, 256, 256, (0.02, 0.01, -0.05), gen.rot_y(3.0))
    pr = O.project_f32(g32, cam, PAR)
    b = O.bin_gaussians(pr, 256, 256)
    assert b.P > 1000
    for t in range(0, b.tiles_x * b.tiles_y, 7):
        s, e = b.ranges[t]
        assert np.array_equal(b.ids[s:e], O.tile_list_bruteforce(pr, t % b.tiles_x, t // b.tiles_x)), t


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def test_single_isotropic_gaussian_closed_form():
    """F(p) = f min(alpha_max, o exp(-|p-mu|^2 / (2 sigma^2))) inside the
    rect's tiles where that is >= alpha_min, else 0; sigma^2 = (f s/z)^2 + lowpass."""
    f, z, s, o = 64.0, 1.3, 0.05, 0.8
    cam = _cam(f=f, cx=32.0, cy=32.0)
    fv = np.array([1.5, -0.25])
    g = _gset([[0, 0, z]], [[s * s, 0, 0, s * s, 0, s * s]], [o], [fv])
    r = O.render(g, cam, PAR)
    sig2 = (f * s / z) ** 2 + O.LOWPASS
    yy, xx = np.mgrid[0:64, 0:64].astype(np.float64)
    a = o * np.exp(-((xx - 32) ** 2 + (yy - 32) ** 2) / (2 * sig2))
    a = np.minimum(a, O.ALPHA_MAX)
    x0, y0, x1, y1 = r.proj.rect[0]
    inrect = (xx // 16 >= x0) & (xx // 16 < x1) & (yy // 16 >= y0) & (yy // 16 < y1)
    keep = inrect & (a >= O.ALPHA_MIN)
    near = np.abs(a - O.ALPHA_MIN) < 1e-5
    exp = np.where(keep, a, 0.0)
    ok = ~near
    assert keep.sum() > 50
    assert np.allclose(r.comp.A[ok], exp[ok], rtol=1e-6, atol=1e-12)
    for c in range(2):
        assert np.allclose(r.comp.F[c][ok], fv[c] * exp[ok], rtol=1e-6, atol=1e-12)


def test_three_gaussians_hand_worked():
    """Three Gaussians over one pixel centre with alpha = 0.5 each, listed
    front to back: F = 0.5 f1 + 0.25 f2 + 0.125 f3, A = 0.875."""
    mu = np.zeros((3, 2))
    conic = np.tile([1.0, 0.0, 1.0], (3, 1))
    opac = np.array([0.5, 0.5, 0.5])
    feat = np.array([[1.0, 2.0], [10.0, -4.0], [100.0, 8.0]])
    bins = _bins_single_tile([0, 1, 2])
    r = O.composite(mu, conic, opac, feat, 1, 1, bins, PAR)
    assert np.allclose(r.F[:, 0, 0], [0.5 * 1 + 0.25 * 10 + 0.125 * 100, 0.5 * 2 - 0.25 * 4 + 0.125 * 8])
    assert r.A[0, 0] == pytest.approx(0.875)
    assert r.last[0, 0] == 3


def test_transmittance_stop_rule_hand_worked():
    """alpha = 0.95 four times: T = 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4
    stops before the fourth, which is not blended."""
    mu = np.zeros((4, 2))
    conic = np.tile([1.0, 0.0, 1.0], (4, 1))
    opac = np.full(4, 0.95)
    feat = np.array([[1.0], [2.0], [3.0], [1000.0]])
    r = O.composite(mu, conic, opac, feat, 1, 1, _bins_single_tile([0, 1, 2, 3]), PAR)
    assert r.F[0, 0, 0] == pytest.approx(0.95 * 1 + 0.95 * 0.05 * 2 + 0.95 * 0.0025 * 3)
    assert r.T[0, 0] == pytest.approx(1.25e-4)
    assert r.last[0, 0] == 3


def test_opaque_front_occludes():
    """alpha_max = 0.99 clamps a fully opaque front Gaussian: pixels it covers
    at its centre show F = 0.99 f_front + 0.01 alpha_back f_back.  With
    alpha_max = 1 the front Gaussian alone would leave T = 0 < t_min, so the
    stop rule discards it and everything behind (F = 0)."""
    mu = np.zeros((2, 2))
    conic = np.tile([1e-4, 0.0, 1e-4], (2, 1))     # sigma = 100 px: alpha ~ o at the centre
    opac = np.array([1.0, 0.6])
    feat = np.array([[3.0], [7.0]])
    r = O.composite(mu, conic, opac, feat, 1, 1, _bins_single_tile([0, 1]), PAR)
    am = float(np.float32(0.99))             # alpha_max as passed (FP32 parameter)
    a_back = 0.6 * math.exp(-0.0)
    assert r.F[0, 0, 0] == pytest.approx(am * 3 + (1 - am) * a_back * 7, rel=1e-12)
    r1 = O.composite(mu, conic, opac, feat, 1, 1, _bins_single_tile([0, 1]), O.params_array(alpha_max=1.0))
    assert r1.F[0, 0, 0] == 0.0 and r1.A[0, 0] == 0.0 and r1.last[0, 0] == 0


def test_weights_plus_transmittance_is_one():
    """sum_j alpha_j T_j + T_final = 1 (telescoping), via unit features."""
    g32, cam, _ = _tiny_projected()
    g1 = O.Gaussians(g32.mean, g32.cov, g32.opac, np.ones((g32.n, 1), np.float32))
    r = O.render(g1, cam, PAR)
    assert np.allclose(r.comp.F[0] + r.comp.T, 1.0, atol=1e-12)
    assert np.allclose(r.comp.A, 1.0 - r.comp.T, atol=0)


def test_constant_features_and_linearity():
    g32, cam, _ = _tiny_projected()
    c = np.array([0.5, -2.0, 3.25], np.float32)
    gc = O.Gaussians(g32.mean, g32.cov, g32.opac, np.tile(c, (g32.n, 1)))
    r = O.render(gc, cam, PAR)
    for k in range(3):
        assert np.allclose(r.comp.F[k], c[k] * r.comp.A, atol=1e-12)
    rng = np.random.default_rng(1)
    f1 = rng.standard_normal((g32.n, 2)).astype(np.float32)
    f2 = rng.standard_normal((g32.n, 2)).astype(np.float32)
    rs = [O.render(O.Gaussians(g32.mean, g32.cov, g32.opac, f), cam, PAR) for f in (f1, f2, f1 + f2)]
    # f1 + f2 in float32 is rounded; compare with the FP64 sum of the parts
    assert np.allclose(rs[2].comp.F, rs[0].comp.F + rs[1].comp.F, atol=1e-6)


def test_identity_camera_reproduces_source_features():
    """Target = source camera, footprint 0.05 px, lowpass 0, opacity 1: each
    pixel sees only its own Gaussian, clamped to alpha_max: F = 0.99 f_self.
    Tile lists from brute force, not from the scan/sort path."""
    sc = gen.scene_tiny()
    v = sc.views[0]
    v2 = gen.SourceView(v.depth, v.mask, (v.depth / v.cam.fx * 0.05)[..., None].repeat(3, 2).astype(np.float32),
                        v.quat, np.ones_like(v.opacity), v.feat, v.cam)
    g32 = O.lift_view(v2, "f32")
    par = O.params_array(lowpass=0.0)
    pr = O.project_f32(g32, v.cam, par)
    tx, ty = O.tile_grid(64, 64)
    ids, ranges = [], np.zeros((tx * ty, 2), np.uint32)
    for t in range(tx * ty):
        lst = O.tile_list_bruteforce(pr, t % tx, t // tx)
        ranges[t] = [sum(len(l) for l in ids), sum(len(l) for l in ids) + len(lst)]
        ids.append(lst)
    ids = np.concatenate(ids)
    bins = O.Bins(np.zeros(g32.n, np.int64), len(ids), np.zeros(len(ids), np.uint64), ids, ranges, tx, ty)
    r = O.composite(pr.mu.astype(np.float64), pr.conic.astype(np.float64), g32.opac.astype(np.float64),
                    g32.feat.astype(np.float64), 64, 64, bins, par)
    expect = 0.99 * np.transpose(v.feat, (2, 0, 1)).astype(np.float64)
    assert np.allclose(r.F, expect, rtol=1e-6, atol=1e-9)
    assert np.allclose(r.A, 0.99)


def test_tiled_composite_matches_bruteforce_lists():
    g32, cam, pr = _tiny_projected()
    b = O.bin_gaussians(pr, cam.width, cam.height)
    r = O.composite(pr.mu.astype(np.float64), pr.conic.astype(np.float64), g32.opac.astype(np.float64),
                    g32.feat.astype(np.float64), cam.width, cam.height, b, PAR)
    ids, ranges = [], np.zeros_like(b.ranges)
    acc = 0
    for t in range(b.tiles_x * b.tiles_y):
        lst = O.tile_list_bruteforce(pr, t % b.tiles_x, t // b.tiles_x)
        ranges[t] = [acc, acc + len(lst)]
        acc += len(lst)
        ids.append(lst)
    bb = O.Bins(b.offsets, acc, b.keys, np.concatenate(ids), ranges, b.tiles_x, b.tiles_y)
    r2 = O.composite(pr.mu.astype(np.float64), pr.conic.astype(np.float64), g32.opac.astype(np.float64),
                     g32.feat.astype(np.float64), cam.width, cam.height, bb, PAR)
    assert np.array_equal(r.F, r2.F) and np.array_equal(r.T, r2.T) and np.array_equal(r.last, r2.last)


def test_pixel_alternatives_flip_one_decision():
    """A pixel whose only ambiguous decision is the alpha threshold has one
    alternative: the output with that Gaussian blended / not blended."""
    mu = np.zeros((2, 2))
    conic = np.tile([1.0, 0.0, 1.0], (2, 1))
    opac = np.array([O.ALPHA_MIN * (1 + 1e-6), 0.5])      # alpha ~ alpha_min: ambiguous
    feat = np.array([[4.0], [1.0]])
    bins = _bins_single_tile([0, 1])
    r = O.composite(mu, conic, opac, feat, 1, 1, bins, PAR)
    assert r.flags[0, 0] == 1
    alts = O.pixel_alternatives(mu, conic, opac, feat, 1, 1, bins, 0, 0, PAR)
    a0 = opac[0]
    assert r.F[0, 0, 0] == pytest.approx(4 * a0 + 1 * 0.5 * (1 - a0))
    assert alts.shape == (1, 2)
    assert alts[0, 0] == pytest.approx(0.5) and alts[0, 1] == pytest.approx(0.5)


def test_threshold_equalities_and_the_stop_alternative():
    """The rules are strict: only alpha < alpha_min skips and only
    T' < t_min stops, so equality blends.  Both equalities are ambiguous
    decisions; the alternative of the stop decision stops before the
    Gaussian.  All values are exact in binary: at the centres q = 0, so
    alpha = o; 0.75 then 0.5 leave T' = 0.25 * 0.5 = 0.125 = t_min."""
    mu = np.zeros((2, 2))
    conic = np.tile([1.0, 0.0, 1.0], (2, 1))
    opac = np.array([0.75, 0.5])
    feat = np.array([[1.0], [3.0]])
    par = O.params_array(t_min=0.125)
    bins = _bins_single_tile([0, 1])
    r = O.composite(mu, conic, opac, feat, 1, 1, bins, par)
    assert r.F[0, 0, 0] == 0.75 * 1.0 + 0.25 * 0.5 * 3.0
    assert r.A[0, 0] == 0.875 and r.last[0, 0] == 2 and r.flags[0, 0] == 1
    alts = O.pixel_alternatives(mu, conic, opac, feat, 1, 1, bins, 0, 0, par)
    assert alts.shape == (1, 2) and alts[0, 0] == 0.75 and alts[0, 1] == 0.75   # F, A = 1 - 0.25
    # alpha = alpha_min exactly (the opacity is the FP32 parameter itself)
    amin = float(np.float32(O.ALPHA_MIN))
    r2 = O.composite(np.zeros((1, 2)), np.array([[1.0, 0.0, 1.0]]), np.array([amin]), np.array([[2.0]]), 1, 1,
                     _bins_single_tile([0]), PAR)
    assert r2.F[0, 0, 0] == 2.0 * amin and r2.last[0, 0] == 1 and r2.flags[0, 0] == 1


# ---------------------------------------------------------------------------
# adjoint (Sec. 4.2: the rasterizer is differentiated end to end)
# ---------------------------------------------------------------------------


def test_adjoint_of_a_clamped_alpha_and_of_the_stop_equality():
    """alpha clamped at alpha_max passes no gradient to the opacity, the mean
    or the conic (alpha does not depend on them there), but the feature
    still gets alpha T g; and T' = t_min exactly is blended in the backward
    as in the forward.  Single pixel at the Gaussians' centres (q = 0)."""
    mu = np.zeros((2, 2))
    conic = np.tile([1.0, 0.0, 1.0], (2, 1))
    feat = np.array([[1.0], [3.0]])
    bins = _bins_single_tile([0, 1])
    gF, gA = np.ones((1, 1, 1)), np.ones((1, 1))
    # gA = 0 here: with gA = 1 the loss would not depend on the front alpha at all
    d_mu, d_conic, d_opac, d_feat = O.backward(mu, conic, np.array([1.0, 0.5]), feat, 1, 1, bins, gF,
                                               np.zeros((1, 1)), PAR)
    am = float(np.float32(O.ALPHA_MAX))
    assert d_opac[0] == 0.0 and not d_mu[0].any() and not d_conic[0].any()
    assert d_feat[0, 0] == pytest.approx(am) and d_opac[1] != 0.0
    par = O.params_array(t_min=0.125)
    d_mu, d_conic, d_opac, d_feat = O.backward(mu, conic, np.array([0.75, 0.5]), feat, 1, 1, bins, gF, gA, par)
    assert d_feat[0, 0] == 0.75 and d_feat[1, 0] == 0.5 * 0.25

def test_adjoint_matches_central_differences_frozen():
    """Central differences (eps = 1e-3 relative) of a random linear loss of
    (F, A) with the forward's decisions frozen, against the FP64 adjoint."""
    sc = gen.scene_paper(seed=9, res=40, C=3)
    g32 = O.lift_scene(sc, "f32")
    cam = gen.make_camera(32.0, 32, 32, (0, 0, 0), np.eye(3))
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, 32, 32)
    mu = pr.mu.astype(np.float64); conic = pr.conic.astype(np.float64)
    opac = g32.opac.astype(np.float64); feat = g32.feat.astype(np.float64)
    rng = np.random.default_rng(4)
    gF = rng.standard_normal((3, 32, 32)); gA = rng.standard_normal((32, 32))
    r0, dec = O.composite(mu, conic, opac, feat, 32, 32, bins, PAR, record=True)

    def loss(mu_, conic_, opac_, feat_):
        r = O.composite(mu_, conic_, opac_, feat_, 32, 32, bins, PAR, dec_in=dec)
        return float((gF * r.F).sum() + (gA * r.A).sum())

    d_mu, d_conic, d_opac, d_feat = O.backward(mu, conic, opac, feat, 32, 32, bins, gF, gA, PAR)
    used = np.unique(bins.ids)
    pick = rng.choice(used, size=12, replace=False)
    nchk = 0
    for j in pick:
        for arr, grad, idx in ((mu, d_mu, 0), (mu, d_mu, 1), (conic, d_conic, 0), (conic, d_conic, 1),
                               (conic, d_conic, 2), (opac, d_opac, None), (feat, d_feat, 1)):
            base = [mu, conic, opac, feat]
            k = [id(b) for b in base].index(id(arr))
            def bump(sign):
                cp = [b.copy() for b in base]
                v = cp[k]
                pos = (j,) if idx is None else (j, idx)
                h = 1e-3 if k == 0 else 1e-3 * max(abs(v[pos]), 1e-2)
                v[pos] += sign * h
                return loss(*cp), h
            lp, h = bump(+1)
            lm, _ = bump(-1)
            fd = (lp - lm) / (2 * h)
            an = grad[(j,) if idx is None else (j, idx)]
            assert abs(fd - an) <= 1e-5 * max(abs(an), abs(fd), 1e-3), (j, k, idx, fd, an)
            nchk += 1
    assert nchk == 84


# ---------------------------------------------------------------------------
# point z-buffer (Sec. 4.1 z-buffers at other cameras; Sec. 4.3 fused depth)
# ---------------------------------------------------------------------------

def test_zbuffer_source_camera_returns_source_depth_map():
    """Points lifted from a depth map and z-buffered into the same camera land
    back on their own pixels: the z-buffer is the source depth map and the id
    of each pixel is its own Gaussian (every pixel is foreground here)."""
    sc = gen.scene_tiny()
    v = sc.views[0]
    g = O.lift_scene(sc, "f32")
    depth, ids = O.zbuffer(g.mean, v.cam)
    H, W = v.depth.shape
    assert np.array_equal(ids.reshape(-1), np.arange(H * W))
    assert np.array_equal(depth.view(np.uint32), np.ascontiguousarray(v.depth, np.float32).view(np.uint32))


def test_zbuffer_rotated_source_camera_roundtrip():
    """Same round trip through a rotated, translated camera: every point lands
    on its own pixel; depths agree to single-precision rounding."""
    sc = gen.scene_paper(seed=3, res=48, C=2)
    v = sc.views[0]
    g = O.lift_view(v, "f32")
    depth, ids = O.zbuffer(g.mean, v.cam)
    fg = np.argwhere(v.mask.reshape(-1) > 0)[:, 0]
    assert np.array_equal(np.sort(ids[ids >= 0]), np.arange(len(fg)))
    assert np.array_equal(np.argwhere(ids.reshape(-1) >= 0)[:, 0], fg)
    d = v.depth.reshape(-1)[fg]
    got = depth.reshape(-1)[fg]
    assert np.allclose(got, d, rtol=2e-6, atol=0)


def test_zbuffer_hand_worked():
    cam = gen.make_camera(8.0, 8, 8, (0, 0, 0), np.eye(3), cx=4.0, cy=4.0)
    pts = np.array([
        [0.0, 0.0, 2.0],        # 0: pixel (4, 4), depth 2
        [0.0, 0.0, 1.5],        # 1: same pixel, nearer: wins
        [0.125, 0.0, 1.0],      # 2: x = 8 * 0.125 + 4 = 5 -> pixel (5, 4)
        [0.125, 0.0, 1.0],      # 3: same pixel and depth: the lower id (2) stays
        [0.0, 0.0, -1.0],       # 4: behind the camera
        [1.0, 0.0, 1.0],        # 5: x = 12, outside the image
        [-0.1875, 0.0, 1.0],    # 6: x = 2.5 exactly -> floor(3.0) = pixel (3, 4)
        [0.0, 0.0, 0.1],        # 7: nearer than z_near = 0.2
        [0.0, 5.0e3, 2.0e4],    # 8: pixel (4, 6) but beyond z_far = 1e4: culled
        [0.0, 0.0, 1.0e4],      # 9: on z_far (open interval): culled
    ], np.float32)
    depth, ids = O.zbuffer(pts, cam)
    exp_ids = np.full((8, 8), -1, np.int32)
    exp_depth = np.zeros((8, 8), np.float32)
    exp_ids[4, 4], exp_depth[4, 4] = 1, 1.5
    exp_ids[4, 5], exp_depth[4, 5] = 2, 1.0
    exp_ids[4, 3], exp_depth[4, 3] = 6, 1.0
    assert np.array_equal(ids, exp_ids)
    assert np.array_equal(depth, exp_depth)


# ---------------------------------------------------------------------------
# adjoints of projection and lifting (gradients to the 3D Gaussians and on
# to the source maps): central differences of the FP64 forward
# ---------------------------------------------------------------------------

def _proj_loss(mean, cov, cam, w_mu, w_con):
    mu, con, _, vis = O.project_f64(O.Gaussians(mean, cov, np.zeros(len(mean)), np.zeros((len(mean), 1))), cam)
    return float((w_mu * mu).sum() + (w_con * con).sum())


def test_projection_adjoint_matches_central_differences():
    rng = np.random.default_rng(41)
    cam = gen.make_camera(300.0, 320, 240, (0.05, -0.02, -0.1), gen.rot_y(7.0) @ gen.rot_x(-4.0), cx=161.0, cy=118.5)
    gs = gen.random_gaussians(5, 12, 1, center=(0.05, 0.0, 1.4), spread=0.25, sigma_range=(0.01, 0.05))
    mean = gs.mean.astype(np.float64)
    mean[0] = [1.2, 0.1, 1.0]      # far off axis: x/z clamped (no gradient through the ratio)
    mean[1] = [-0.1, -1.0, 0.9]    # y/z clamped
    cov = gs.cov.astype(np.float64)
    w_mu, w_con = rng.standard_normal((12, 2)), rng.standard_normal((12, 3))
    gm, gc = O.project_backward(mean, cov, cam, w_mu, w_con)
    for arr, g in ((mean, gm), (cov, gc)):
        for idx in np.ndindex(arr.shape):
            # steps relative to the Gaussian's scale (metres for means, the
            # largest variance for covariances)
            h = 1e-6 * max(1.0, abs(arr[idx])) if arr is mean else 1e-4 * cov[idx[0], [0, 3, 5]].max()
            up, dn = arr.copy(), arr.copy()
            up[idx] += h
            dn[idx] -= h
            args_up = (up, cov) if arr is mean else (mean, up)
            args_dn = (dn, cov) if arr is mean else (mean, dn)
            fd = (_proj_loss(*args_up, cam, w_mu, w_con) - _proj_loss(*args_dn, cam, w_mu, w_con)) / (2 * h)
            scale = max(abs(g[idx]), np.abs(g).max() * 1e-3, 1e-9)
            assert abs(fd - g[idx]) <= 1e-5 * scale, (idx, fd, g[idx])


def test_projection_adjoint_anisotropic_intrinsics_and_clamp_band():
    """The same check with fx != fy, so the clamp limits differ between the
    axes (1.3 * 0.5 W / fx = 0.693 in x, 1.3 * 0.5 H / fy = 0.6 in y): one
    Gaussian lies between the two limits in x (inside, so its ratio carries
    gradient), others beyond the y limit and beyond the negative x limit."""
    rng = np.random.default_rng(42)
    cam = gen.Camera(300.0, 260.0, 161.0, 118.5, 320, 240, np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    gs = gen.random_gaussians(6, 8, 1, center=(0.0, 0.0, 1.3), spread=0.2, sigma_range=(0.01, 0.05))
    mean = gs.mean.astype(np.float64)
    mean[0] = [0.65 * 1.2, 0.1, 1.2]     # x/z = 0.65: inside in x, past the y limit's value
    mean[1] = [0.2, 0.64 * 1.1, 1.1]     # y/z = 0.64 > 0.6: clamped in y
    mean[2] = [-0.8, 0.05, 1.0]          # x/z = -0.8 < -0.693: clamped in x
    cov = gs.cov.astype(np.float64)
    w_mu, w_con = rng.standard_normal((8, 2)), rng.standard_normal((8, 3))
    w_mu[:3] = 0.0   # the three placed Gaussians' mean gradients come through the conic alone
    gm, gc = O.project_backward(mean, cov, cam, w_mu, w_con)
    for arr, g in ((mean, gm), (cov, gc)):
        for idx in np.ndindex(arr.shape):
            h = 1e-6 * max(1.0, abs(arr[idx])) if arr is mean else 1e-4 * cov[idx[0], [0, 3, 5]].max()
            up, dn = arr.copy(), arr.copy()
            up[idx] += h
            dn[idx] -= h
            args_up = (up, cov) if arr is mean else (mean, up)
            args_dn = (dn, cov) if arr is mean else (mean, dn)
            fd = (_proj_loss(*args_up, cam, w_mu, w_con) - _proj_loss(*args_dn, cam, w_mu, w_con)) / (2 * h)
            scale = max(abs(g[idx]), np.abs(g).max() * 1e-3, 1e-9)
            assert abs(fd - g[idx]) <= 1e-5 * scale, (idx, fd, g[idx])


def _lift_loss(view, w):
    g = O.lift_view(view, "f64")
    return float((w["mean"] * g.mean).sum() + (w["cov"] * g.cov).sum() + (w["op"] * g.opac).sum()
                 + (w["ft"] * g.feat).sum())


def test_lift_adjoint_matches_central_differences():
    rng = np.random.default_rng(43)
    H, W, C = 5, 6, 2
    cam = gen.make_camera(6.0, W, H, (0.1, -0.05, 0.02), gen.rot_y(10.0) @ gen.rot_x(5.0), cx=2.7, cy=2.2)
    mask = (rng.uniform(size=(H, W)) > 0.3).astype(np.uint8)
    quat = rng.standard_normal((H, W, 4)) * 0.3 + np.array([1.3, 0, 0, 0])
    view = gen.SourceView(rng.uniform(0.8, 1.6, (H, W)).astype(np.float32), mask,
                          rng.uniform(0.01, 0.05, (H, W, 3)).astype(np.float32), quat.astype(np.float32),
                          rng.uniform(0.3, 0.9, (H, W)).astype(np.float32),
                          rng.standard_normal((H, W, C)).astype(np.float32), cam)
    n = int(mask.sum())
    w = dict(mean=rng.standard_normal((n, 3)), cov=rng.standard_normal((n, 6)) * 50, op=rng.standard_normal(n),
             ft=rng.standard_normal((n, C)))
    g = O.lift_backward(view, w["mean"], w["cov"], w["op"], w["ft"])
    for name, key in (("depth", "depth"), ("scale", "scale"), ("quat", "quat"), ("opacity", "opacity"),
                      ("feat", "feat")):
        arr = getattr(view, name)
        grad = g[key]
        for idx in np.ndindex(arr.shape):
            if not mask[idx[0], idx[1]]:
                assert grad[idx] == 0.0
                continue
            v = float(arr[idx])
            h = 1e-3 * max(abs(v), 0.05)
            up, dn = arr.copy(), arr.copy()
            up[idx] = np.float32(v + h)
            dn[idx] = np.float32(v - h)
            step = float(up[idx]) - float(dn[idx])
            vu = gen.SourceView(*(up if f == name else getattr(view, f) for f in
                                  ("depth", "mask", "scale", "quat", "opacity", "feat", "cam")))
            vd = gen.SourceView(*(dn if f == name else getattr(view, f) for f in
                                  ("depth", "mask", "scale", "quat", "opacity", "feat", "cam")))
            fd = (_lift_loss(vu, w) - _lift_loss(vd, w)) / step
            scale = max(abs(grad[idx]), np.abs(grad).max() * 1e-3)
            assert abs(fd - grad[idx]) <= 1e-4 * scale, (name, idx, fd, grad[idx])


def test_chained_adjoints_match_central_differences_of_source_maps():
    """The three adjoints chained (compositing, projection, lifting) against
    central differences of the FP64 forward (lift, project, composite with
    the base decisions and tile lists frozen) w.r.t. entries of the source
    depth, scale, quaternion, opacity and feature maps."""
    sc = gen.scene_paper(seed=17, res=24, C=2)
    cam = gen.make_camera(30.0, 32, 32, (0.01, 0.0, -0.02), gen.rot_y(3.0))
    g32 = O.lift_scene(sc, "f32")
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, 32, 32)
    rng = np.random.default_rng(8)
    gF = rng.standard_normal((2, 32, 32)); gA = rng.standard_normal((32, 32))

    def forward(views):
        g = O.Gaussians(*(np.concatenate([getattr(O.lift_view(v, "f64"), k) for v in views], 0)
                          for k in ("mean", "cov", "opac", "feat")))
        mu, conic, _, _ = O.project_f64(g, cam, PAR)
        return g, mu, conic

    g0, mu0, con0 = forward(sc.views)
    r0, dec = O.composite(mu0, con0, g0.opac, g0.feat, 32, 32, bins, PAR, record=True)

    def loss(views):
        g, mu, conic = forward(views)
        r = O.composite(mu, conic, g.opac, g.feat, 32, 32, bins, PAR, dec_in=dec)
        return float((gF * r.F).sum() + (gA * r.A).sum())

    d_mu, d_con, d_op, d_ft = O.backward(mu0, con0, g0.opac, g0.feat, 32, 32, bins, gF, gA, PAR)
    g_mean, g_cov = O.project_backward(g0.mean, g0.cov, cam, d_mu, d_con)
    n0 = int(sc.views[0].mask.sum())
    grads = O.lift_backward(sc.views[0], g_mean[:n0], g_cov[:n0], d_op[:n0], d_ft[:n0])
    # pixels of view 0 whose Gaussian lands in a used tile list
    used = set(np.unique(bins.ids).tolist())
    fg = np.argwhere(sc.views[0].mask.reshape(-1) > 0)[:, 0]
    cand = [(p, k) for k, p in enumerate(fg) if k in used]
    picks = [cand[i] for i in rng.choice(len(cand), size=8, replace=False)]
    H, W = sc.views[0].depth.shape
    checked = 0
    for p, k in picks:
        y, x = divmod(int(p), W)
        for name, sub in (("depth", ()), ("scale", (0,)), ("scale", (2,)), ("quat", (1,)), ("quat", (0,)),
                          ("opacity", ()), ("feat", (1,))):
            arr = getattr(sc.views[0], name)
            pos = (y, x) + sub
            v0 = float(arr[pos])
            h = 1e-3 * max(abs(v0), 0.05)
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2[pos] = np.float32(v0 + sgn * h)
                vals.append((float(a2[pos]), loss([gen.SourceView(*(a2 if f == name else getattr(sc.views[0], f)
                                                                      for f in ("depth", "mask", "scale", "quat",
                                                                                "opacity", "feat", "cam")))]
                                                  + list(sc.views[1:]))))
            fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
            an = grads[name][pos]
            scale = max(abs(an), np.abs(grads[name]).max() * 1e-2)
            assert abs(fd - an) <= 2e-3 * scale, (name, pos, fd, an)
            checked += 1
    assert checked == 56


# ---------------------------------------------------------------------------
# tight binning (a variant of the binning; not in the paper's rasterizer)
# ---------------------------------------------------------------------------

def test_key_ln_matches_math_log():
    xs = np.concatenate([np.geomspace(1.0, 1e4, 2000), [1.0, 2.0, 1.41421354, 1.4142137, 255.0, 0.95 * 255.0]])
    xs = xs.astype(np.float32)
    err = max(abs(O.key_ln(float(x)) - math.log(float(x))) for x in xs)
    assert err <= 1.5e-6
    # within 2 single-precision ulps of ln x (ulps of 0.5 below |ln x| = 0.5)
    ulps = max(abs(O.key_ln(float(x)) - math.log(float(x)))
               / float(np.spacing(np.float32(max(abs(math.log(float(x))), 0.5)))) for x in xs)
    assert ulps <= 2.0, ulps
    assert O.key_ln(1.0) == 0.0 and O.key_ln(2.0) == np.float32(math.log(2.0))


def _tight_scene():
    """Anisotropic random Gaussians (some below alpha_min in opacity, some
    large) in a ragged 150 x 100 target."""
    gs = gen.random_gaussians(31, 4000, 2, center=(0, 0, 1.2), spread=0.45, sigma_range=(0.001, 0.03))
    rng = np.random.default_rng(32)
    op = gs.opac.copy()
    op[rng.choice(len(op), 200, replace=False)] = rng.uniform(0.0005, 0.0039, 200).astype(np.float32)
    g32 = O.Gaussians(gs.mean, gs.cov, op, gs.feat)
    cam = _cam(f=120.0, W=150, H=100)
    return g32, cam


def _pairs(proj, W, H):
    b = O.bin_gaussians(proj, W, H)
    return b, set(zip((b.keys >> 32).astype(np.int64).tolist(), b.ids.astype(np.int64).tolist()))


def test_tight_binning_drops_only_tiles_without_a_blendable_pixel():
    """Brute force over every pixel of every dropped (Gaussian, tile) pair:
    alpha = o exp(-Q/2) < alpha_min there (FP64), so the full rect would
    not have blended it anywhere in that tile."""
    g32, cam = _tight_scene()
    W, H = cam.width, cam.height
    pr = O.project_f32(g32, cam, PAR)
    pt = O.tighten(pr, g32.opac, W, H, PAR)
    b0, full = _pairs(pr, W, H)
    b1, tight = _pairs(pt, W, H)
    assert tight <= full and len(tight) < 0.9 * len(full)
    amin = float(PAR[2])
    tx = (W + 15) // 16
    for t, i in full - tight:
        x0, y0 = 16 * (t % tx), 16 * (t // tx)
        xs = np.arange(x0, min(x0 + 16, W), dtype=np.float64)
        ys = np.arange(y0, min(y0 + 16, H), dtype=np.float64)
        dx = xs[None, :] - float(pr.mu[i, 0])
        dy = ys[:, None] - float(pr.mu[i, 1])
        a, b, c = (float(v) for v in pr.conic[i])
        Q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        alpha = float(g32.opac[i]) * np.exp(-0.5 * Q)
        assert alpha.max() < amin, (t, i)
    # Gaussians whose opacity is below alpha_min have no tile at all
    low = np.where(g32.opac < amin)[0]
    assert np.all(pt.ntiles[low] == 0) and np.any(pr.ntiles[low] > 0)


def test_tight_binning_culls_opacity_just_below_alpha_min():
    """alpha = o e^q <= o, so a Gaussian with o < alpha_min is blended
    nowhere and keeps no tile, however close o is to alpha_min: the rounding
    margin of the kept-tile test must not let it through."""
    g32, cam = _tight_scene()
    W, H = cam.width, cam.height
    amin = np.float32(PAR[2])
    pr0 = O.project_f32(g32, cam, PAR)
    idx = np.where(pr0.ntiles > 0)[0][:24]
    op = g32.opac.copy()
    eps = [2.0 ** -k for k in range(9, 24)] + [0.0] * 9
    op[idx] = [np.nextafter(amin, np.float32(0)) if e == 0.0 else np.float32(amin * (1.0 - e)) for e in eps]
    assert np.all(op[idx] < amin)
    g = O.Gaussians(g32.mean, g32.cov, op, g32.feat)
    pr = O.project_f32(g, cam, PAR)
    pt = O.tighten(pr, op, W, H, PAR)
    assert np.all(pr.ntiles[idx] > 0)   # the full rect keeps them
    assert np.all(pt.ntiles[idx] == 0)


def test_tight_binning_full_masks_and_whole_rects():
    """A 32-tile rect whose tiles the alpha_min ellipse all reaches keeps all
    32 (every mask bit, the last included); a rect of more than 32 tiles is
    kept whole and emits every tile.  The image is 32 x 4 tiles."""
    cam = gen.make_camera(100.0, 512, 64, (0, 0, 0), np.eye(3), cx=256.0, cy=32.0)
    z = 2.0
    s1, s2 = 20.0 * z / 100.0, 50.0 * z / 100.0
    mean = np.array([[0.0, 0.0, z], [1.0, 0.0, z]], np.float32)
    cov = np.array([[s1 * s1, 0, 0, s1 * s1, 0, 1e-6], [s2 * s2, 0, 0, s2 * s2, 0, 1e-6]], np.float32)
    g = O.Gaussians(mean, cov, np.array([0.99, 0.99], np.float32), np.ones((2, 1), np.float32))
    pr = O.project_f32(g, cam, PAR)
    pt = O.tighten(pr, g.opac, cam.width, cam.height, PAR)
    area = (pr.rect[:, 2] - pr.rect[:, 0]) * (pr.rect[:, 3] - pr.rect[:, 1])
    assert area[0] == 32 and area[1] > 32
    assert pt.ntiles[0] == 32 and pt.ntiles[1] == area[1]
    b = O.bin_gaussians(pt, cam.width, cam.height)
    assert (b.ids == 0).sum() == 32 and (b.ids == 1).sum() == area[1]


def test_tight_binning_keeps_tiles_the_ellipse_reaches():
    """The kept tiles are not over-conservative: for each kept pair, dense
    sampling of the tile's pixel-centre rectangle (FP64) finds a point with
    Q within 2% of 2 ln(o / alpha_min) (the margin is 0.1% + 2^-8)."""
    g32, cam = _tight_scene()
    W, H = cam.width, cam.height
    pr = O.project_f32(g32, cam, PAR)
    pt = O.tighten(pr, g32.opac, W, H, PAR)
    b1, tight = _pairs(pt, W, H)
    amin = float(PAR[2])
    tx = (W + 15) // 16
    g = np.linspace(0.0, 1.0, 121)
    checked = 0
    for t, i in sorted(tight):
        area = (pr.rect[i, 2] - pr.rect[i, 0]) * (pr.rect[i, 3] - pr.rect[i, 1])
        if area > 32:
            continue
        x0, y0 = 16 * (t % tx), 16 * (t // tx)
        x1, y1 = min(x0 + 15, W - 1), min(y0 + 15, H - 1)
        dx = (x0 + g * (x1 - x0))[None, :] - float(pr.mu[i, 0])
        dy = (y0 + g * (y1 - y0))[:, None] - float(pr.mu[i, 1])
        a, b, c = (float(v) for v in pr.conic[i])
        Q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        kappa = 2 * math.log(float(g32.opac[i]) / amin)
        assert Q.min() <= kappa * 1.02 + 0.05, (t, i, Q.min(), kappa)
        checked += 1
    assert checked > 1000


def test_tight_binning_renders_the_same_maps():
    """Dropping tiles that hold no blendable pixel changes no decision: the
    FP64 composite with tight bins equals the full-rect one bit for bit,
    and each pixel's last blended Gaussian is the same one."""
    for g32, cam in [_tight_scene(), (O.lift_scene(gen.scene_paper(seed=5, res=96, C=3), "f32"),
                                      gen.make_camera(110.0, 120, 90, (0.02, 0, 0), gen.rot_y(3.0)))]:
        r0 = O.render(g32, cam, PAR)
        r1 = O.render(g32, cam, PAR, tight=True)
        assert r1.bins.P < r0.bins.P
        assert np.array_equal(r0.comp.F, r1.comp.F) and np.array_equal(r0.comp.T, r1.comp.T)
        assert np.array_equal(r0.comp.flags, r1.comp.flags)
        yy, xx = np.mgrid[0:cam.height, 0:cam.width]
        t = (yy // 16) * r0.bins.tiles_x + xx // 16
        gid = []
        for rr in (r0, r1):
            pos = rr.bins.ranges[t, 0].astype(np.int64) + rr.comp.last.astype(np.int64) - 1
            ids = rr.bins.ids.astype(np.int64)[np.clip(pos, 0, max(rr.bins.P - 1, 0))]
            gid.append(np.where(rr.comp.last > 0, ids, -1))
        assert np.array_equal(gid[0], gid[1]) and (gid[0] >= 0).mean() > 0.3
