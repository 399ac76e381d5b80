"""Seeded synthetic inputs: determinism and the workload sizes."""
import numpy as np

from paper_2405_14866_gb300 import gen


def test_tiny_is_deterministic_per_seed():
    a, b, c = gen.scene_tiny(0), gen.scene_tiny(0), gen.scene_tiny(1)
    for k in ("depth", "scale", "opacity", "feat"):
        assert np.array_equal(getattr(a.views[0], k), getattr(b.views[0], k))
    assert not np.array_equal(a.views[0].feat, c.views[0].feat)
    assert a.n_foreground == 4096


def test_tiny_inputs_follow_the_recipe():
    v = gen.scene_tiny().views[0]
    vv, uu = np.mgrid[0:64, 0:64]
    assert np.allclose(v.depth, 1.0 + 0.1 * np.sin(uu / 9) * np.cos(vv / 7), atol=1e-6)
    k = v.scale[..., 0] / (v.depth / 64.0)
    assert k.min() >= 0.8 - 1e-5 and k.max() <= 1.5 + 1e-5
    assert np.array_equal(v.scale[..., 0], v.scale[..., 1])
    assert 0.3 <= v.opacity.min() and v.opacity.max() <= 0.95
    assert v.feat.shape == (64, 64, 8)
    assert np.array_equal(v.quat[..., 0], np.ones((64, 64), np.float32))


def test_workload_gaussian_counts():
    # foreground pixels = Gaussians: ~1.26M (2 views, 60% ellipse),
    # ~2.10M (4 views, 50%), ~315K per differentiation sample (2 x 512^2, 60%)
    n_paper = 2 * int(gen.ellipse_mask(1024, 1024, 0.45, 0.425).sum())
    n_prec = 4 * int(gen.ellipse_mask(1024, 1024, 0.42, 0.379).sum())
    n_diff = 2 * int(gen.ellipse_mask(512, 512, 0.45, 0.425).sum())
    assert abs(n_paper - 1.26e6) / 1.26e6 < 0.01
    assert abs(n_prec - 2.10e6) / 2.10e6 < 0.01
    assert abs(n_diff - 315e3) / 315e3 < 0.01


def test_value_noise_range_and_rig():
    rng = np.random.default_rng(0)
    n = gen.value_noise(rng, 64, 80)
    assert n.min() == 0.0 and n.max() == 1.0
    cams = gen._rig_two(64, 64.0)
    # camera centres at x = -+0.15 m, optical axes verging by 10 degrees
    for cam, x in zip(cams, (-0.15, 0.15)):
        centre = -cam.R.T.astype(np.float64) @ cam.t.astype(np.float64)
        assert np.allclose(centre, [x, 0, 0], atol=1e-6)
    z0 = cams[0].R[2].astype(np.float64)
    z1 = cams[1].R[2].astype(np.float64)
    assert abs(np.degrees(np.arccos(np.clip(z0 @ z1, -1, 1))) - 10.0) < 1e-4


def test_look_at_is_opencv():
    # straight down +z from the origin: the identity (x right, y down)
    assert np.allclose(gen.look_at_c2w((0, 0, 0), (0, 0, 5)), np.eye(3))
    R = gen.look_at_c2w((0.3, -0.1, -1.0), (0.0, 0.0, 1.2))
    assert np.allclose(R.T @ R, np.eye(3)) and np.isclose(np.linalg.det(R), 1.0)
    assert R[1, 1] > 0.9          # camera y stays close to world y (down)


def _pix(cam, x):
    """Pixel of world point x in `cam` (FP64 from the stored FP32 pose)."""
    p = cam.R.astype(np.float64) @ x + cam.t.astype(np.float64)
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy]), p[2]


def test_display_transform_geometry():
    """Sec. 3.1: 180 deg turn about the eye-display midpoint, then 0.5 scale
    about the eye centre.  Checked on the composite map: the remote eye
    centre lands on the display centre, the remote user's plane on the
    display plane, distances halve, the remote display lands between the
    local display and the local eye, and left and right swap (the two users
    face each other)."""
    s, Rm, tm = gen.display_transform(1.2, 0.5)
    T = lambda x: s * Rm @ np.asarray(x, np.float64) + tm
    assert np.allclose(T([0, 0, 1.2]), 0.0)
    assert np.isclose(T([0.3, -0.2, 1.2])[2], 0.0)
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=3), rng.normal(size=3)
    assert np.isclose(np.linalg.norm(T(a) - T(b)), 0.5 * np.linalg.norm(a - b))
    assert np.allclose(T([0, 0, 0]), [0, 0, 0.6])
    assert T([0.1, 0, 1.2])[0] < 0 and T([0, 0.1, 1.2])[1] > 0


def test_display_eye_camera_sees_what_the_local_eye_sees():
    """The remote-frame eye camera projects every remote point where the
    local eye, looking at the display centre, sees its displayed image."""
    s, Rm, tm = gen.display_transform()
    rng = np.random.default_rng(4)
    res = 512
    f = res * 1.25 / (2 * gen.PANEL_HALF_HEIGHT)
    for _ in range(5):
        eye = np.array([rng.uniform(-0.43, 0.43), rng.uniform(-0.05, 0.05), rng.uniform(1.1, 1.4)])
        cr = gen.display_eye_camera(eye, res)
        cl = gen.make_camera(f, res, res, eye, gen.look_at_c2w(eye, (0, 0, 0)))
        for _ in range(20):
            x = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.8, 1.6)])
            ur, zr = _pix(cr, x)
            ul, zl = _pix(cl, s * Rm @ x + tm)
            assert np.allclose(ur, ul, atol=2e-3) and np.isclose(zl, s * zr, rtol=1e-5)
    # the display centre (remote eye centre) is at the image centre
    u, _ = _pix(gen.display_eye_camera([0.2, 0.0, 1.3], res), np.array([0.0, 0.0, 1.2]))
    assert np.allclose(u, (res - 1) / 2, atol=1e-3)


def test_display_eye_cameras_cover_the_viewing_range():
    cams = gen.display_eye_cameras(np.random.default_rng(1), 256, 200)
    assert len(cams) == 400
    centres = np.array([-c.R.T.astype(np.float64) @ c.t.astype(np.float64) for c in cams])
    # local head x in +-0.4, z in 1.25 +- 0.15, eyes +-3.2 cm, mapped by x -> -2x, z -> 1.2 - 2z
    assert np.all(np.abs(centres[:, 0]) <= 2 * (0.4 + 0.032) + 1e-5)
    assert centres[:, 0].min() < -0.7 and centres[:, 0].max() > 0.7
    assert np.all((centres[:, 2] >= 1.2 - 2 * 1.4 - 1e-5) & (centres[:, 2] <= 1.2 - 2 * 1.1 + 1e-5))
    # pairs: 2 x 6.4 cm apart in the remote frame, both looking at the remote eye centre
    assert np.allclose(np.linalg.norm(centres[0::2] - centres[1::2], axis=1), 0.128, atol=1e-5)
    for c in cams[:10]:
        u, z = _pix(c, np.array([0.0, 0.0, 1.2]))
        assert z > 0 and np.allclose(u, 127.5, atol=1e-3)


def test_paper_rig_scene():
    sc = gen.scene_paper_rig(seed=5, res=64, C=4, n_viewers=2, target_res=80)
    four = gen._rig_four(64, 64.0)
    assert len(sc.views) == 3 and len(sc.targets) == 4
    for v, k in zip(sc.views, (0, 2, 3)):
        assert np.array_equal(v.cam.R, four[k].R) and np.array_equal(v.cam.t, four[k].t)
    assert sc.feat_dtype == gen.FEAT_BF16 and sc.targets[0].width == 80
    n = 3 * int(gen.ellipse_mask(1024, 1024, 0.42, 0.379).sum())
    assert abs(n - 1.575e6) / 1.575e6 < 0.01
