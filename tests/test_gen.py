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
