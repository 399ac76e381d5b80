"""CUDA path vs the FP64 oracle, through the C ABI.

Bit-exact: lifted Gaussians (single-precision key mode), projected record,
tile rects, depth keys, radii, (tile, depth, id) pair order and tile ranges.
Within tolerance: the feature and alpha maps (1e-4 FP32; BF16 storage
2e-2 against the oracle fed the original FP32 features, 1e-4 against the
oracle fed the same BF16-rounded features).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import _lib as L
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu
PAR = O.params_array()


def _f32bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _render(g, cam, save=True, params=None):
    ctx = api.Context()
    F, A = ctx.render(g, cam, params=params, save=save)
    torch.cuda.synchronize()
    return ctx, F, A


def _scenes():
    tiny = gen.scene_tiny()
    paper = gen.scene_paper(seed=11, res=128, C=16)
    paper.targets = [gen.make_camera(150.0, 200, 136, (0.01, 0.0, -0.02), gen.rot_y(2.0))]  # ragged tiles
    prec = gen.scene_precision(seed=12, res=96, C=8)
    prec.targets = [gen.make_camera(120.0, 160, 120, (0, 0, 0), np.eye(3))]
    return {"tiny": tiny, "paper": paper, "precision": prec}


SCENES = _scenes()


@pytest.mark.parametrize("name", list(SCENES))
def test_build_bitexact(name):
    sc = SCENES[name]
    g, keep = P.gpu_build(sc)
    d = {k: v.cpu() for k, v in g.get().items()}
    o = O.lift_scene(sc, "f32")
    assert g.count() == o.n == sc.n_foreground
    assert np.array_equal(_f32bits(d["mean"].numpy()), _f32bits(o.mean))
    assert np.array_equal(_f32bits(d["cov"].numpy()), _f32bits(o.cov))
    assert np.array_equal(_f32bits(d["opac"].numpy()), _f32bits(o.opac))
    feat = d["feat"].float().numpy()
    assert np.array_equal(_f32bits(feat), _f32bits(o.feat))   # BF16 rounding is round-to-nearest-even on both


@pytest.mark.parametrize("name", list(SCENES))
def test_projection_and_bins_bitexact(name):
    sc = SCENES[name]
    cam = sc.targets[0]
    g, keep = P.gpu_build(sc)
    ctx, F, A = _render(g, cam)
    g32 = O.lift_scene(sc, "f32")
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    st = ctx.stats()
    assert st["device_status"] == 0
    assert st["n_pairs"] == bins.P and st["n_visible"] == int((pr.ntiles > 0).sum())
    assert np.array_equal(ctx.export("rect").cpu().numpy(), pr.rect)
    assert np.array_equal(ctx.export("depthkey").cpu().numpy().view(np.uint32), pr.dkey)
    assert np.array_equal(ctx.export("radius").cpu().numpy(), pr.radius)
    vis = pr.ntiles > 0
    assert np.array_equal(_f32bits(ctx.export("mean2d").cpu().numpy())[vis], _f32bits(pr.mu)[vis])
    assert np.array_equal(_f32bits(ctx.export("conic").cpu().numpy())[vis], _f32bits(pr.conic)[vis])
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)


@pytest.mark.parametrize("name", list(SCENES))
def test_feature_map_matches_oracle(name):
    sc = SCENES[name]
    cam = sc.targets[0]
    g, keep = P.gpu_build(sc)
    ctx, F, A = _render(g, cam)
    g32 = O.lift_scene(sc, "f32")
    orc = O.render(g32, cam, PAR)
    tol = P.TOL_F32
    stats = P.compare_render(F, A, orc, g32, cam, PAR, tol)
    assert stats["n_flagged"] <= 0.02 * stats["n_pixels"]
    if sc.feat_dtype == api.BF16:
        # storage error included: oracle fed the original FP32 features
        g_orig = O.lift_scene(sc, "f32", bf16_features=False)
        orc2 = O.render(g32, cam, PAR, feat64=g_orig.feat)
        P.compare_render(F, A, orc2, g32, cam, PAR, P.TOL_BF16, feat64=g_orig.feat)


def test_saved_state_matches_oracle():
    sc = SCENES["paper"]
    cam = sc.targets[0]
    g, keep = P.gpu_build(sc)
    ctx, F, A = _render(g, cam, save=True)
    g32 = O.lift_scene(sc, "f32")
    orc = O.render(g32, cam, PAR)
    plain = orc.comp.flags == 0
    last = ctx.export("last").cpu().numpy()
    T = ctx.export("tfinal").cpu().numpy()
    assert np.array_equal(last[plain], orc.comp.last[plain])
    assert np.allclose(T[plain], orc.comp.T[plain], rtol=1e-4, atol=1e-7)


def test_rasterize_equals_render():
    sc = SCENES["paper"]
    cam = sc.targets[0]
    g, keep = P.gpu_build(sc)
    ctx, F, A = _render(g, cam)
    mean2d, conic = ctx.export("mean2d"), ctx.export("conic")
    radius = ctx.export("radius").round().to(torch.int32)
    dk = ctx.export("depthkey")
    depth = dk.view(torch.float32).clone()
    depth[dk == -1] = 0.0
    d = g.get()
    ctx2 = api.Context()
    F2, A2 = ctx2.rasterize(mean2d, conic, d["opac"], depth, radius, d["feat"], cam.width, cam.height)
    torch.cuda.synchronize()
    assert torch.equal(F, F2) and torch.equal(A, A2)


@pytest.mark.parametrize("C,dtype", [(1, api.F32), (3, api.F32), (5, api.BF16), (8, api.BF16), (12, api.BF16),
                                     (16, api.F32), (24, api.F32), (32, api.F32), (32, api.BF16), (33, api.F32),
                                     (64, api.BF16), (64, api.F32)])
def test_channel_counts_and_dtypes(C, dtype):
    gs = gen.random_gaussians(3, 3000, C, center=(0, 0, 1.2), spread=0.25)
    g32 = O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat)
    if dtype == api.BF16:
        g32.feat = O.round_bf16(g32.feat)
    cam = gen.make_camera(90.0, 77, 61, (0, 0, 0), np.eye(3))
    g = P.gpu_gaussians(g32, dtype)
    ctx, F, A = _render(g, cam)
    orc = O.render(g32, cam, PAR)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32)


def test_empty_and_fully_culled():
    cam = gen.make_camera(64.0, 40, 24, (0, 0, 0), np.eye(3))
    # every Gaussian behind the camera or beyond the image
    gs = gen.random_gaussians(4, 500, 4, center=(0, 0, -2.0), spread=0.5)
    g = P.gpu_gaussians(O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat))
    ctx, F, A = _render(g, cam)
    assert ctx.stats()["n_pairs"] == 0 and ctx.stats()["n_visible"] == 0
    assert not F.any() and not A.any()
    # no Gaussians at all
    g0 = api.Gaussians.create(16, 4)
    ctx0, F0, A0 = _render(g0, cam)
    assert not F0.any() and not A0.any() and ctx0.stats()["n_gaussians"] == 0


def test_large_gaussian_covering_every_tile():
    cam = gen.make_camera(64.0, 100, 70, (0, 0, 0), np.eye(3))
    mean = np.array([[0.0, 0.0, 1.0], [0.05, 0.02, 1.5]], np.float32)
    cov = np.array([[0.5, 0.0, 0.0, 0.5, 0.0, 0.1], [1e-4, 0, 0, 1e-4, 0, 1e-4]], np.float32)
    g32 = O.Gaussians(mean, cov, np.array([0.6, 0.9], np.float32), np.array([[1.0, -2.0], [3.0, 0.5]], np.float32))
    g = P.gpu_gaussians(g32)
    ctx, F, A = _render(g, cam)
    orc = O.render(g32, cam, PAR)
    assert ctx.stats()["n_pairs"] == orc.bins.P > 35
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32)


def test_async_mode_reports_capacity_overflow():
    sc = SCENES["tiny"]
    cam = sc.targets[0]
    g, keep = P.gpu_build(sc)
    ctx = api.Context()
    ctx.reserve(4096, 1000, 64, 64, 8)        # fewer pairs than the render needs
    F, A = ctx.render(g, cam, async_=True)
    with pytest.raises(L.TsplatError) as e:
        ctx.status()
    assert e.value.status == 3
    ctx2 = api.Context()
    ctx2.reserve(4096, 20000, 64, 64, 8)
    F2, A2 = ctx2.render(g, cam, async_=True)
    ctx2.status()
    _, F3, A3 = _render(g, cam, save=False)
    assert torch.equal(F2, F3) and torch.equal(A2, A3)


def test_build_from_bf16_feature_maps_equals_fp32_maps():
    """Source feature maps given in BF16 (rounded on the host) build the same
    BF16 store, bit for bit, as FP32 maps rounded during the lift."""
    sc = gen.scene_precision(seed=51, res=64, C=32)
    g1, _ = P.gpu_build(sc)
    up = api.upload_scene(sc, feat_dtype=api.BF16)
    views = [api.source_view(v["depth"], v["mask"], v["scale"], v["quat"], v["opacity"], v["feat"], v["cam"])
             for v in up["views"]]
    assert views[0].feat_dtype == api.BF16
    g2 = api.Gaussians.build(views, sc.C, api.BF16)
    torch.cuda.synchronize()
    a, b = g1.get(), g2.get()
    assert a.keys() == b.keys()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_large_ragged_image_many_tiles():
    """4500 x 4500 target (282 x 282 = 79,524 tiles, more than one scan
    block's 1024 threads cover one each; ragged last tile row and column):
    bins bit-exact, feature map on sampled tiles, including the ragged ones."""
    cam = gen.make_camera(2200.0, 4500, 4500, (0, 0, 0), np.eye(3))
    gs = gen.random_gaussians(21, 30000, 3, center=(0, 0, 1.6), spread=0.75, sigma_range=(0.0005, 0.004))
    g32 = O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat)
    g = P.gpu_gaussians(g32)
    ctx, F, A = _render(g, cam, save=False)
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    assert ctx.stats()["n_pairs"] == bins.P > 30000
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    tx = (cam.width + 15) // 16
    rng = np.random.default_rng(3)
    busy = np.argsort(-counts)[:6].tolist()
    ragged = [tx * tx - 1, tx * (tx // 2) + tx - 1, (tx - 1) * tx + tx // 2]
    tiles = sorted(set(busy + ragged + rng.choice(tx * tx, 6, replace=False).tolist()))
    orc = O.render(g32, cam, PAR, tiles=tiles)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32, tiles=tiles)
