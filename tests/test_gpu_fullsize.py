"""The two 1024x1024 workloads at full size, in the launch configuration
bench.py times (lifting into an existing store, asynchronous render into a
reserved context):
- the headline: four source views, ~2.10 M Gaussians, 32-channel features
  stored BF16 (source feature maps given in BF16);
- the paper-shaped workload: two source views (30 cm baseline verging
  10 degrees), ~1.26 M Gaussians, 32-channel FP32 features.

Bit-exact over every Gaussian and pair: the lifted store, the projected
record, tile rects, depth keys and the (tile, depth, id) order.  The feature
and alpha maps are compared over the whole image with the FP64 oracle
(1e-4 against the oracle fed the stored features; for BF16 storage also
2e-2 against the oracle fed the original FP32 features).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu
PAR = O.params_array()


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _full_size(sc):
    cam = sc.targets[0]
    up = api.upload_scene(sc, feat_dtype=sc.feat_dtype)
    views = [api.source_view(v["depth"], v["mask"], v["scale"], v["quat"], v["opacity"], v["feat"], v["cam"])
             for v in up["views"]]
    g = api.Gaussians.build(views, sc.C, sc.feat_dtype)
    ctx = api.Context()
    F0, A0 = ctx.render(g, cam)
    st = ctx.stats()
    ctx.reserve(g.capacity, int(st["n_pairs"] * 1.25) + 65536, cam.width, cam.height, sc.C)
    F, A = torch.empty_like(F0), torch.empty_like(A0)
    g.build_into(views)
    ctx.render(g, cam, async_=True, out_feat=F, out_alpha=A)
    ctx.status()
    assert torch.equal(F, F0) and torch.equal(A, A0)

    g32 = O.lift_scene(sc, "f32")
    d = {k: v.cpu() for k, v in g.get().items()}
    assert g.count() == g32.n == sc.n_foreground
    assert np.array_equal(_bits(d["mean"].numpy()), _bits(g32.mean))
    assert np.array_equal(_bits(d["cov"].numpy()), _bits(g32.cov))
    assert np.array_equal(_bits(d["opac"].numpy()), _bits(g32.opac))
    assert np.array_equal(_bits(d["feat"].float().numpy()), _bits(g32.feat))

    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    st = ctx.stats()
    assert st["n_pairs"] == bins.P and st["device_status"] == 0
    assert np.array_equal(ctx.export("rect").cpu().numpy(), pr.rect)
    assert np.array_equal(ctx.export("depthkey").cpu().numpy().view(np.uint32), pr.dkey)
    vis = pr.ntiles > 0
    assert np.array_equal(_bits(ctx.export("mean2d").cpu().numpy())[vis], _bits(pr.mu)[vis])
    assert np.array_equal(_bits(ctx.export("conic").cpu().numpy())[vis], _bits(pr.conic)[vis])
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)

    orc = O.render(g32, cam, PAR)
    stats = P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32)
    assert stats["n_flagged"] <= 1e-2 * stats["n_pixels"], stats
    if sc.feat_dtype == api.BF16:
        g_orig = O.lift_scene(sc, "f32", bf16_features=False)
        orc2 = O.render(g32, cam, PAR, feat64=g_orig.feat)
        P.compare_render(F, A, orc2, g32, cam, PAR, P.TOL_BF16, feat64=g_orig.feat)
    assert torch.isfinite(F).all() and float(A.min()) >= 0.0 and float(A.max()) <= 1.0
    return bins.P


def test_headline_full_size():
    sc = gen.scene_precision()
    assert sc.feat_dtype == api.BF16 and sc.C == 32 and len(sc.views) == 4
    assert _full_size(sc) > 4_500_000


def test_paper_shaped_fp32_full_size():
    sc = gen.scene_paper()
    assert sc.feat_dtype == api.F32 and sc.C == 32 and len(sc.views) == 2
    assert _full_size(sc) > 2_500_000
