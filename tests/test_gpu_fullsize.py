"""The 1024x1024 headline workload at full size, in the launch
configuration bench.py times (lifting into an existing store, asynchronous
render into a reserved context, BF16 source feature maps).

Bit-exact over every Gaussian and pair: the lifted store, the projected
record, tile rects, depth keys and the (tile, depth, id) order.  The
feature and alpha maps are compared on sampled tiles (the 12 tiles with the
most pairs and 12 seeded random ones) that the FP64 oracle composites one by
one: 1e-4 against the oracle fed the stored BF16 features, 2e-2 against the
oracle fed the original FP32 features.
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


def test_headline_full_size():
    sc = gen.scene_precision()
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

    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    rng = np.random.default_rng(17)
    tiles = sorted(set(np.argsort(-counts)[:12].tolist()) | set(rng.choice(len(counts), 12, replace=False).tolist()))
    orc = O.render(g32, cam, PAR, tiles=tiles)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32, tiles=tiles)
    g_orig = O.lift_scene(sc, "f32", bf16_features=False)
    orc2 = O.render(g32, cam, PAR, tiles=tiles, feat64=g_orig.feat)
    P.compare_render(F, A, orc2, g32, cam, PAR, P.TOL_BF16, feat64=g_orig.feat, tiles=tiles)
    # properties over the whole map: alpha in [0, 1], finite features
    assert torch.isfinite(F).all() and float(A.min()) >= 0.0 and float(A.max()) <= 1.0
