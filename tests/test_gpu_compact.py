"""Source views with compact maps (TSPLAT_SRC_COMPACT): only the foreground
pixels' rows of the depth, scale, quaternion, opacity and feature maps.

The lifted store must equal, bit for bit, the store lifted from the full
maps and the oracle's key-mode lifting, including views whose pixel counts
are not multiples of the lifting block (ragged block layout per view)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import _lib as L
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu


def _views(sc, compact, feat_dtype):
    up = api.upload_scene(sc, feat_dtype=feat_dtype, compact=compact)
    vs = [api.source_view(v["depth"], v["mask"], v["scale"], v["quat"], v["opacity"], v["feat"], v["cam"],
                          compact=compact) for v in up["views"]]
    return vs, up


def _mixed_scene():
    """Three views of different, ragged sizes (100x100, 60x61, 96x90)."""
    a = gen.scene_paper(seed=41, res=100, C=8)
    b = gen.scene_tiny(seed=42, res=64, C=8)
    c = gen.scene_precision(seed=43, res=96, C=8)
    views = [a.views[0], b.views[0], c.views[2]]
    cut = [(100, 100), (61, 60), (90, 96)]
    out = []
    for v, (H, W) in zip(views, cut):
        cam = gen.Camera(v.cam.fx, v.cam.fy, v.cam.cx, v.cam.cy, W, H, v.cam.R, v.cam.t, v.cam.z_near, v.cam.z_far)
        out.append(gen.SourceView(v.depth[:H, :W], v.mask[:H, :W], v.scale[:H, :W], v.quat[:H, :W],
                                  v.opacity[:H, :W], v.feat[:H, :W], cam))
    return gen.Scene("mixed-ragged", out, a.targets, 8, gen.FEAT_F32, 41)


CASES = {"tiny": gen.scene_tiny(), "paper": gen.scene_paper(seed=11, res=128, C=16),
         "precision": gen.scene_precision(seed=12, res=96, C=8), "mixed": _mixed_scene()}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("feat_dtype", [api.F32, api.BF16])
def test_compact_build_equals_full_and_oracle(name, feat_dtype):
    sc = CASES[name]
    g32 = O.lift_scene(sc, "f32", bf16_features=feat_dtype == api.BF16)
    stores = []
    for compact in (False, True):
        vs, keep = _views(sc, compact, feat_dtype)
        g = api.Gaussians.build(vs, sc.C, feat_dtype)
        torch.cuda.synchronize()
        assert g.count() == g32.n == sc.n_foreground
        stores.append({k: v.cpu() for k, v in g.get().items()})
    for k in stores[0]:
        assert torch.equal(stores[0][k], stores[1][k]), k
    d = stores[1]
    bits = lambda a: np.ascontiguousarray(a, np.float32).view(np.uint32)
    assert np.array_equal(bits(d["mean"].numpy()), bits(g32.mean))
    assert np.array_equal(bits(d["cov"].numpy()), bits(g32.cov))
    assert np.array_equal(bits(d["opac"].numpy()), bits(g32.opac))
    assert np.array_equal(bits(d["feat"].float().numpy()), bits(g32.feat))


def test_compact_renders_the_same_view():
    sc = CASES["paper"]
    cam = gen.make_camera(150.0, 200, 136, (0.01, 0.0, -0.02), gen.rot_y(2.0))
    out = []
    for compact in (False, True):
        vs, keep = _views(sc, compact, api.F32)
        g = api.Gaussians.build(vs, sc.C, api.F32)
        F, A = api.Context().render(g, cam)
        torch.cuda.synchronize()
        out.append((F, A))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_compact_rejections():
    sc = CASES["tiny"]
    vs, keep = _views(sc, True, api.F32)
    g = api.Gaussians.build(vs, sc.C, api.F32)
    torch.cuda.synchronize()
    n = g.count()
    dm = torch.zeros((g.capacity, 3), device="cuda")
    dc = torch.zeros((g.capacity, 6), device="cuda")
    do = torch.zeros((g.capacity,), device="cuda")
    df = torch.zeros((g.capacity, sc.C), device="cuda")
    with pytest.raises(L.TsplatError) as e:
        g.build_backward(vs, dm, dc, do, df)
    assert e.value.status == 7 and n > 0
    with pytest.raises(L.TsplatError) as e:
        g.build_into_noalloc(vs)
    assert e.value.status == 7
    # compact maps need a mask
    v0 = keep["views"][0]
    bad = api.source_view(v0["depth"], None, v0["scale"], v0["quat"], v0["opacity"], v0["feat"], v0["cam"],
                          compact=True)
    with pytest.raises(L.TsplatError) as e:
        g.build_into([bad])
    assert e.value.status == 1
