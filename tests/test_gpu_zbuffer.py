"""Point z-buffer on the GPU against the oracle, bit for bit (depth bits and
ids): points lifted from the source views' depth maps, z-buffered into the
source cameras themselves (the round trip), into the other source cameras
(as the cascade's initial disparities at cam2/cam3, Sec. 4.1) and into the
novel view (the fused depth, Sec. 4.3)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu


def _check(g, mean, cam):
    ctx = api.Context()
    D, I = ctx.zbuffer(g, cam)
    torch.cuda.synchronize()
    d, i = O.zbuffer(mean, cam)
    assert np.array_equal(I.cpu().numpy(), i)
    assert np.array_equal(D.cpu().numpy().view(np.uint32), d.view(np.uint32))
    return int((i >= 0).sum())


@pytest.mark.parametrize("which", ["tiny", "paper", "precision"])
def test_zbuffer_matches_oracle(which):
    sc = {"tiny": gen.scene_tiny, "paper": lambda: gen.scene_paper(seed=13, res=128, C=4),
          "precision": lambda: gen.scene_precision(seed=14, res=96, C=4)}[which]()
    g, _ = P.gpu_build(sc)
    g32 = O.lift_scene(sc, "f32")
    hit = [_check(g, g32.mean, cam) for cam in [v.cam for v in sc.views] + list(sc.targets)]
    assert min(hit) > 0


def test_zbuffer_ties_culling_and_empty():
    cam = gen.make_camera(40.0, 48, 32, (0, 0, 0), np.eye(3))
    rng = np.random.default_rng(9)
    pts = np.concatenate([
        np.stack([rng.uniform(-0.5, 0.5, 400), rng.uniform(-0.3, 0.3, 400), rng.uniform(0.5, 2.0, 400)], 1),
        np.repeat([[0.01, 0.02, 1.0]], 5, axis=0),          # equal depths on one pixel: lowest id wins
        [[0.0, 0.0, -1.0], [0.0, 0.0, 0.1], [5.0, 0.0, 1.0]],  # behind, nearer than z_near, outside
    ]).astype(np.float32)
    n = len(pts)
    g32 = O.Gaussians(pts, np.tile(np.array([1e-4, 0, 0, 1e-4, 0, 1e-4], np.float32), (n, 1)),
                      np.full(n, 0.5, np.float32), np.zeros((n, 2), np.float32))
    g = P.gpu_gaussians(g32)
    _check(g, pts, cam)
    g0 = api.Gaussians.create(8, 2)
    D, I = api.Context().zbuffer(g0, cam)
    torch.cuda.synchronize()
    assert not D.any() and bool((I == -1).all())


def test_zbuffer_full_size():
    sc = gen.scene_precision()
    g, _ = P.gpu_build(sc)
    g32 = O.lift_scene(sc, "f32")
    for cam in (sc.targets[0], sc.views[2].cam):
        assert _check(g, g32.mean, cam) > 100000
