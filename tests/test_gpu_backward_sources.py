"""Backward through the projection and the lifting on the GPU against the
FP64 oracle adjoints, fed the same upstream gradients: the GPU's dL/dmean2d
and dL/dconic go into both implementations of the projection adjoint, and
the GPU's dL/dmean3d, dL/dcov3d, dL/dopacity and dL/dfeature into both
implementations of the lifting adjoint (per source view).  Metric per
output group: e = |g - r| / max(|r|, rho), rho = RMS of the oracle's group;
gate 1e-3 (single precision against double)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _close(name, g, r):
    g = np.asarray(g, np.float64).reshape(r.shape)
    rho = np.sqrt((r ** 2).mean()) + 1e-30
    e = np.abs(g - r) / np.maximum(np.abs(r), rho)
    assert e.max() <= TOL, (name, float(e.max()), np.unravel_index(e.argmax(), e.shape))


# two small cases, and one sample of the differentiation workload at the size
# the benchmark times (2 x 512^2 sources, ~315K Gaussians, 16 channels)
@pytest.mark.parametrize("seed,res,C", [(61, 64, 4), (62, 64, 4), (300, 512, 16)])
def test_backward_to_source_maps(seed, res, C):
    sc = gen.scene_diff_sample(seed=seed, res=res, C=C)
    cam = (gen.make_camera(60.0, 64, 56, (0.02, -0.01, 0.0), gen.rot_y(2.0)) if res == 64 else sc.targets[0])
    views, keep = P.device_views(sc)
    g = api.Gaussians.build(views, sc.C, api.F32)
    ctx = api.Context()
    F, A = ctx.render(g, cam, save=True)
    rng = np.random.default_rng(seed)
    dF = torch.from_numpy(rng.standard_normal(F.shape).astype(np.float32)).cuda()
    dA = torch.from_numpy(rng.standard_normal(A.shape).astype(np.float32)).cuda()
    d_mu, d_con, d_op, d_ft = ctx.backward(dF, dA)
    d_mean, d_cov = ctx.backward_project(g, d_mu, d_con)
    torch.cuda.synchronize()
    g32 = O.lift_scene(sc, "f32")
    n = g32.n
    gm_ref, gc_ref = O.project_backward(g32.mean, g32.cov, cam, d_mu.cpu().numpy().astype(np.float64),
                                        d_con.cpu().numpy().astype(np.float64))
    assert np.abs(gm_ref).max() > 0 and np.abs(gc_ref).max() > 0
    _close("d_mean3d", d_mean[:n].cpu().numpy(), gm_ref)
    _close("d_cov3d", d_cov[:n].cpu().numpy(), gc_ref)

    grads = g.build_backward(views, d_mean, d_cov, d_op, d_ft)
    torch.cuda.synchronize()
    gm64, gc64 = d_mean[:n].cpu().numpy().astype(np.float64), d_cov[:n].cpu().numpy().astype(np.float64)
    op64, ft64 = d_op[:n].cpu().numpy().astype(np.float64), d_ft[:n].cpu().numpy().astype(np.float64)
    off = 0
    for v, got in zip(sc.views, grads):
        k = int(v.mask.sum())
        ref = O.lift_backward(v, gm64[off:off + k], gc64[off:off + k], op64[off:off + k], ft64[off:off + k])
        off += k
        _close("depth", got["depth"].cpu().numpy(), ref["depth"])
        _close("scale", got["scale"].cpu().numpy(), ref["scale"])
        _close("quat", got["quat"].cpu().numpy(), ref["quat"])
        assert np.array_equal(got["opacity"].cpu().numpy().astype(np.float64), ref["opacity"])
        assert np.array_equal(got["feat"].cpu().numpy().astype(np.float64), ref["feat"])
    assert off == n
