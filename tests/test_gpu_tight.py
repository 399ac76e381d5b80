"""Tight binning (TSPLAT_RENDER_TIGHT) on the GPU against the oracle.

Bit-exact: the kept (tile, depth, id) pairs, the tile ranges and the counts
against the oracle's tight binning.  Within tolerance: the maps against the
FP64 oracle composite of the tight lists (1e-4), and against the GPU's own
full-rect render (1e-5: only the order of FP32 accumulation differs).  The
backward over tight lists gives the full-rect gradients.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu
PAR = O.params_array()
TIGHT = api.cparams(tight=True)


def _low_opacity_set():
    gs = gen.random_gaussians(31, 4000, 6, center=(0, 0, 1.2), spread=0.45, sigma_range=(0.001, 0.03))
    rng = np.random.default_rng(32)
    op = gs.opac.copy()
    op[rng.choice(len(op), 200, replace=False)] = rng.uniform(0.0005, 0.0039, 200).astype(np.float32)
    return O.Gaussians(gs.mean, gs.cov, op, gs.feat), gen.make_camera(120.0, 150, 100, (0, 0, 0), np.eye(3))


def _cases():
    out = {}
    tiny = gen.scene_tiny()
    out["tiny"] = (tiny, tiny.targets[0])
    paper = gen.scene_paper(seed=11, res=128, C=16)
    out["paper"] = (paper, gen.make_camera(150.0, 200, 136, (0.01, 0.0, -0.02), gen.rot_y(2.0)))
    prec = gen.scene_precision(seed=12, res=96, C=8)
    out["precision"] = (prec, gen.make_camera(120.0, 160, 120, (0, 0, 0), np.eye(3)))
    rig = gen.scene_paper_rig(seed=15, res=96, C=8, target_res=112)
    out["rig3"] = (rig, rig.targets[1])
    return out


CASES = _cases()


def _smooth(a, b, rel):
    a = a.detach().double().cpu().numpy()
    b = b.detach().double().cpu().numpy()
    rho = np.sqrt((b ** 2).mean()) + 1e-30
    return float(np.abs(a - b).max() / rho) <= rel


def _check(g, g32, cam, feat64=None):
    ctx = api.Context()
    F, A = ctx.render(g, cam, params=TIGHT)
    torch.cuda.synchronize()
    st = ctx.stats()
    pr = O.tighten(O.project_f32(g32, cam, PAR), g32.opac, cam.width, cam.height, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    full = O.bin_gaussians(O.project_f32(g32, cam, PAR), cam.width, cam.height)
    assert st["device_status"] == 0 and st["n_pairs"] == bins.P < full.P
    assert st["n_visible"] == int((pr.ntiles > 0).sum())
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    orc = O.render(g32, cam, PAR, tight=True)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32)
    F0, A0 = api.Context().render(g, cam)
    torch.cuda.synchronize()
    assert _smooth(F, F0, 1e-5) and _smooth(A, A0, 1e-5)
    return bins.P / full.P


@pytest.mark.parametrize("name", list(CASES))
def test_tight_bins_bitexact_and_maps(name):
    sc, cam = CASES[name]
    g, _ = P.gpu_build(sc)
    _check(g, O.lift_scene(sc, "f32"), cam)


def test_tight_low_opacity_and_anisotropic():
    g32, cam = _low_opacity_set()
    frac = _check(P.gpu_gaussians(g32), g32, cam)
    assert frac < 0.9


def test_tight_batched_equals_single():
    sc = gen.scene_paper_rig(seed=15, res=96, C=8, n_viewers=2, target_res=112)
    g, _ = P.gpu_build(sc)
    Fs, As = api.Context().render_batch(g, sc.targets, params=TIGHT)
    torch.cuda.synchronize()
    for cam, F, A in zip(sc.targets, Fs, As):
        F1, A1 = api.Context().render(g, cam, params=TIGHT)
        torch.cuda.synchronize()
        assert torch.equal(F, F1) and torch.equal(A, A1)


def test_tight_rasterize_equals_render():
    sc, cam = CASES["paper"]
    g, _ = P.gpu_build(sc)
    ctx = api.Context()
    F, A = ctx.render(g, cam, params=TIGHT)
    torch.cuda.synchronize()
    ref = api.Context()
    ref.render(g, cam)
    mean2d, conic = ref.export("mean2d"), ref.export("conic")
    radius = ref.export("radius").round().to(torch.int32)
    dk = ref.export("depthkey")
    depth = dk.view(torch.float32).clone()
    depth[dk == -1] = 0.0
    d = g.get()
    F2, A2 = api.Context().rasterize(mean2d, conic, d["opac"], depth, radius, d["feat"], cam.width, cam.height,
                                     params=TIGHT)
    torch.cuda.synchronize()
    assert torch.equal(F, F2) and torch.equal(A, A2)


def test_tight_backward_gives_full_rect_gradients():
    sc, cam = CASES["paper"]
    g, _ = P.gpu_build(sc)
    n = g.count()
    dF = torch.randn((sc.C, cam.height, cam.width), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    dA = torch.randn((cam.height, cam.width), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    grads = []
    for params in (None, api.cparams(tight=True)):
        ctx = api.Context()
        ctx.render(g, cam, params=params, save=True)
        grads.append(ctx.backward(dF, dA, n=n))
        torch.cuda.synchronize()
    for a, b in zip(*grads):
        assert _smooth(a, b, 1e-4)


def test_tight_full_size_headline():
    """1024^2 headline workload: every kept pair bit-exact, maps on sampled
    tiles, and the pair count the sort and composite see."""
    sc = gen.scene_precision()
    cam = sc.targets[0]
    g, _ = P.gpu_build(sc)
    g32 = O.lift_scene(sc, "f32")
    ctx = api.Context()
    F, A = ctx.render(g, cam, params=TIGHT)
    torch.cuda.synchronize()
    pr = O.tighten(O.project_f32(g32, cam, PAR), g32.opac, cam.width, cam.height, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    assert ctx.stats()["n_pairs"] == bins.P
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    rng = np.random.default_rng(29)
    tiles = sorted(set(np.argsort(-counts)[:8].tolist()) | set(rng.choice(len(counts), 8, replace=False).tolist()))
    orc = O.render(g32, cam, PAR, tiles=tiles, tight=True)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32, tiles=tiles)
