"""Edge cases of the render path on the GPU against the oracle.

- Every Gaussian at exactly the same depth: each bucket's order is the id
  order alone (one long run of equal keys); and two interleaved depths
  (heavy ties).  Pairs and ranges bit-exact.
- Buckets larger than the shared-memory sort: the depth-slab path, a slab
  beyond shared memory, and a bucket of a single depth.
- Zero covariances (the footprint is the low-pass filter alone).
- Non-finite depths and scales: culled by the projection as in the oracle.
- Limits: channel counts outside [1, 64], batches beyond 8 views.
- The tile order the kernels schedule by: a permutation of the tile slots,
  longest pair list first, empty tiles last.
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


def _check_tile_order(ctx, ranges):
    """The scheduling order: every tile slot once; tiles with pairs first,
    in falling pair count up to the width of a count bucket (a quarter
    octave; the device's log2 is approximate, hence the slack); then the
    tiles without pairs.  (The order within a bucket is not unique.)"""
    order = ctx.export("tile_order").cpu().numpy().view(np.uint32).astype(np.int64)
    T = ranges.shape[0]
    assert np.array_equal(np.sort(order), np.arange(T))
    cnt = (ranges[:, 1].astype(np.int64) - ranges[:, 0])[order]
    k = int((cnt > 0).sum())
    assert (cnt[:k] > 0).all() and (cnt[k:] == 0).all()
    c = cnt[:k].astype(np.float64)
    assert np.all(c[1:] <= c[:-1] * 2.0 ** 0.25 * 1.001 + 1.0)
    return k


def _check_bins_and_maps(g32, cam, tol=P.TOL_F32):
    g = P.gpu_gaussians(g32)
    ctx = api.Context()
    F, A = ctx.render(g, cam)
    torch.cuda.synchronize()
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    assert ctx.stats()["n_pairs"] == bins.P
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    _check_tile_order(ctx, bins.ranges)
    orc = O.render(g32, cam, PAR)
    P.compare_render(F, A, orc, g32, cam, PAR, tol)
    return bins


@pytest.mark.parametrize("n_depths", [1, 2])
def test_equal_depths_keep_id_order(n_depths):
    rng = np.random.default_rng(61)
    n = 20000 + 123                      # several sort tiles and a ragged tail
    z = np.where(np.arange(n) % n_depths == 0, 1.5, 1.25).astype(np.float32)
    mean = np.stack([rng.uniform(-0.6, 0.6, n) * z, rng.uniform(-0.6, 0.6, n) * z, z], 1).astype(np.float32)
    s = rng.uniform(0.001, 0.006, n).astype(np.float32)
    cov = np.zeros((n, 6), np.float32)
    cov[:, 0] = cov[:, 3] = cov[:, 5] = s * s
    cov[::7] = 0.0                       # zero covariance: the low-pass footprint alone
    opac = rng.uniform(0.3, 0.95, n).astype(np.float32)
    feat = rng.standard_normal((n, 4)).astype(np.float32)
    cam = gen.make_camera(200.0, 256, 240, (0, 0, 0), np.eye(3))
    bins = _check_bins_and_maps(O.Gaussians(mean, cov, opac, feat), cam)
    # within each tile the ids ascend per depth run
    ids, keys = bins.ids.astype(np.int64), bins.keys
    same = keys[1:] == keys[:-1]
    assert np.all(ids[1:][same] > ids[:-1][same]) and same.sum() > n


def test_nonfinite_maps_are_culled():
    sc = gen.scene_tiny(seed=62)
    v = sc.views[0]
    rng = np.random.default_rng(63)
    H, W = v.depth.shape
    idx = rng.choice(H * W, 300, replace=False)
    d = v.depth.reshape(-1).copy()
    d[idx[:100]] = np.nan
    d[idx[100:150]] = np.inf
    sc_ = v.scale.reshape(-1, 3).copy()
    sc_[idx[150:250], 1] = np.nan
    sc_[idx[250:], 0] = np.inf
    v.depth = d.reshape(H, W)
    v.scale = sc_.reshape(H, W, 3)
    g, keep = P.gpu_build(sc)
    g32 = O.lift_scene(sc, "f32")
    cam = sc.targets[0]
    ctx = api.Context()
    F, A = ctx.render(g, cam)
    torch.cuda.synchronize()
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    assert ctx.stats()["n_pairs"] == bins.P
    assert ctx.stats()["n_visible"] == int((pr.ntiles > 0).sum()) <= H * W - 300
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert torch.isfinite(F).all() and torch.isfinite(A).all()
    orc = O.render(g32, cam, PAR)
    P.compare_render(F, A, orc, g32, cam, PAR, P.TOL_F32)


def test_limits_are_rejected():
    for C in (0, 65):
        with pytest.raises(L.TsplatError) as e:
            api.Gaussians.create(16, C)
        assert e.value.status == 1
    gs = gen.random_gaussians(64, 500, 4, center=(0, 0, 1.5), spread=0.3)
    g = P.gpu_gaussians(O.Gaussians(gs.mean, gs.cov, gs.opac, gs.feat))
    cams = [gen.make_camera(60.0, 48 + 8 * k, 40, (0.01 * k, 0, 0), np.eye(3)) for k in range(9)]
    Fs, As = api.Context().render_batch(g, cams[:8])       # the largest batch
    torch.cuda.synchronize()
    for cam, F in zip(cams[:8], Fs):
        F1, _ = api.Context().render(g, cam)
        torch.cuda.synchronize()
        assert torch.equal(F, F1)
    with pytest.raises(L.TsplatError) as e:
        api.Context().render_batch(g, cams)
    assert e.value.status == 1


def test_runs_below_the_sorted_bits():
    """The shared-memory sort passes over the highest 16 significant bits of
    a tile's depth keys (here about 22), then orders each run of keys that
    agree on them by (key, id): clusters of 2 to 200 Gaussians whose depths
    lie within 100 ulps of each other (duplicates included) make runs both
    short enough for the in-place insertion and longer than 32 (the fallback
    to full passes).  Pairs and ranges bit-exact."""
    rng = np.random.default_rng(91)
    sizes = np.resize([2, 5, 20, 32, 33, 60, 200], 60)
    base = rng.uniform(1.0, 1.5, sizes.size).astype(np.float32).view(np.uint32)
    zb = np.concatenate([base[k] + rng.integers(0, 100, m).astype(np.uint32) for k, m in enumerate(sizes)])
    z = zb.view(np.float32)
    n = z.size
    perm = rng.permutation(n)                # cluster members spread over the id range
    z = z[perm]
    xy = rng.uniform(-0.05, 0.05, size=(n, 2)) * z[:, None]
    mean = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    cov = np.zeros((n, 6), np.float32)
    cov[:, 0] = cov[:, 3] = cov[:, 5] = (0.003 * z) ** 2
    opac = rng.uniform(0.02, 0.3, n).astype(np.float32)
    feat = rng.standard_normal((n, 2)).astype(np.float32)
    cam = gen.make_camera(300.0, 64, 48, (0, 0, 0), np.eye(3), cx=32.0, cy=24.0)
    bins = _check_bins_and_maps(O.Gaussians(mean, cov, opac, feat), cam)
    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    assert 1000 < counts.max() <= 3840     # the shared-memory path
    keys = bins.keys.astype(np.int64)
    assert (keys[1:] == keys[:-1]).sum() > 100   # duplicate keys: ties broken by id


@pytest.mark.parametrize("mix", ["spread", "one_slab_heavy", "all_equal"])
def test_buckets_beyond_shared_memory(mix):
    """15 K Gaussians on a few tiles: buckets larger than the shared-memory
    sort take the depth-slab path; a slab larger than shared memory (here a
    run of equal depths) and a bucket of one depth take global passes.
    Pairs and ranges bit-exact."""
    rng = np.random.default_rng(71)
    n = 15000
    if mix == "spread":
        z = rng.uniform(1.0, 2.0, n)
    elif mix == "one_slab_heavy":
        z = np.where(np.arange(n) % 3 == 0, rng.uniform(1.0, 2.0, n), 1.5)
    else:
        z = np.full(n, 1.5)
    z = z.astype(np.float32)
    xy = rng.normal(0.0, 0.004, size=(n, 2)) * z[:, None]
    mean = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    cov = np.zeros((n, 6), np.float32)
    cov[:, 0] = cov[:, 3] = cov[:, 5] = (0.002 * z) ** 2
    opac = rng.uniform(0.02, 0.2, n).astype(np.float32)
    feat = rng.standard_normal((n, 2)).astype(np.float32)
    cam = gen.make_camera(400.0, 64, 48, (0, 0, 0), np.eye(3), cx=40.0, cy=24.0)
    bins = _check_bins_and_maps(O.Gaussians(mean, cov, opac, feat), cam)
    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    assert counts.max() > 6144


@pytest.mark.parametrize("mix,n", [("spread", 60000), ("one_slab_heavy", 60000), ("clusters", 60000),
                                   ("spread", 12000), ("clusters", 12000)])
def test_wide_bucket_sort(mix, n):
    """More than 1500 instances of store capacity per tile slot (a store of
    capacity 60 K on the 16 tiles of a 64x64 view) select the bucket sort
    with twelve-warp blocks: with 60 K Gaussians every bucket exceeds shared
    memory (depth slabs, a slab of one depth, clusters of depths within 100
    ulps); with 12 K they are sorted in shared memory (runs below the sorted
    bits, in place and past the fallback).  Pairs and ranges bit-exact."""
    rng = np.random.default_rng(95)
    if mix == "spread":
        z = rng.uniform(1.0, 2.0, n).astype(np.float32)
    elif mix == "one_slab_heavy":
        z = np.where(np.arange(n) % 3 == 0, rng.uniform(1.0, 2.0, n), 1.5).astype(np.float32)
    else:
        base = rng.uniform(1.0, 1.5, n // 40).astype(np.float32).view(np.uint32)
        z = (np.repeat(base, 40) + rng.integers(0, 100, n).astype(np.uint32)).view(np.float32)
        z = z[rng.permutation(n)]
    xy = rng.uniform(-0.25, 0.25, size=(n, 2)) * z[:, None]
    mean = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    cov = np.zeros((n, 6), np.float32)
    cov[:, 0] = cov[:, 3] = cov[:, 5] = (0.002 * z) ** 2
    opac = rng.uniform(0.02, 0.2, n).astype(np.float32)
    feat = rng.standard_normal((n, 2)).astype(np.float32)
    g32 = O.Gaussians(mean, cov, opac, feat)
    cam = gen.make_camera(128.0, 64, 64, (0, 0, 0), np.eye(3))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    g = api.Gaussians.create(60000, 2)
    g.set(t(mean), t(cov), t(opac), t(feat))
    ctx = api.Context()
    F, A = ctx.render(g, cam)
    torch.cuda.synchronize()
    pr = O.project_f32(g32, cam, PAR)
    bins = O.bin_gaussians(pr, cam.width, cam.height)
    assert ctx.stats()["n_pairs"] == bins.P
    assert np.array_equal(ctx.export("pairs").cpu().numpy().view(np.uint32), bins.ids)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    P.compare_render(F, A, O.render(g32, cam, PAR), g32, cam, PAR, P.TOL_F32)
    counts = bins.ranges[:, 1].astype(np.int64) - bins.ranges[:, 0]
    assert (counts > 0).sum() == 16
    assert (counts.min() > 3840) if n == 60000 else (counts.max() <= 3840)


@pytest.mark.parametrize("res", [(64, 48), (1000, 776), (2048, 2048)])
def test_tile_order_is_longest_first_permutation(res):
    """One chunk of the scan (12 tiles, all with pairs, one of 18 K pairs),
    a ragged last chunk (3,087 tiles), and 16,384 tiles (4 chunks), on the
    oracle's bit-exact ranges."""
    W, H = res
    rng = np.random.default_rng(81)
    n = 30000
    z = rng.uniform(1.0, 3.0, n).astype(np.float32)
    # clustered means: tile counts from 0 to thousands
    ctr = rng.normal(0.0, 0.25, size=(n, 2)) * rng.choice([0.2, 1.0], size=(n, 1))
    mean = np.concatenate([ctr * z[:, None], z[:, None]], 1).astype(np.float32)
    s = rng.uniform(0.0005, 0.01, n).astype(np.float32)
    cov = np.zeros((n, 6), np.float32)
    cov[:, 0] = cov[:, 3] = cov[:, 5] = s * s
    g32 = O.Gaussians(mean, cov, rng.uniform(0.1, 0.9, n).astype(np.float32),
                      rng.standard_normal((n, 2)).astype(np.float32))
    cam = gen.make_camera(0.8 * W, W, H, (0, 0, 0), np.eye(3))
    g = P.gpu_gaussians(g32)  # the context reads the store's count until its next render
    ctx = api.Context()
    ctx.render(g, cam)
    torch.cuda.synchronize()
    bins = O.bin_gaussians(O.project_f32(g32, cam, PAR), W, H)
    assert np.array_equal(ctx.export("ranges").cpu().numpy().view(np.uint32), bins.ranges)
    k = _check_tile_order(ctx, bins.ranges)
    assert k > 0 and (W == 64 or k < bins.ranges.shape[0])
    del g
