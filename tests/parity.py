"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle).

Error metric per output element: e = |g - r| / max(|r|, rho_c), with rho_c
the RMS over all pixels of the oracle's channel c (alpha: RMS of A).  A
pixel whose oracle decisions are ambiguous (a threshold met within the
oracle's margins) passes if the GPU matches any of its admissible outputs.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O
from paper_2405_14866_gb300 import api

# gates (FP32 features; BF16 stored features vs the oracle fed the original FP32)
TOL_F32 = 1e-4
TOL_BF16 = 2e-2


def device_views(scene):
    up = api.upload_scene(scene)
    keep = up["views"]
    views = [api.source_view(v["depth"], v["mask"], v["scale"], v["quat"], v["opacity"], v["feat"], v["cam"])
             for v in keep]
    return views, keep


def gpu_build(scene, feat_dtype=None):
    views, keep = device_views(scene)
    fd = scene.feat_dtype if feat_dtype is None else feat_dtype
    g = api.Gaussians.build(views, scene.C, fd)
    torch.cuda.synchronize()
    return g, keep


def gpu_gaussians(g32: O.Gaussians, feat_dtype=api.F32):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    return api.Gaussians.from_arrays(t(g32.mean), t(g32.cov), t(g32.opac), t(g32.feat), feat_dtype)


def rel_err(g, r, rho):
    return np.abs(g - r) / np.maximum(np.abs(r), rho)


def compare_render(F_gpu, A_gpu, orc: O.Render, g32: O.Gaussians, cam, par, tol, feat64=None, tiles=None,
                   max_unchecked_frac=1e-3):
    """Assert the GPU maps match the oracle render within `tol`; returns a
    dict of error statistics.  Only the listed tiles are compared when
    `tiles` is given (the oracle composited those tiles only)."""
    C, H, W = orc.comp.F.shape
    F = F_gpu.detach().cpu().numpy().astype(np.float64)
    A = A_gpu.detach().cpu().numpy().astype(np.float64)
    Fr, Ar = orc.comp.F, orc.comp.A
    mask = np.ones((H, W), bool)
    if tiles is not None:
        mask[:] = False
        tx = (W + 15) // 16
        for t in tiles:
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            mask[y0:y0 + 16, x0:x0 + 16] = True
    rho = np.sqrt((Fr[:, mask] ** 2).mean(axis=1)) + 1e-30
    rhoA = np.sqrt((Ar[mask] ** 2).mean()) + 1e-30
    eF = rel_err(F, Fr, rho[:, None, None])
    eA = rel_err(A, Ar, rhoA)
    flagged = (orc.comp.flags > 0) & mask
    plain = mask & ~flagged
    stats = dict(maxF=float(eF[:, plain].max(initial=0)), maxA=float(eA[plain].max(initial=0)),
                 rmsF=float(np.sqrt((eF[:, plain] ** 2).mean())) if plain.any() else 0.0,
                 n_flagged=int(flagged.sum()), n_pixels=int(mask.sum()))
    bad = np.argwhere((eF[:, plain].max(axis=0) > tol) | (eA[plain] > tol))
    assert stats["maxF"] <= tol and stats["maxA"] <= tol, (stats, bad[:5])
    # ambiguous pixels: one of the admissible outputs must match
    feat = np.ascontiguousarray(g32.feat if feat64 is None else feat64, np.float64)
    opac = np.ascontiguousarray(g32.opac, np.float64)
    unchecked = 0
    for (y, x) in np.argwhere(flagged):
        alts = O.pixel_alternatives(orc.mu64, orc.conic64, opac, feat, W, H, orc.bins, int(x), int(y), par)
        if alts is None:
            unchecked += 1
            continue
        cands = np.concatenate([np.concatenate([Fr[:, y, x], [Ar[y, x]]])[None], alts], 0)
        got = np.concatenate([F[:, y, x], [A[y, x]]])
        scale = np.maximum(np.abs(cands), np.concatenate([rho, [rhoA]])[None])
        err = (np.abs(cands - got[None]) / scale).max(axis=1)
        assert err.min() <= tol, ((y, x), err)
    stats["n_unchecked"] = unchecked
    assert unchecked <= max(2, max_unchecked_frac * stats["n_pixels"]), stats
    return stats
