"""tsplat_build_into_noalloc against tsplat_build_into, through the C ABI.

The allocation-free variant serves callers that may not allocate device
memory while they run (a fixed-budget frame loop, a process whose device
memory belongs to another allocator).  It must lift
exactly the same Gaussians as the regular call -- lifting is bit-exact, so
the comparison is too -- on two calls in a row, and refuse inputs beyond its
fixed scratch limit.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2405_14866_gb300 import _lib as L
from paper_2405_14866_gb300 import api, gen
from tests import parity as P

pytestmark = pytest.mark.gpu


def _lift_both(sc):
    views, keep = P.device_views(sc)
    cap = sum(v.depth.size for v in sc.views)
    ref = api.Gaussians.create(cap, sc.C, sc.feat_dtype)
    ref.build_into(views)
    na = api.Gaussians.create(cap, sc.C, sc.feat_dtype)
    na.build_into_noalloc(views)
    torch.cuda.synchronize()
    return ref, na


def test_noalloc_build_matches_build_on_two_calls():
    # two different workloads in a row: the shared scratch keeps the first
    # call's contents when the second one runs
    for sc in (gen.scene_paper(seed=21, res=96, C=16), gen.scene_precision(seed=22, res=72, C=8)):
        ref, na = _lift_both(sc)
        assert na.count() == ref.count() == sc.n_foreground
        a, b = ref.get(), na.get()
        for k in ("mean", "cov", "opac", "feat"):
            x, y = a[k].cpu(), b[k].cpu()
            assert torch.equal(x.view(torch.int16) if x.dtype == torch.bfloat16 else x.view(torch.int32),
                               y.view(torch.int16) if y.dtype == torch.bfloat16 else y.view(torch.int32)), k


def test_noalloc_build_rejects_inputs_beyond_its_scratch():
    dummy = torch.zeros(16, device="cuda")
    cam = gen.make_camera(100.0, 16000, 16000, (0, 0, 0), np.eye(3))  # 256 Mi pixels > 64 Mi limit
    v = api.source_view(dummy, None, dummy, None, dummy, dummy, cam, check=False)
    g = api.Gaussians.create(16, 4)
    with pytest.raises(L.TsplatError) as e:
        g.build_into_noalloc([v])
    assert e.value.status == 3 and "scratch limit" in str(e.value)
