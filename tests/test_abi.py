"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/tsplat.h declares (no GPU work: host-only calls)."""
import ctypes
import os
import re
import subprocess

from paper_2405_14866_gb300 import _lib as L
from paper_2405_14866_gb300 import build as B

HEADERS = [os.path.join(B.ROOT, "include", f) for f in sorted(os.listdir(os.path.join(B.ROOT, "include")))
           if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(tsplat_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tsplat_\w+)", out))
    assert set(names) <= exported


def test_binding_signatures_cover_the_header():
    assert set(declared()) == set(L.declared_symbols())


def test_struct_layouts_match_header():
    assert ctypes.sizeof(L.CCamera) == 4 * 4 + 2 * 4 + 9 * 4 + 3 * 4 + 2 * 4
    assert ctypes.sizeof(L.CParams) == 6 * 4
    assert ctypes.sizeof(L.CSrcView) == 6 * 8 + 2 * 4 + ctypes.sizeof(L.CCamera)


def test_host_only_calls():
    lib = L.lib()
    p = L.CParams()
    lib.tsplat_render_params_default(ctypes.byref(p))
    assert abs(p.lowpass - 0.3) < 1e-7 and abs(p.alpha_max - 0.99) < 1e-7
    assert abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.t_min - 1e-4) < 1e-10 and p.flags == 0
    assert b"sm_103a" in lib.tsplat_version()


def test_invalid_arguments_are_rejected_without_device_work():
    lib = L.lib()
    h = ctypes.c_void_p()
    assert lib.tsplat_gaussians_create(10, 0, 0, ctypes.byref(h)) == 1      # C = 0
    assert b"C = 0" in lib.tsplat_last_error()
    assert lib.tsplat_gaussians_create(10, 8, 7, ctypes.byref(h)) == 1      # bad dtype
    assert lib.tsplat_build(None, 1, 8, 0, ctypes.byref(h), None) == 1
    assert lib.tsplat_backward(None, None, None, None, None, None, None, None) == 1


def test_sources_use_no_multicast_and_no_trap():
    bad = re.compile(r"multicast|__trap|asm\s*\(\s*\"trap")
    for src in B.sources():
        assert not bad.search(open(src).read()), src


def test_binding_constants_match_header():
    """The binding's enum values (feature types, render flags, source-view
    flags, export items) and its count of timed stages are the header's."""
    src = "\n".join(open(h).read() for h in HEADERS)
    exports = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"TSPLAT_EXPORT_(\w+) = (\d+)", src)}
    assert exports == L.EXPORT
    flags = {m.group(1): 1 << int(m.group(2)) for m in re.finditer(r"TSPLAT_RENDER_(\w+) = 1u << (\d+)", src)}
    assert flags == {"ASYNC": L.RENDER_ASYNC, "SAVE": L.RENDER_SAVE, "PROFILE": L.RENDER_PROFILE,
                     "TIGHT": L.RENDER_TIGHT}
    assert re.search(r"TSPLAT_F32 = (\d+), TSPLAT_BF16 = (\d+)", src).groups() == (str(L.F32), str(L.BF16))
    from paper_2405_14866_gb300 import api
    assert int(re.search(r"TSPLAT_SRC_COMPACT = (\d+)", src).group(1)) == api.SRC_COMPACT
    assert int(re.search(r"\*n_out = (\d+)", src).group(1)) == len(L.STAGES)


def test_product_path_fails_loudly_without_a_gpu():
    """No CPU fallback: without a CUDA device the product calls raise."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2405_14866_gb300 import api
    with pytest.raises(L.TsplatError):
        api.Context()
    with pytest.raises(L.TsplatError):
        api.Gaussians.create(16, 4)


def test_context_holds_the_last_render_inputs(monkeypatch):
    """A context keeps the store it last rendered (and a rasterize call's
    arrays) until its next render, so a temporary store passed to render is
    not freed while the context still reads its count and features.  The C
    calls are stubbed: this is the binding's own bookkeeping."""
    import gc
    import weakref

    import numpy as np
    import torch

    from paper_2405_14866_gb300 import api, gen
    calls = []
    monkeypatch.setattr(L, "call", lambda name, *a: calls.append(name))
    monkeypatch.setattr(api, "_ptr", lambda t: None)
    monkeypatch.setattr(api, "_stream", lambda s=None: None)

    class Store:
        C, handle = 2, None

    cam = gen.make_camera(10.0, 8, 8, (0, 0, 0), np.eye(3))
    F, A = torch.empty(2, 8, 8), torch.empty(8, 8)
    ctx = api.Context()
    s = Store()
    ref = weakref.ref(s)
    ctx.render(s, cam, out_feat=F, out_alpha=A)
    del s
    gc.collect()
    assert ref() is not None                      # held by the context
    ctx.render_batch(Store(), [cam], out_feat=[F], out_alpha=[A])
    gc.collect()
    assert ref() is None                          # released by the next render
    feat = torch.empty(5, 2)
    fref = weakref.ref(feat)
    ctx.rasterize(torch.empty(5, 2), torch.empty(5, 3), torch.empty(5), torch.empty(5), torch.empty(5), feat,
                  8, 8, out_feat=F, out_alpha=A)
    del feat
    gc.collect()
    assert fref() is not None
    ctx.close()
    gc.collect()
    assert fref() is None
    assert calls.count("tsplat_render") == 1 and calls.count("tsplat_render_batch") == 1


def test_backward_rejects_gradients_of_the_wrong_shape(monkeypatch):
    """tsplat_backward reads a C x H x W dF and an H x W dA of the last render
    through plain pointers, so the binding checks their shapes and types before
    the call (a short buffer would be read out of bounds on the device).  The C
    calls are stubbed: this is the binding's own check."""
    import numpy as np
    import pytest
    import torch

    from paper_2405_14866_gb300 import api, gen
    from paper_2405_14866_gb300.autograd import SplatFn
    calls = []
    monkeypatch.setattr(L, "call", lambda name, *a: calls.append(name))
    monkeypatch.setattr(api, "_ptr", lambda t: None)
    monkeypatch.setattr(api, "_stream", lambda s=None: None)

    class Store:
        C, handle = 3, None

    cam = gen.make_camera(10.0, 8, 6, (0, 0, 0), np.eye(3))
    ctx = api.Context()
    ctx.render(Store(), cam, out_feat=torch.empty(3, 6, 8), out_alpha=torch.empty(6, 8), save=True)
    outs = tuple(torch.empty(s) for s in ((4, 2), (4, 3), (4,), (4, 3)))
    for dF, dA in ((torch.zeros(3, 1, 1), None), (torch.zeros(2, 6, 8), None), (torch.zeros(3, 8, 6), None),
                   (torch.zeros(3, 6, 8, dtype=torch.float64), None), (torch.zeros(3, 6, 8), torch.zeros(8, 6)),
                   (None, torch.zeros(6, 8))):
        with pytest.raises(ValueError):
            ctx.backward(dF, dA, out=outs)
    assert "tsplat_backward" not in calls
    ctx.backward(torch.zeros(3, 6, 8), torch.zeros(6, 8), out=outs)
    assert calls.count("tsplat_backward") == 1
    # a batched render keeps no backward state: any gradient is refused
    ctx.render_batch(Store(), [cam], out_feat=[torch.empty(3, 6, 8)], out_alpha=[torch.empty(6, 8)])
    with pytest.raises(ValueError):
        ctx.backward(torch.zeros(3, 6, 8), None, out=outs)

    # SplatFn: a loss that uses only A gives dF = None; the backward supplies
    # a whole C x H x W zero gradient, not a 1 x 1 one
    class Ctx:
        pass
    seen = {}

    grads = (torch.zeros(4, 2), torch.zeros(4, 3), torch.zeros(4), torch.zeros(4, 3))

    class FakeContext:
        def backward(self, dF, dA, n, C):
            seen["dF"], seen["dA"] = tuple(dF.shape), tuple(dA.shape)
            return grads

    c = Ctx()
    c.context, c.n, c.C, c.hw, c.feat_dtype = FakeContext(), 4, 3, (6, 8), torch.float32
    monkeypatch.setattr(torch, "zeros", lambda shape, device=None, **k: torch.empty(shape).fill_(0.0))
    SplatFn.backward(c, None, torch.ones(6, 8))
    assert seen["dF"] == (3, 6, 8) and seen["dA"] == (6, 8)
