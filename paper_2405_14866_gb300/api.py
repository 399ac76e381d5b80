"""Python surface of libtsplat: the C-ABI calls with torch tensors.

Every function marshals arguments (device pointers, sizes, the current CUDA
stream) and calls the library; all computation runs in its CUDA kernels.
PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _lib as L

F32, BF16 = L.F32, L.BF16
SERVER_NO_GRAPH = 1  # TSPLAT_SERVER_NO_GRAPH


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tsplat: tensors must live on the CUDA device")
    if not t.is_contiguous():
        raise ValueError("tsplat: tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def ccamera(cam) -> L.CCamera:
    """tsplat_camera from any object with fx, fy, cx, cy, width, height, R, t,
    z_near, z_far (e.g. gen.Camera)."""
    c = L.CCamera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.z_near, c.z_far = float(getattr(cam, "z_near", 0.2)), float(getattr(cam, "z_far", 1e4))
    return c


def cparams(lowpass=0.3, alpha_max=0.99, alpha_min=1.0 / 255.0, t_min=1e-4, frustum_clamp=1.3,
            save=False, async_=False, profile=False, tight=False) -> L.CParams:
    """tsplat_render_params; `tight` selects tight binning (TSPLAT_RENDER_TIGHT)."""
    p = L.CParams()
    p.lowpass, p.alpha_max, p.alpha_min, p.t_min, p.frustum_clamp = lowpass, alpha_max, alpha_min, t_min, frustum_clamp
    p.flags = ((L.RENDER_SAVE if save else 0) | (L.RENDER_ASYNC if async_ else 0) | (L.RENDER_PROFILE if profile else 0)
               | (L.RENDER_TIGHT if tight else 0))
    return p


def _with_flags(params: Optional[L.CParams], save: bool, async_: bool, profile: bool = False) -> L.CParams:
    if params is None:
        return cparams(save=save, async_=async_, profile=profile)
    p = L.CParams.from_buffer_copy(params)
    if save:
        p.flags |= L.RENDER_SAVE
    if async_:
        p.flags |= L.RENDER_ASYNC
    if profile:
        p.flags |= L.RENDER_PROFILE
    return p


def launch_count() -> int:
    """Kernel launches issued by libtsplat in this process."""
    return int(L.lib().tsplat_launch_count())


SRC_COMPACT = 1  # TSPLAT_SRC_COMPACT


def source_view(depth, mask, scale, quat, opacity, feat, cam, feat_dtype=None, compact=False,
                check=True) -> L.CSrcView:
    """tsplat_src_view from CUDA tensors (H,W), (H,W) u8 or None, (H,W,3),
    (H,W,4) or None, (H,W), (H,W,C) f32 or bf16 (feat_dtype defaults to the
    feature tensor's type).  compact=True: every map but the mask holds the
    foreground pixels only, in row-major order ((n_fg,), (n_fg,3), ...).
    The tensors must stay alive until the build has run.  check=False skips
    the shape checks (for tests of the library's own argument checks)."""
    H, W = int(cam.height), int(cam.width)
    if not check:
        pass
    elif mask is not None and tuple(mask.shape) != (H, W):
        raise ValueError(f"tsplat: mask shape {tuple(mask.shape)} != camera size ({H}, {W})")
    rows = H * W if not compact else None   # compact: the foreground count (checked by the shapes' agreement)
    n = depth.numel()
    if check and ((rows is not None and n != rows) or scale.numel() != 3 * n or opacity.numel() != n or
                  feat.numel() % max(n, 1) != 0 or (quat is not None and quat.numel() != 4 * n)):
        raise ValueError("tsplat: source maps do not match the camera size (or each other)")
    v = L.CSrcView()
    v.depth, v.mask, v.scale, v.quat = _ptr(depth), _ptr(mask), _ptr(scale), _ptr(quat)
    v.opacity, v.feat = _ptr(opacity), _ptr(feat)
    if feat_dtype is None:
        feat_dtype = BF16 if feat.dtype == torch.bfloat16 else F32
    v.feat_dtype = feat_dtype
    v.flags = SRC_COMPACT if compact else 0
    v.cam = ccamera(cam)
    return v


def upload_scene(scene, device="cuda", feat_dtype=F32, compact=False) -> Dict:
    """Copy a gen.Scene's per-view maps to the device (feature maps as FP32,
    or rounded to BF16 on the host with feat_dtype=BF16).  compact=True
    keeps only the foreground pixels' rows of every map but the mask (pass
    compact=True to source_view with these)."""
    views = []
    fdt = torch.bfloat16 if feat_dtype == BF16 else torch.float32
    for v in scene.views:
        fg = np.asarray(v.mask) != 0
        pick = (lambda a: a[fg]) if compact else (lambda a: a)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(pick(np.asarray(a))))
        views.append(dict(
            depth=t(v.depth).to(device),
            mask=torch.from_numpy(np.ascontiguousarray(v.mask)).to(device),
            scale=t(v.scale).to(device),
            quat=t(v.quat).to(device),
            opacity=t(v.opacity).to(device),
            feat=t(v.feat).to(fdt).to(device),
            cam=v.cam))
    return dict(views=views, C=scene.C, feat_dtype=scene.feat_dtype, compact=compact)


class Gaussians:
    """A library-owned, device-resident set of Gaussians (tsplat_gaussians)."""

    def __init__(self, handle: ctypes.c_void_p, C: int, feat_dtype: int, capacity: int):
        self.handle = handle
        self.C = C
        self.feat_dtype = feat_dtype
        self.capacity = capacity

    @classmethod
    def create(cls, capacity: int, C: int, feat_dtype: int = F32) -> "Gaussians":
        h = ctypes.c_void_p()
        L.call("tsplat_gaussians_create", capacity, C, feat_dtype, ctypes.byref(h))
        return cls(h, C, feat_dtype, capacity)

    @classmethod
    def from_arrays(cls, mean, cov, opac, feat, feat_dtype: int = F32, stream=None) -> "Gaussians":
        n, C = feat.shape
        g = cls.create(max(n, 1), C, feat_dtype)
        g.set(mean, cov, opac, feat, stream)
        return g

    def set(self, mean, cov, opac, feat, stream=None):
        n = mean.shape[0]
        din = BF16 if feat.dtype == torch.bfloat16 else F32
        if din == F32 and feat.dtype != torch.float32:
            raise ValueError("features must be float32 or bfloat16")
        L.call("tsplat_gaussians_set", self.handle, n, _ptr(mean), _ptr(cov), _ptr(opac), _ptr(feat), din, _stream(stream))

    @classmethod
    def build(cls, views: Sequence[L.CSrcView], C: int, feat_dtype: int = F32, stream=None) -> "Gaussians":
        arr = (L.CSrcView * len(views))(*views)
        h = ctypes.c_void_p()
        L.call("tsplat_build", arr, len(views), C, feat_dtype, ctypes.byref(h), _stream(stream))
        cap = sum(v.cam.width * v.cam.height for v in views)
        return cls(h, C, feat_dtype, cap)

    def build_into(self, views: Sequence[L.CSrcView], stream=None):
        arr = (L.CSrcView * len(views))(*views)
        L.call("tsplat_build_into", self.handle, arr, len(views), _stream(stream))

    def build_into_noalloc(self, views: Sequence[L.CSrcView], stream=None):
        """build_into without device allocation (fixed library scratch; see tsplat.h)."""
        arr = (L.CSrcView * len(views))(*views)
        L.call("tsplat_build_into_noalloc", self.handle, arr, len(views), _stream(stream))

    def build_backward(self, views: Sequence[L.CSrcView], d_mean3d, d_cov3d, d_opac, d_feat, stream=None):
        """Per-view gradients of the source maps this store was built from:
        a list of dicts depth (H,W), scale (H,W,3), quat (H,W,4) or None,
        opacity (H,W), feat (H,W,C)."""
        dev = torch.device("cuda")
        outs, structs = [], []
        for v in views:
            H, W = v.cam.height, v.cam.width
            o = dict(depth=torch.empty((H, W), device=dev), scale=torch.empty((H, W, 3), device=dev),
                     quat=torch.empty((H, W, 4), device=dev) if v.quat else None,
                     opacity=torch.empty((H, W), device=dev), feat=torch.empty((H, W, self.C), device=dev))
            outs.append(o)
            structs.append(L.CSrcGrads(_ptr(o["depth"]), _ptr(o["scale"]), _ptr(o["quat"]), _ptr(o["opacity"]),
                                       _ptr(o["feat"])))
        arr = (L.CSrcView * len(views))(*views)
        garr = (L.CSrcGrads * len(views))(*structs)
        L.call("tsplat_build_backward", self.handle, arr, len(views), _ptr(d_mean3d.contiguous()),
               _ptr(d_cov3d.contiguous()), _ptr(d_opac.contiguous()), _ptr(d_feat.contiguous()), garr, _stream(stream))
        return outs

    def count(self) -> int:
        n = ctypes.c_int64()
        L.call("tsplat_gaussians_count", self.handle, ctypes.byref(n))
        return int(n.value)

    def get(self, stream=None) -> Dict[str, torch.Tensor]:
        n = self.count()
        dev = torch.device("cuda")
        fdt = torch.bfloat16 if self.feat_dtype == BF16 else torch.float32
        out = dict(mean=torch.empty((n, 3), device=dev), cov=torch.empty((n, 6), device=dev),
                   opac=torch.empty((n,), device=dev), feat=torch.empty((n, self.C), device=dev, dtype=fdt))
        if n:
            L.call("tsplat_gaussians_get", self.handle, _ptr(out["mean"]), _ptr(out["cov"]), _ptr(out["opac"]),
                   _ptr(out["feat"]), _stream(stream))
        return out

    def close(self):
        if self.handle:
            L.lib().tsplat_gaussians_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Render context (tsplat_ctx): scratch of one stream + saved state."""

    def __init__(self):
        h = ctypes.c_void_p()
        L.call("tsplat_ctx_create", ctypes.byref(h))
        self.handle = h
        self.n = None
        # the context reads the last render's inputs (the store's count and
        # features) until its next render: hold them until then
        self._keep = ()
        self._last_shape = (0, 0, 0)  # (C, H, W) of the last single-view render

    def reserve(self, max_gaussians: int, max_pairs: int, max_width: int, max_height: int, C: int = 32):
        L.call("tsplat_ctx_reserve", self.handle, max_gaussians, max_pairs, max_width, max_height, C)

    def render(self, g: Gaussians, cam, params: Optional[L.CParams] = None, save=False, async_=False,
               out_feat=None, out_alpha=None, stream=None, profile=False):
        cc = ccamera(cam)
        W, H = cc.width, cc.height
        if out_feat is None:
            out_feat = torch.empty((g.C, H, W), device="cuda")
        if out_alpha is None:
            out_alpha = torch.empty((H, W), device="cuda")
        p = _with_flags(params, save, async_, profile)
        L.call("tsplat_render", g.handle, ctypes.byref(cc), ctypes.byref(p), _ptr(out_feat), _ptr(out_alpha),
               self.handle, _stream(stream))
        self.n = None
        self._keep = (g,)
        self._last_shape = (g.C, H, W)
        return out_feat, out_alpha

    def render_batch(self, g: Gaussians, cams, params: Optional[L.CParams] = None, async_=False, out_feat=None,
                     out_alpha=None, stream=None, profile=False):
        """Render several views of `g` in one pass; returns lists (F_v, A_v)."""
        K = len(cams)
        cc = (L.CCamera * K)(*[ccamera(c) for c in cams])
        if out_feat is None:
            out_feat = [torch.empty((g.C, c.height, c.width), device="cuda") for c in cc]
        if out_alpha is None:
            out_alpha = [torch.empty((c.height, c.width), device="cuda") for c in cc]
        fp = (ctypes.c_void_p * K)(*[t.data_ptr() for t in out_feat])
        ap = (ctypes.c_void_p * K)(*[t.data_ptr() for t in out_alpha])
        p = _with_flags(params, False, async_, profile)
        L.call("tsplat_render_batch", g.handle, cc, K, ctypes.byref(p), fp, ap, self.handle, _stream(stream))
        self.n = None
        self._keep = (g,)
        self._last_shape = (0, 0, 0)  # a batched render keeps no backward state
        return out_feat, out_alpha

    def rasterize(self, mean2d, conic, opac, depth, radius, feat, width: int, height: int,
                  params: Optional[L.CParams] = None, save=False, async_=False, out_feat=None, out_alpha=None,
                  stream=None):
        n, C = feat.shape
        dt = BF16 if feat.dtype == torch.bfloat16 else F32
        if out_feat is None:
            out_feat = torch.empty((C, height, width), device="cuda")
        if out_alpha is None:
            out_alpha = torch.empty((height, width), device="cuda")
        p = _with_flags(params, save, async_)
        L.call("tsplat_rasterize", n, _ptr(mean2d), _ptr(conic), _ptr(opac), _ptr(depth), _ptr(radius), _ptr(feat),
               C, dt, width, height, ctypes.byref(p), _ptr(out_feat), _ptr(out_alpha), self.handle, _stream(stream))
        self.n = n
        self._keep = (mean2d, conic, opac, depth, radius, feat)
        self._last_shape = (C, height, width)
        return out_feat, out_alpha

    def backward(self, dF, dA=None, n: Optional[int] = None, C: Optional[int] = None, stream=None, out=None):
        """Gradients (d_mean2d (N,2), d_conic (N,3), d_opac (N,), d_feat (N,C)); `out` = preallocated
        tensors of at least N rows (no synchronization then)."""
        # the library reads dF as C x H x W and dA as H x W FP32 of the last render
        C_r, H_r, W_r = self._last_shape
        if dF is None or tuple(dF.shape) != (C_r, H_r, W_r) or dF.dtype != torch.float32:
            raise ValueError(f"tsplat: dF must be float32 of shape {(C_r, H_r, W_r)}, got "
                             f"{None if dF is None else (tuple(dF.shape), dF.dtype)}")
        if dA is not None and (tuple(dA.shape) != (H_r, W_r) or dA.dtype != torch.float32):
            raise ValueError(f"tsplat: dA must be float32 of shape {(H_r, W_r)}, got {(tuple(dA.shape), dA.dtype)}")
        if out is not None:
            outs = tuple(out)
        else:
            st = self.stats()
            n = n if n is not None else (self.n if self.n is not None else st["n_gaussians"])
            C = C if C is not None else st["C"]
            dev = torch.device("cuda")
            outs = (torch.empty((n, 2), device=dev), torch.empty((n, 3), device=dev), torch.empty((n,), device=dev),
                    torch.empty((n, C), device=dev))
        L.call("tsplat_backward", self.handle, _ptr(dF.contiguous()), _ptr(None if dA is None else dA.contiguous()),
               *(_ptr(o) for o in outs), _stream(stream))
        return outs

    def backward_project(self, g: Gaussians, d_mean2d, d_conic, stream=None, out=None):
        """dL/dmean3d (cap,3), dL/dcov3d (cap,6) from the 2D gradients of the last
        render (tsplat_render with save=True) of `g`; `out` = preallocated pair."""
        dev = torch.device("cuda")
        if out is not None:
            dm, dc = out
        else:
            dm = torch.empty((g.capacity, 3), device=dev)
            dc = torch.empty((g.capacity, 6), device=dev)
        L.call("tsplat_backward_project", self.handle, g.handle, _ptr(d_mean2d.contiguous()),
               _ptr(d_conic.contiguous()), _ptr(dm), _ptr(dc), _stream(stream))
        return dm, dc

    def zbuffer(self, g: Gaussians, cam, out_depth=None, out_id=None, stream=None):
        """Point z-buffer of g's means in `cam`: (depth (H,W) f32, 0 where empty;
        id (H,W) int32, -1 where empty)."""
        cc = ccamera(cam)
        if out_depth is None:
            out_depth = torch.empty((cc.height, cc.width), device="cuda")
        if out_id is None:
            out_id = torch.empty((cc.height, cc.width), device="cuda", dtype=torch.int32)
        L.call("tsplat_zbuffer", g.handle, ctypes.byref(cc), _ptr(out_depth), _ptr(out_id), self.handle,
               _stream(stream))
        return out_depth, out_id

    def timings(self) -> Dict[str, float]:
        """Stage durations (ms) of the last profiled render (synchronizes)."""
        ms = (ctypes.c_float * len(L.STAGES))()
        n = ctypes.c_int32()
        L.call("tsplat_ctx_timings", self.handle, ms, len(L.STAGES), ctypes.byref(n))
        return {L.STAGES[i]: float(ms[i]) for i in range(n.value)}

    def stats(self) -> Dict[str, int]:
        s = L.CStats()
        L.call("tsplat_ctx_stats_get", self.handle, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in L.CStats._fields_}

    def status(self):
        L.call("tsplat_ctx_status", self.handle)

    def export(self, what: str) -> torch.Tensor:
        st = self.stats()
        n, P, T = st["n_gaussians"], st["n_pairs"], st["tiles_x"] * st["tiles_y"]
        shapes = {"rect": ((n, 4), torch.int32), "depthkey": ((n,), torch.int32), "mean2d": ((n, 2), torch.float32),
                  "conic": ((n, 3), torch.float32), "radius": ((n,), torch.float32),
                  "pairs": ((min(P, st["pair_capacity"]),), torch.int32), "ranges": ((T, 2), torch.int32),
                  "tfinal": ((st["height"], st["width"]), torch.float32), "last": ((st["height"], st["width"]), torch.int32),
                  "tile_order": ((T,), torch.int32)}  # a single-view render's slots
        shape, dt = shapes[what]
        t = torch.empty(shape, device="cuda", dtype=dt)
        nbytes = t.numel() * t.element_size()
        if nbytes:
            L.call("tsplat_ctx_export", self.handle, L.EXPORT[what], _ptr(t), nbytes, _stream())
        torch.cuda.current_stream().synchronize()
        return t

    def close(self):
        if self.handle:
            L.lib().tsplat_ctx_destroy(self.handle)
            self.handle = None
        self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching view server (tsplat_server): submit target views
    of the current frame; a worker thread batches them into CUDA-graph
    replays on up to `max_lanes` overlapping lanes."""

    def __init__(self, max_views_per_batch=8, max_lanes=3, max_width=1024, max_height=1024, max_gaussians=1 << 22,
                 C=32, feat_dtype=BF16, pairs_per_gaussian=2.5, pairs_per_pixel=1.0, budget_bytes=8 << 30,
                 params: Optional[L.CParams] = None,
                 graphs: bool = True, max_inflight_views: int = 0):
        cfg = L.CServerConfig()
        L.lib().tsplat_server_config_default(ctypes.byref(cfg))
        cfg.max_views_per_batch, cfg.max_lanes = max_views_per_batch, max_lanes
        cfg.max_width, cfg.max_height, cfg.max_gaussians = max_width, max_height, max_gaussians
        cfg.C, cfg.feat_dtype, cfg.pairs_per_pixel, cfg.budget_bytes = C, feat_dtype, pairs_per_pixel, budget_bytes
        cfg.pairs_per_gaussian = pairs_per_gaussian
        cfg.flags = 0 if graphs else SERVER_NO_GRAPH
        cfg.max_inflight_views = max_inflight_views
        if params is not None:
            cfg.params = params
        h = ctypes.c_void_p()
        L.call("tsplat_server_create", ctypes.byref(cfg), ctypes.byref(h))
        self.handle = h
        self.C = C

    def update_frame(self, g: Gaussians):
        L.call("tsplat_server_update_frame", self.handle, g.handle)

    def prepare(self, g: Gaussians, timeout_ms: float = 60000.0):
        """Capture the graphs of every batch size for the store `g` ahead of use."""
        L.call("tsplat_server_prepare", self.handle, g.handle, timeout_ms)

    def release_frame(self, g: Gaussians, timeout_ms: float = 30000.0):
        """Block until no batch in flight renders the (replaced) frame `g`."""
        L.call("tsplat_server_release_frame", self.handle, g.handle, timeout_ms)

    def submit(self, cam, out_feat, out_alpha=None) -> int:
        cc = cam if isinstance(cam, L.CCamera) else ccamera(cam)
        rid = ctypes.c_uint64()
        L.call("tsplat_server_submit", self.handle, ctypes.byref(cc), _ptr(out_feat), _ptr(out_alpha), ctypes.byref(rid))
        return int(rid.value)

    def poll(self, rid: int):
        """Latency in ms when done, else None."""
        lat = ctypes.c_double()
        st = L.lib().tsplat_server_poll(self.handle, rid, ctypes.byref(lat))
        if st == 6:
            return None
        if st != 0:
            raise L.TsplatError("tsplat_server_poll", st, L.lib().tsplat_last_error().decode())
        return float(lat.value)

    def wait(self, rid: int, timeout_ms: float = 30000.0) -> float:
        lat = ctypes.c_double()
        L.call("tsplat_server_wait", self.handle, rid, timeout_ms, ctypes.byref(lat))
        return float(lat.value)

    def stats(self) -> Dict[str, float]:
        s = L.CServerStats()
        L.call("tsplat_server_get_stats", self.handle, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in L.CServerStats._fields_ if k != "reserved"}

    def reset_stats(self):
        L.call("tsplat_server_reset_stats", self.handle)

    def close(self):
        if self.handle:
            L.lib().tsplat_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
