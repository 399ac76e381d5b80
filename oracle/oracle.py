"""Python front end of the FP64 CPU oracle (``tsplat_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the library path.  It
shares no code with the CUDA library; both are fed the same arrays from the
seeded generator.

Every function follows the step of Tele-Aloha Sec. 4.2 (lifting of
foreground pixels with the camera, render equation F = R_G({G}, Pi_novel)
with the cited 3DGS rasterizer) that is documented beside its C counterpart.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsplat_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_tsplat.so")
# an alternative build of the oracle (used to check that the pins catch
# planted mistakes); when set, no build is attempted
_SO_OVERRIDE = os.environ.get("TSPLAT_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

# default render parameters (the 3DGS rasterizer's constants)
LOWPASS, ALPHA_MAX, ALPHA_MIN, T_MIN, FRUSTUM_CLAMP = 0.3, 0.99, 1.0 / 255.0, 1e-4, 1.3
TILE = 16
# relative margins under which a discrete decision counts as ambiguous
MARGIN_ALPHA, MARGIN_T, MARGIN_Q = 2e-5, 5e-4, 1e-5

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(_SO_OVERRIDE or build())
            _lib.orc_lift_f64.restype = ctypes.c_int64
            _lib.orc_lift_f32.restype = ctypes.c_int64
            _lib.orc_scan.restype = ctypes.c_int64
            _lib.orc_tile_list_bruteforce.restype = ctypes.c_int64
            _lib.orc_pixel_alternatives.restype = ctypes.c_int
            _lib.orc_num_threads.restype = ctypes.c_int
            _lib.orc_key_ln_f32.restype = ctypes.c_float
            _lib.orc_key_ln_f32.argtypes = [ctypes.c_float]
    return _lib


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return ctypes.c_void_p(a.ctypes.data)


def _i64(x):
    return ctypes.c_int64(int(x))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def cam_array(cam) -> np.ndarray:
    """Camera as float32[20]: fx fy cx cy W H R[9] t[3] z_near z_far."""
    a = np.empty(20, np.float32)
    a[0:6] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height]
    a[6:15] = np.asarray(cam.R, np.float32).reshape(9)
    a[15:18] = np.asarray(cam.t, np.float32).reshape(3)
    a[18:20] = [cam.z_near, cam.z_far]
    return a


def params_array(lowpass=LOWPASS, alpha_max=ALPHA_MAX, alpha_min=ALPHA_MIN, t_min=T_MIN,
                 frustum_clamp=FRUSTUM_CLAMP) -> np.ndarray:
    return np.array([lowpass, alpha_max, alpha_min, t_min, frustum_clamp], np.float32)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().orc_round_bf16(_i64(x.size), _p(x), _p(out))
    return out


# ---------------------------------------------------------------------------
# lifting
# ---------------------------------------------------------------------------

@dataclass
class Gaussians:
    mean: np.ndarray   # (N,3)
    cov: np.ndarray    # (N,6)
    opac: np.ndarray   # (N,)
    feat: np.ndarray   # (N,C)

    @property
    def n(self):
        return self.mean.shape[0]

    def astype(self, dt):
        return Gaussians(self.mean.astype(dt), self.cov.astype(dt), self.opac.astype(dt), self.feat.astype(dt))


def lift_view(view, prec: str = "f32") -> Gaussians:
    """Lift the foreground pixels of one source view (Sec. 4.2)."""
    H, W = view.depth.shape
    C = view.feat.shape[2]
    n_max = int(view.mask.sum()) if view.mask is not None else H * W
    dt = np.float64 if prec == "f64" else np.float32
    mean = np.empty((n_max, 3), dt)
    cov = np.empty((n_max, 6), dt)
    op = np.empty((n_max,), dt)
    ft = np.empty((n_max, C), dt)
    depth = np.ascontiguousarray(view.depth, np.float32)
    mask = None if view.mask is None else np.ascontiguousarray(view.mask, np.uint8)
    scale = np.ascontiguousarray(view.scale, np.float32)
    quat = None if view.quat is None else np.ascontiguousarray(view.quat, np.float32)
    opac = np.ascontiguousarray(view.opacity, np.float32)
    feat = np.ascontiguousarray(view.feat, np.float32)
    cam = cam_array(view.cam)
    fn = lib().orc_lift_f64 if prec == "f64" else lib().orc_lift_f32
    n = fn(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_int(C), _p(depth), _p(mask), _p(scale), _p(quat),
           _p(opac), _p(feat), _p(cam), _p(mean), _p(cov), _p(op), _p(ft))
    assert n == n_max
    return Gaussians(mean, cov, op, ft)


def lift_scene(scene, prec: str = "f32", bf16_features: Optional[bool] = None) -> Gaussians:
    """Lift all views; Gaussian ids follow (view, row, column) order.  With
    BF16 storage the features are rounded to BF16 (kept as float32)."""
    parts = [lift_view(v, prec) for v in scene.views]
    g = Gaussians(*(np.concatenate([getattr(p, k) for p in parts], 0)
                    for k in ("mean", "cov", "opac", "feat")))
    if bf16_features is None:
        bf16_features = scene.feat_dtype == 1
    if bf16_features and prec == "f32":
        g.feat = round_bf16(g.feat)
    return g


# ---------------------------------------------------------------------------
# projection (key mode in FP32, values in FP64)
# ---------------------------------------------------------------------------

@dataclass
class Projected:
    rect: np.ndarray     # (N,4) int32
    ntiles: np.ndarray   # (N,) int32
    dkey: np.ndarray     # (N,) uint32
    radius: np.ndarray   # (N,) float32
    mu: np.ndarray       # (N,2) float32
    conic: np.ndarray    # (N,3) float32
    mask: Optional[np.ndarray] = None   # (N,) uint32 kept-tile masks (tight binning)


def project_f32(g32: Gaussians, cam, par=None) -> Projected:
    par = params_array() if par is None else par
    n = g32.n
    mean = np.ascontiguousarray(g32.mean, np.float32)
    cov = np.ascontiguousarray(g32.cov, np.float32)
    out = Projected(np.empty((n, 4), np.int32), np.empty(n, np.int32), np.empty(n, np.uint32),
                    np.empty(n, np.float32), np.empty((n, 2), np.float32), np.empty((n, 3), np.float32))
    lib().orc_project_f32(_i64(n), _p(mean), _p(cov), _p(cam_array(cam)), _p(par),
                          _p(out.rect), _p(out.ntiles), _p(out.dkey), _p(out.radius), _p(out.mu), _p(out.conic))
    return out


def key_ln(x: float) -> float:
    """ln x (x >= 1) in key mode, as the tight binning evaluates it."""
    return float(lib().orc_key_ln_f32(ctypes.c_float(x)))


def tighten(proj: Projected, opac: np.ndarray, width: int, height: int, par=None) -> Projected:
    """Tight binning: keep only the tiles of each rect (of at most 32 tiles)
    whose pixel-centre rectangle reaches Q <= 2 ln(o / alpha_min) (with a
    rounding margin).  Returns a copy whose ntiles count the kept tiles and
    whose mask holds them; Gaussians left with no tile are culled."""
    par = params_array() if par is None else par
    n = proj.rect.shape[0]
    out = Projected(proj.rect.copy(), proj.ntiles.copy(), proj.dkey.copy(), proj.radius.copy(), proj.mu.copy(),
                    proj.conic.copy(), np.empty(n, np.uint32))
    lib().orc_tight_tiles_f32(_i64(n), _p(out.rect), _p(out.mu), _p(out.conic),
                              _p(np.ascontiguousarray(opac, np.float32)), _p(par), ctypes.c_int(width),
                              ctypes.c_int(height), _p(out.mask), _p(out.ntiles))
    gone = (proj.ntiles > 0) & (out.ntiles == 0)
    out.rect[gone] = 0
    out.dkey[gone] = 0xFFFFFFFF
    out.radius[gone] = 0
    out.mu[gone] = 0
    out.conic[gone] = 0
    return out


def project_backward(mean, cov, cam, g_mu, g_conic, par=None):
    """Adjoint of project_f64: (dL/dmean (N,3), dL/dcov (N,6)) from dL/dmu (N,2)
    and dL/dconic (N,3)."""
    par = params_array() if par is None else par
    mean = np.ascontiguousarray(mean, np.float64)
    cov = np.ascontiguousarray(cov, np.float64)
    n = mean.shape[0]
    gm = np.empty((n, 3)); gc = np.empty((n, 6))
    lib().orc_project_backward_f64(_i64(n), _p(mean), _p(cov), _p(cam_array(cam)), _p(par),
                                   _p(np.ascontiguousarray(g_mu, np.float64)),
                                   _p(np.ascontiguousarray(g_conic, np.float64)), _p(gm), _p(gc))
    return gm, gc


def lift_backward(view, g_mean, g_cov, g_op, g_ft):
    """Adjoint of lift_view (FP64) for one source view: per-pixel gradients
    dict(depth (H,W), scale (H,W,3), quat (H,W,4) or None, opacity (H,W),
    feat (H,W,C)) from the per-Gaussian gradients."""
    H, W = view.depth.shape
    C = view.feat.shape[-1]
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
    out = dict(depth=np.empty((H, W)), scale=np.empty((H, W, 3)),
               quat=None if view.quat is None else np.empty((H, W, 4)), opacity=np.empty((H, W)),
               feat=np.empty((H, W, C)))
    mask = None if view.mask is None else np.ascontiguousarray(view.mask, np.uint8)
    lib().orc_lift_backward_f64(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_int(C), _p(f32(view.depth)), _p(mask),
                                _p(f32(view.scale)), _p(f32(view.quat)), _p(cam_array(view.cam)),
                                _p(np.ascontiguousarray(g_mean, np.float64)), _p(np.ascontiguousarray(g_cov, np.float64)),
                                _p(np.ascontiguousarray(g_op, np.float64)), _p(np.ascontiguousarray(g_ft, np.float64)),
                                _p(out["depth"]), _p(out["scale"]), _p(out["quat"]), _p(out["opacity"]), _p(out["feat"]))
    return out


def zbuffer(mean: np.ndarray, cam):
    """Point z-buffer of the (N,3) FP32 points: (depth (H,W) f32, 0 where
    empty; id (H,W) int32, -1 where empty)."""
    mean = np.ascontiguousarray(mean, np.float32)
    depth = np.empty((cam.height, cam.width), np.float32)
    ids = np.empty((cam.height, cam.width), np.int32)
    lib().orc_zbuffer(_i64(mean.shape[0]), _p(mean), _p(cam_array(cam)), _p(depth), _p(ids))
    return depth, ids


def project_f64(g: Gaussians, cam, par=None):
    """Returns (mu (N,2), conic (N,3), depth (N,), visible (N,) bool) in FP64."""
    par = params_array() if par is None else par
    n = g.n
    mean = np.ascontiguousarray(g.mean, np.float64)
    cov = np.ascontiguousarray(g.cov, np.float64)
    mu = np.empty((n, 2)); conic = np.empty((n, 3)); depth = np.empty(n); vis = np.empty(n, np.uint8)
    lib().orc_project_f64(_i64(n), _p(mean), _p(cov), _p(cam_array(cam)), _p(par),
                          _p(mu), _p(conic), _p(depth), _p(vis))
    return mu, conic, depth, vis.astype(bool)


# ---------------------------------------------------------------------------
# binning
# ---------------------------------------------------------------------------

@dataclass
class Bins:
    offsets: np.ndarray  # (N,) int64
    P: int
    keys: np.ndarray     # (P,) uint64 sorted
    ids: np.ndarray      # (P,) uint32 sorted
    ranges: np.ndarray   # (T,2) uint32
    tiles_x: int
    tiles_y: int


def tile_grid(width: int, height: int):
    return (width + TILE - 1) // TILE, (height + TILE - 1) // TILE


def _emit(proj: Projected, offsets, tx, keys, vals):
    n = proj.rect.shape[0]
    if proj.mask is None:
        lib().orc_emit(_i64(n), _p(proj.rect), _p(offsets), _p(proj.dkey), ctypes.c_int(tx), _p(keys), _p(vals))
    else:
        lib().orc_emit_masked(_i64(n), _p(proj.rect), _p(proj.mask), _p(offsets), _p(proj.dkey), ctypes.c_int(tx),
                              _p(keys), _p(vals))


def bin_gaussians(proj: Projected, width: int, height: int) -> Bins:
    n = proj.rect.shape[0]
    tx, ty = tile_grid(width, height)
    offsets = np.empty(n, np.int64)
    P = int(lib().orc_scan(_i64(n), _p(proj.ntiles), _p(offsets)))
    keys = np.empty(max(P, 1), np.uint64)
    vals = np.empty(max(P, 1), np.uint32)
    _emit(proj, offsets, tx, keys, vals)
    lib().orc_sort_pairs(_i64(P), _p(keys), _p(vals))
    keys, vals = keys[:P], vals[:P]
    ranges = np.empty((tx * ty, 2), np.uint32)
    lib().orc_ranges(_i64(P), _p(np.ascontiguousarray(keys)), ctypes.c_int(tx * ty), _p(ranges))
    return Bins(offsets, P, keys, vals, ranges, tx, ty)


def emit_unsorted(proj: Projected, width: int, height: int):
    """Pairs in emission order (before the sort): (keys, vals)."""
    n = proj.rect.shape[0]
    tx, _ = tile_grid(width, height)
    offsets = np.empty(n, np.int64)
    P = int(lib().orc_scan(_i64(n), _p(proj.ntiles), _p(offsets)))
    keys = np.empty(max(P, 1), np.uint64)
    vals = np.empty(max(P, 1), np.uint32)
    _emit(proj, offsets, tx, keys, vals)
    return keys[:P], vals[:P]


def tile_list_bruteforce(proj: Projected, tx: int, ty: int) -> np.ndarray:
    n = proj.rect.shape[0]
    out = np.empty(max(n, 1), np.uint32)
    m = lib().orc_tile_list_bruteforce(_i64(n), _p(proj.rect), _p(proj.dkey), ctypes.c_int(tx), ctypes.c_int(ty), _p(out))
    return out[:m].copy()


# ---------------------------------------------------------------------------
# compositing and its adjoint
# ---------------------------------------------------------------------------

@dataclass
class Composite:
    F: np.ndarray       # (C,H,W) f64
    A: np.ndarray       # (H,W)
    T: np.ndarray       # (H,W)
    last: np.ndarray    # (H,W) int32
    flags: np.ndarray   # (H,W) uint8 number of ambiguous decisions


def _margins(margins):
    if margins is None:
        margins = (MARGIN_ALPHA, MARGIN_T, MARGIN_Q)
    return np.asarray(margins, np.float64)


def composite(mu, conic, opac, feat, width, height, bins: Bins, par=None, margins=None,
              tiles: Optional[Sequence[int]] = None, dec_in=None, record=False):
    par = params_array() if par is None else par
    C = feat.shape[1]
    mu = np.ascontiguousarray(mu, np.float64)
    conic = np.ascontiguousarray(conic, np.float64)
    opac = np.ascontiguousarray(opac, np.float64)
    feat = np.ascontiguousarray(feat, np.float64)
    F = np.zeros((C, height, width))
    A = np.zeros((height, width))
    T = np.ones((height, width))
    last = np.zeros((height, width), np.int32)
    flags = np.zeros((height, width), np.uint8)
    tl = None if tiles is None else np.ascontiguousarray(np.asarray(tiles, np.int32))
    dec_out = np.full(max(256 * bins.P, 1), 3, np.uint8) if record else None
    din = None if dec_in is None else np.ascontiguousarray(dec_in, np.uint8)
    ids = np.ascontiguousarray(bins.ids if bins.P > 0 else np.zeros(1, np.uint32))
    lib().orc_composite(_i64(mu.shape[0]), _p(mu), _p(conic), _p(opac), _p(feat), ctypes.c_int(C),
                        ctypes.c_int(width), ctypes.c_int(height), _p(np.ascontiguousarray(bins.ranges)), _p(ids),
                        _p(par), _p(_margins(margins)), ctypes.c_int(0 if tl is None else len(tl)), _p(tl),
                        _p(F), _p(A), _p(T), _p(last), _p(flags), _p(din), _p(dec_out))
    res = Composite(F, A, T, last, flags)
    if record:
        return res, dec_out
    return res


def pixel_alternatives(mu, conic, opac, feat, width, height, bins: Bins, x: int, y: int,
                       par=None, margins=None, max_flip: int = 3):
    """Alternative (F, A) of a pixel with ambiguous decisions: array
    (n_alt, C+1), or None if it has more than max_flip ambiguous decisions."""
    par = params_array() if par is None else par
    C = feat.shape[1]
    out = np.empty(((1 << max_flip) - 1, C + 1))
    ids = np.ascontiguousarray(bins.ids if bins.P > 0 else np.zeros(1, np.uint32))
    n = lib().orc_pixel_alternatives(_p(np.ascontiguousarray(mu, np.float64)), _p(np.ascontiguousarray(conic, np.float64)),
                                     _p(np.ascontiguousarray(opac, np.float64)), _p(np.ascontiguousarray(feat, np.float64)),
                                     ctypes.c_int(C), ctypes.c_int(width), ctypes.c_int(height),
                                     _p(np.ascontiguousarray(bins.ranges)), _p(ids), _p(par), _p(_margins(margins)),
                                     ctypes.c_int(x), ctypes.c_int(y), ctypes.c_int(max_flip), _p(out))
    if n < 0:
        return None
    return out[:n].copy()


def backward(mu, conic, opac, feat, width, height, bins: Bins, dF, dA=None, par=None):
    """FP64 adjoint: returns (d_mu (N,2), d_conic (N,3), d_opac (N,), d_feat (N,C))."""
    par = params_array() if par is None else par
    n, C = feat.shape
    d_mu = np.zeros((n, 2)); d_conic = np.zeros((n, 3)); d_opac = np.zeros(n); d_feat = np.zeros((n, C))
    ids = np.ascontiguousarray(bins.ids if bins.P > 0 else np.zeros(1, np.uint32))
    dAa = None if dA is None else np.ascontiguousarray(dA, np.float64)
    lib().orc_backward(_i64(n), _p(np.ascontiguousarray(mu, np.float64)), _p(np.ascontiguousarray(conic, np.float64)),
                       _p(np.ascontiguousarray(opac, np.float64)), _p(np.ascontiguousarray(feat, np.float64)),
                       ctypes.c_int(C), ctypes.c_int(width), ctypes.c_int(height),
                       _p(np.ascontiguousarray(bins.ranges)), _p(ids), _p(par),
                       _p(np.ascontiguousarray(dF, np.float64)), _p(dAa),
                       _p(d_mu), _p(d_conic), _p(d_opac), _p(d_feat))
    return d_mu, d_conic, d_opac, d_feat


# ---------------------------------------------------------------------------
# whole path
# ---------------------------------------------------------------------------

@dataclass
class Render:
    proj: Projected
    bins: Bins
    mu64: np.ndarray
    conic64: np.ndarray
    comp: Composite


def render(g32: Gaussians, cam, par=None, margins=None, tiles=None, feat64=None,
           values: str = "key", tight: bool = False) -> Render:
    """Key-mode binning of FP32 Gaussians, then FP64 compositing.

    values="key": the compositing consumes the projected record (mu, conic)
    exactly as the key mode rounds it to FP32, widened to FP64 -- the input
    the compositing stage of a single-precision implementation receives.
    values="f64": mu and conic are re-derived in FP64 from the same
    Gaussians (end-to-end comparison, includes FP32 rounding of mu).
    `feat64` overrides the features that are composited (e.g. the original
    FP32 features when the stored ones were rounded to BF16).  `tight`
    bins with the tight-binning variant (see `tighten`)."""
    par = params_array() if par is None else par
    proj = project_f32(g32, cam, par)
    if tight:
        proj = tighten(proj, g32.opac, cam.width, cam.height, par)
    bins = bin_gaussians(proj, cam.width, cam.height)
    if values == "key":
        mu64, conic64 = proj.mu.astype(np.float64), proj.conic.astype(np.float64)
    else:
        mu64, conic64, _, _ = project_f64(g32.astype(np.float64), cam, par)
    feat = g32.feat if feat64 is None else feat64
    comp = composite(mu64, conic64, g32.opac.astype(np.float64), feat.astype(np.float64),
                     cam.width, cam.height, bins, par, margins, tiles)
    return Render(proj, bins, mu64, conic64, comp)
