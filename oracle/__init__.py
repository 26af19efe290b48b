"""FP64 CPU oracle of the Instant4D rasterizer and grid pruning -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product (``paper_2510_01119_gb300``) never does, and this package imports
nothing from the product: the two share no code.  The arithmetic lives in ``i4d_oracle.c``
(plain C, float64) and ``adam.py`` (numpy float64); this file only marshals numpy arrays.

Paper: Instant4D (arXiv 2510.01119).  Eq. 5 back-projection, Sec. 3.2 grid pruning, Eq. 7-8
conditional mean/covariance, Eq. 9 and the temporal-opacity cull of Sec. 3.3, the isotropic
variant of Sec. 3.3, and the 3D splatting renderer of Sec. 3.1 (Eq. 3) that the method builds on.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .adam import adam_step  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "i4d_oracle.c")
_LIB = os.path.join(_HERE, "libi4d_oracle.so")
_lock = threading.Lock()
_lib = None

MODE_FULL, MODE_ISO_ROT, MODE_ISO_IDENTITY = 0, 1, 2

# projected-record columns (must follow the enum in i4d_oracle.c)
PCOLS = ["visible", "u", "v", "depth", "ot", "ca", "cb", "cc", "radius", "r", "g", "b",
         "margin", "radius_margin",
         "m3x", "m3y", "m3z", "s3xx", "s3xy", "s3xz", "s3yy", "s3yz", "s3zz"]
P = {name: k for k, name in enumerate(PCOLS)}
# 2D-gradient columns
GCOLS = ["u", "v", "ca", "cb", "cc", "ot", "r", "g", "b"]

# Thresholds the paper leaves to the 3D splatting renderer it builds on (readings C3, C4).
DEFAULT_SETTINGS = dict(alpha_max=0.99, alpha_min=1.0 / 255.0, T_min=1e-4, q_max=9.0,
                        ot_min=1.0 / 255.0, z_near=0.2, dilation=0.3, fov_clamp=1.3)
_SETTING_ORDER = ["alpha_max", "alpha_min", "T_min", "q_max", "ot_min", "z_near", "dilation", "fov_clamp"]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no CUDA); returns the shared-library path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_tile_lists.restype = ctypes.c_long
        lib.orc_prune.restype = ctypes.c_long
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def settings_array(**overrides) -> np.ndarray:
    s = dict(DEFAULT_SETTINGS)
    for k, v in overrides.items():
        if k not in s:
            raise KeyError(k)
        s[k] = v
    return np.array([s[k] for k in _SETTING_ORDER], dtype=np.float64)


def camera_array(cam: dict) -> np.ndarray:
    """cam: dict(R (3,3) world->camera, t (3,), fx, fy, cx, cy, W, H, time)."""
    a = np.zeros(20, dtype=np.float64)
    a[0:9] = np.asarray(cam["R"], dtype=np.float64).reshape(9)
    a[9:12] = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    a[12], a[13], a[14], a[15] = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    a[16], a[17], a[18] = cam["W"], cam["H"], cam["time"]
    return a


def _gauss_arrays(g: dict):
    n = g["mean4"].shape[0]
    sh = g.get("sh")
    sh_arr = np.zeros((n, 15, 3), dtype=np.float64)
    if sh is not None and sh.size:
        k = sh.shape[1]
        sh_arr[:, :k, :] = sh
    return (n, int(g.get("sh_deg", 0)), int(g.get("mode", MODE_FULL)), _f64(g["mean4"]), _f64(g["logscale4"]),
            _f64(g["ql"]), _f64(g["qr"]), _f64(g["opacity"]), _f64(g["rgb"]), np.ascontiguousarray(sh_arr))


def _sch_arrays(g: dict):
    """SCH variant (sch_terms N_t > 1): (N_t, coefficients (n, N_t - 1, (deg + 1)^2, 3) as float64 or None)."""
    nt = int(g.get("sch_terms", 0))
    if nt <= 1:
        return 0, None
    return nt, _f64(np.asarray(g["sch"]).reshape(g["mean4"].shape[0], nt - 1, (int(g.get("sh_deg", 0)) + 1) ** 2, 3))


def project(g: dict, cam: dict, settings=None) -> np.ndarray:
    """Eq. 7-8 slicing, temporal opacity, EWA projection and colour for every Gaussian -> (n, 23).
    visible = not culled (temporal opacity, near plane, degenerate 2D covariance); margin = the
    smallest relative distance of those decisions from their thresholds; radius_margin = that of
    the 3-sigma radius ceil(3 sqrt(lambda_max)) from an integer."""
    lib = _load()
    n, deg, mode, m4, ls4, ql, qr, op, rgb, sh = _gauss_arrays(g)
    S = settings if settings is not None else settings_array()
    out = np.zeros((n, len(PCOLS)), dtype=np.float64)
    nt, sch = _sch_arrays(g)
    rc = lib.orc_project(n, deg, mode, _ptr(m4), _ptr(ls4), _ptr(ql), _ptr(qr), _ptr(op), _ptr(rgb), _ptr(sh),
                         nt, _ptr(sch), _ptr(camera_array(cam)), _ptr(S), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_project failed ({rc})")
    return out


def render(proj: np.ndarray, cam: dict, bg=(0.0, 0.0, 0.0), settings=None, pix=None, depth_margin=False,
           impact_min: float = 0.0):
    """Per-pixel depth-sorted compositing -> (img (npix,3), T_final, n_contrib, margin), plus the
    depth-order margin when depth_margin.  margin / depth margin: smallest relative distance from a
    threshold / smallest relative depth gap of two consecutive blended fragments, over the decisions
    whose flip could move the pixel's colour by more than impact_min."""
    lib = _load()
    n = proj.shape[0]
    W, H = int(cam["W"]), int(cam["H"])
    S = settings if settings is not None else settings_array()
    pix_arr = None if pix is None else np.ascontiguousarray(pix, dtype=np.int32)
    npix = W * H if pix is None else pix_arr.shape[0]
    img = np.zeros((npix, 3), dtype=np.float64)
    T = np.zeros(npix, dtype=np.float64)
    nc = np.zeros(npix, dtype=np.int32)
    mg = np.zeros(npix, dtype=np.float64)
    dmg = np.zeros(npix, dtype=np.float64)
    rc = lib.orc_render(n, _ptr(np.ascontiguousarray(proj)), _ptr(camera_array(cam)), _ptr(_f64(bg)), _ptr(S),
                        npix, _ptr(pix_arr), ctypes.c_double(impact_min), _ptr(img), _ptr(T), _ptr(nc), _ptr(mg),
                        _ptr(dmg))
    if rc != 0:
        raise RuntimeError(f"orc_render failed ({rc})")
    return (img, T, nc, mg, dmg) if depth_margin else (img, T, nc, mg)


def render_alternatives(proj: np.ndarray, cam: dict, pix, margin: float, depth_margin: float, impact_min: float,
                        max_alt: int = 1024, bg=(0.0, 0.0, 0.0), settings=None):
    """Every valid colour of each pixel in `pix` when its decisions within `margin` of a threshold
    (coverage, alpha, cull, near plane, the T stop) may go either way and fragments whose depths
    differ by less than depth_margin (relative) may come in either order, counting only decisions
    whose flip moves the colour by more than impact_min: (alt (npix, max_alt, 3), n_alt (npix,)),
    n_alt = the number of branches (alt[:, 0] is the computed one), -1 when there are too many."""
    lib = _load()
    S = settings if settings is not None else settings_array()
    pix_arr = np.ascontiguousarray(pix, dtype=np.int32)
    npix = pix_arr.shape[0]
    alt = np.zeros((npix, max_alt, 3), dtype=np.float64)
    n_alt = np.zeros(npix, dtype=np.int32)
    rc = lib.orc_render_alternatives(proj.shape[0], _ptr(np.ascontiguousarray(proj)), _ptr(camera_array(cam)),
                                     _ptr(_f64(bg)), _ptr(S), npix, _ptr(pix_arr), ctypes.c_double(margin),
                                     ctypes.c_double(depth_margin), ctypes.c_double(impact_min), int(max_alt),
                                     _ptr(alt), _ptr(n_alt))
    if rc != 0:
        raise RuntimeError(f"orc_render_alternatives failed ({rc})")
    return alt, n_alt


def render_bwd(g: dict, cam: dict, dL_dimg: np.ndarray, bg=(0.0, 0.0, 0.0), settings=None, pix=None):
    """Analytic backward for one camera -> (grad2d (n,9), dict of parameter gradients)."""
    lib = _load()
    n, deg, mode, m4, ls4, ql, qr, op, rgb, sh = _gauss_arrays(g)
    W, H = int(cam["W"]), int(cam["H"])
    S = settings if settings is not None else settings_array()
    pix_arr = None if pix is None else np.ascontiguousarray(pix, dtype=np.int32)
    npix = W * H if pix is None else pix_arr.shape[0]
    gimg = _f64(dL_dimg).reshape(npix, 3)
    g2 = np.zeros((n, 9), dtype=np.float64)
    grads = dict(mean4=np.zeros((n, 4)), logscale4=np.zeros((n, 4)), ql=np.zeros((n, 4)), qr=np.zeros((n, 4)),
                 opacity=np.zeros(n), rgb=np.zeros((n, 3)), sh=np.zeros((n, 15, 3)))
    nt, sch = _sch_arrays(g)
    if nt > 1:
        grads["sch"] = np.zeros_like(sch)
    rc = lib.orc_render_bwd(n, deg, mode, _ptr(m4), _ptr(ls4), _ptr(ql), _ptr(qr), _ptr(op), _ptr(rgb), _ptr(sh),
                            nt, _ptr(sch), _ptr(camera_array(cam)), _ptr(_f64(bg)), _ptr(S), npix, _ptr(pix_arr), _ptr(gimg),
                            _ptr(g2), _ptr(grads["mean4"]), _ptr(grads["logscale4"]), _ptr(grads["ql"]),
                            _ptr(grads["qr"]), _ptr(grads["opacity"]), _ptr(grads["rgb"]), _ptr(grads["sh"]),
                            _ptr(grads.get("sch")))
    if rc != 0:
        raise RuntimeError(f"orc_render_bwd failed ({rc})")
    grads["sh"] = grads["sh"][:, : (deg + 1) ** 2 - 1, :]
    return g2, grads


def tile_lists(proj: np.ndarray, cam: dict, tile=(16, 16), tile_offset: int = 0, settings=None,
               margin: float = 1e-4):
    """Binning (Sec. 3.1): every (tile, Gaussian) pair whose tile holds a pixel centre where the
    Gaussian can be blended (q <= q_max and o_t exp(-q/2) >= alpha_min), ordered by (tile, depth, id).
    Returns (tiles, ids, status): status 1 = needed, 2 = only pixel centres within `margin` (relative)
    of a threshold, so a float32 evaluation may take or drop the pair."""
    lib = _load()
    S = settings if settings is not None else settings_array()
    P = np.ascontiguousarray(proj)
    cap = 1 << 16
    while True:
        tiles = np.zeros(cap, dtype=np.int32)
        ids = np.zeros(cap, dtype=np.int32)
        st = np.zeros(cap, dtype=np.int32)
        cnt = lib.orc_tile_lists(P.shape[0], _ptr(P), _ptr(camera_array(cam)), int(tile[0]), int(tile[1]),
                                 int(tile_offset), _ptr(S), ctypes.c_double(margin), ctypes.c_long(cap), _ptr(tiles),
                                 _ptr(ids), _ptr(st))
        if cnt == -1 and cap < (1 << 34):
            cap *= 4
            continue
        if cnt < 0:
            raise RuntimeError(f"orc_tile_lists failed ({cnt})")
        return tiles[:cnt], ids[:cnt], st[:cnt]


def backproject(cam: dict, depth: np.ndarray) -> np.ndarray:
    """Eq. 5 for every pixel of one depth map -> (H*W, 3) float64 world points."""
    lib = _load()
    H, W = depth.shape
    assert W == int(cam["W"]) and H == int(cam["H"])
    out = np.zeros((H * W, 3), dtype=np.float64)
    lib.orc_backproject(_ptr(camera_array(cam)), _ptr(np.ascontiguousarray(depth, dtype=np.float32)), _ptr(out))
    return out


def backproject_f32(cam: dict, depth: np.ndarray) -> np.ndarray:
    """Eq. 5 as a fixed sequence of correctly rounded float32 operations (camera rounded to float32
    first) -> (H*W, 3) float32: the reading under which pruning the back-projected cloud is
    bit-reproducible.  Pinned against the float64 form within its rounding-error bound."""
    lib = _load()
    H, W = depth.shape
    assert W == int(cam["W"]) and H == int(cam["H"])
    out = np.zeros((H * W, 3), dtype=np.float32)
    lib.orc_backproject_f32(_ptr(camera_array(cam)), _ptr(np.ascontiguousarray(depth, dtype=np.float32)), _ptr(out))
    return out


def backproject_video_f32(vid: dict) -> np.ndarray:
    """backproject_f32 of every frame of a depth video, frames concatenated (point index
    f*H*W + py*W + px) -> (F*H*W, 3) float32."""
    F, H, W = vid["depth"].shape
    out = np.empty((F * H * W, 3), dtype=np.float32)
    for f, c in enumerate(vid["cams"]):
        out[f * H * W:(f + 1) * H * W] = backproject_f32(c, vid["depth"][f])
    return out


def prune(xyz: np.ndarray, voxel_static: float, voxel_dynamic: float = None, min_support: int = 1,
          rgb: np.ndarray = None, t: np.ndarray = None, dyn: np.ndarray = None):
    """Grid pruning of a float32 point cloud (Sec. 3.2).  The voxel index of a coordinate is the
    floor of one float32 product with the float32 reciprocal of the voxel size."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    npts = xyz.shape[0]
    inv_s = np.float32(1.0) / np.float32(voxel_static)
    vd = voxel_dynamic if voxel_dynamic is not None else voxel_static
    inv_d = np.float32(0.0) if vd == 0 else np.float32(1.0) / np.float32(vd)  # 0: dynamic points unpruned
    cap = max(npts, 1)
    rep = np.zeros(cap, dtype=np.uint32)
    cnt = np.zeros(cap, dtype=np.int32)
    cen = np.zeros((cap, 3), dtype=np.float64)
    mrgb = np.zeros((cap, 3), dtype=np.float64)
    mt = np.zeros(cap, dtype=np.float64)
    flag = np.zeros(cap, dtype=np.uint8)
    rgb_a = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.float32)
    t_a = None if t is None else np.ascontiguousarray(t, dtype=np.float32)
    dyn_a = None if dyn is None else np.ascontiguousarray(dyn, dtype=np.uint8)
    k = lib.orc_prune(ctypes.c_long(npts), _ptr(xyz), _ptr(rgb_a), _ptr(t_a), _ptr(dyn_a), ctypes.c_float(inv_s),
                      ctypes.c_float(inv_d), int(min_support), ctypes.c_long(cap), _ptr(rep), _ptr(cnt), _ptr(cen),
                      _ptr(mrgb), _ptr(mt), _ptr(flag))
    if k < 0:
        raise RuntimeError(f"orc_prune failed ({k})")
    return dict(rep=rep[:k], count=cnt[:k], centroid=cen[:k], rgb=mrgb[:k], t=mt[:k], flag=flag[:k])


def sh_basis(d: np.ndarray) -> np.ndarray:
    """The 15 real SH basis values of degree 1..3 at unit direction d."""
    lib = _load()
    out = np.zeros(15, dtype=np.float64)
    lib.orc_sh_basis(_ptr(_f64(d)), _ptr(out))
    return out


def cov4(logscale4, ql, qr, mode: int = MODE_FULL) -> np.ndarray:
    """The 4D covariance R diag(s^2) R^T of one Gaussian -> (4, 4)."""
    lib = _load()
    out = np.zeros(16, dtype=np.float64)
    lib.orc_cov4(int(mode), _ptr(_f64(logscale4)), _ptr(_f64(ql)), _ptr(_f64(qr)), _ptr(out))
    return out.reshape(4, 4)


def init_heuristic(pruned: dict, spatial_scale, st_dynamic: float, st_static: float = 1.0,
                   opacity: float = 0.1) -> dict:
    """4D Gaussians from pruned voxels (Sec. 4.1; Sec. 3.3 "Motion-Aware Gaussian"): mean = (centroid,
    mean time); s_t = st_dynamic for dynamic voxels, st_static for static ones; isotropic spatial
    scale; R = I; opacity logit of `opacity`; colour = mean colour."""
    n = len(pruned["rep"])
    mean4 = np.c_[pruned["centroid"], pruned["t"]]
    ls = np.zeros((n, 4))
    ls[:, :3] = np.log(np.asarray(spatial_scale, np.float64)).reshape(-1, 1)
    ls[:, 3] = np.where(pruned["flag"] != 0, np.log(st_dynamic), np.log(st_static))
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return dict(mean4=mean4, logscale4=ls, ql=q, qr=q.copy(), opacity=np.full(n, np.log(opacity / (1 - opacity))),
                rgb=pruned["rgb"], sh=np.zeros((n, 0, 3)), sh_deg=0, mode=MODE_FULL)
