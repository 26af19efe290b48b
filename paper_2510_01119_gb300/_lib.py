"""ctypes binding of libi4d.so: argument marshalling only (torch tensors -> device pointers).

Every computation runs in the CUDA library; there is no CPU fallback.  Loading fails loudly when
the library has not been built (``paper_2510_01119_gb300.build.build()``) or no GPU is present
at call time.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libi4d.so")

MAX_VIEWS = 64
GRAD2D_FLOATS = 9  # I4D_GRAD2D_FLOATS: floats per (view, Gaussian) record of the 2D-gradient scratch
MODE_FULL, MODE_ISO_ROT, MODE_ISO_IDENTITY = 0, 1, 2
LOSS_L1, LOSS_MSE = 0, 1
STATUS = {0: "ok", -1: "invalid argument", -2: "capacity exceeded", -3: "CUDA error", -4: "workspace too small"}

c_f = ctypes.c_float
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t


class Camera(ctypes.Structure):
    _fields_ = [("R", c_f * 9), ("t", c_f * 3), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("time", c_f), ("pad", c_f * 3)]


class Views(ctypes.Structure):
    _fields_ = [("n_views", c_i32), ("tile_w", c_i32), ("tile_h", c_i32), ("width", c_i32 * MAX_VIEWS),
                ("height", c_i32 * MAX_VIEWS)]


class Gaussians(ctypes.Structure):
    _fields_ = [("params", c_vp), ("n", c_i32), ("sh_deg", c_i32), ("mode", c_i32), ("sch_terms", c_i32)]


class Settings(ctypes.Structure):
    _fields_ = [("alpha_max", c_f), ("alpha_min", c_f), ("T_min", c_f), ("q_max", c_f), ("ot_min", c_f),
                ("z_near", c_f), ("dilation", c_f), ("fov_clamp", c_f), ("bg", c_f * 3), ("pad", c_f)]


class Tune(ctypes.Structure):
    _fields_ = [("batch", c_i32), ("reserved", c_i32 * 7)]


class AdamGroup(ctypes.Structure):
    _fields_ = [("begin", c_i64), ("end", c_i64), ("lr_init", c_f * 4), ("lr_final", c_f * 4),
                ("decay_steps", c_i32), ("pad", c_i32)]


class I4DError(RuntimeError):
    pass


_lib = None

_SIGS = {
    "i4d_version": (c_i32, []),
    "i4d_status_string": (ctypes.c_char_p, [c_i32]),
    "i4d_default_settings": (None, [ctypes.POINTER(Settings)]),
    "i4d_param_floats": (c_i64, [c_i32]),
    "i4d_param_floats_sch": (c_i64, [c_i32, c_i32]),
    "i4d_total_tiles": (c_i64, [ctypes.POINTER(Views)]),
    "i4d_total_pixels": (c_i64, [ctypes.POINTER(Views)]),
    "i4d_slice_project": (c_i32, [ctypes.POINTER(Gaussians), ctypes.POINTER(Views), c_vp, ctypes.POINTER(Settings),
                                  c_vp, c_vp, c_vp]),
    "i4d_bin_tiles_workspace_size": (c_sz, [ctypes.POINTER(Views), c_i32, c_i64]),
    "i4d_bin_tiles": (c_i32, [ctypes.POINTER(Views), c_i32, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz,
                              c_vp]),
    "i4d_render_fwd": (c_i32, [ctypes.POINTER(Views), c_i32, c_vp, c_vp, c_vp, ctypes.POINTER(Settings),
                               ctypes.POINTER(Tune), c_vp, c_vp, c_vp, c_vp, c_vp]),
    "i4d_render_bwd": (c_i32, [ctypes.POINTER(Gaussians), ctypes.POINTER(Views), c_vp, ctypes.POINTER(Settings),
                               c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "i4d_loss": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp]),
    "i4d_psnr": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "i4d_photometric_loss_workspace_size": (c_sz, [ctypes.POINTER(Views)]),
    "i4d_adaptive_voxel_workspace_size": (c_sz, [c_i32]),
    "i4d_adaptive_voxel": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, ctypes.c_float, c_vp, c_vp, c_sz, c_vp]),
    "i4d_motion_masks_workspace_size": (c_sz, [c_i32]),
    "i4d_motion_masks": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "i4d_photometric_loss": (c_i32, [ctypes.POINTER(Views), c_vp, c_vp, ctypes.c_float, c_vp, c_vp, c_vp, c_vp, c_sz,
                                     c_vp]),
    "i4d_adam_step": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(AdamGroup), c_i32, c_vp, c_f, c_f, c_f,
                              c_vp]),
    "i4d_prune_workspace_size": (c_sz, [c_i64, c_i64]),
    "i4d_prune_points": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_f, c_f, c_i32, c_i64, c_i64, c_vp,
                                 c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "i4d_prune_points_xyz": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_f, c_f, c_i32, c_i64, c_i64, c_vp, c_vp, c_vp,
                                     c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "i4d_init_heuristic": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_f, c_f, c_f, c_f, c_vp, c_vp]),
    "i4d_render_bwd_noalloc_max_records": (c_i64, []),
    "i4d_render_bwd_noalloc": (c_i32, [ctypes.POINTER(Gaussians), ctypes.POINTER(Views), c_vp,
                                       ctypes.POINTER(Settings), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                       c_vp]),
    "i4d_knn_workspace_size": (c_sz, [c_i64, c_i64]),
    "i4d_knn_features": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_f, c_i32, ctypes.POINTER(c_f), c_vp, c_vp, c_i64,
                                 c_vp, c_vp, c_sz, c_vp]),
    "i4d_motion_targets": (c_i32, [ctypes.POINTER(Gaussians), c_vp, c_vp]),
    "i4d_mlp_weight_count": (c_i64, []),
    "i4d_mlp_forward": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "i4d_mlp_grad_workspace_size": (c_sz, [c_i64]),
    "i4d_mlp_grad": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_f, c_f, c_f, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "i4d_init_learned": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_f, c_f, c_f, c_vp, c_vp, c_vp]),
    "i4d_profile_enable": (c_i32, [c_i32]),
    "i4d_profile_reset": (None, []),
    "i4d_profile_count": (c_i32, []),
    "i4d_profile_read": (c_i32, [c_i32, ctypes.c_char_p, c_i32, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(c_i64)]),
    "i4d_measure_fp32_peak": (c_i32, [c_i32, c_i32, ctypes.POINTER(ctypes.c_double), c_vp]),
}


def exported_names():
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load libi4d.so (no build here); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise I4DError(f"libi4d.so not built at {path}: run paper_2510_01119_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int, what: str) -> None:
    if rc != 0:
        raise I4DError(f"{what} failed: {STATUS.get(rc, rc)}")


def ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise I4DError("libi4d takes CUDA tensors only")
    if not t.is_contiguous():
        raise I4DError("libi4d takes contiguous tensors only")
    return ctypes.c_void_p(t.data_ptr())


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_settings(**overrides) -> Settings:
    s = Settings()
    load().i4d_default_settings(ctypes.byref(s))
    for k, v in overrides.items():
        if k == "bg":
            for i in range(3):
                s.bg[i] = float(v[i])
        else:
            setattr(s, k, float(v))
    return s


def make_views(sizes, tile=(16, 16)) -> Views:
    """sizes: list of (W, H)."""
    if not 1 <= len(sizes) <= MAX_VIEWS:
        raise I4DError("1..64 views per launch")
    v = Views()
    v.n_views = len(sizes)
    v.tile_w, v.tile_h = int(tile[0]), int(tile[1])
    for k, (W, H) in enumerate(sizes):
        v.width[k], v.height[k] = int(W), int(H)
    return v


# ---- same-named wrappers of the C ABI (tensors in, status checked) ------------------------------------
def i4d_slice_project(g: Gaussians, views: Views, cams, settings, proj, touched, stream=None):
    check(load().i4d_slice_project(ctypes.byref(g), ctypes.byref(views), ptr(cams), ctypes.byref(settings), ptr(proj),
                                   ptr(touched), stream_ptr(stream)), "i4d_slice_project")


def i4d_bin_tiles_workspace_size(views: Views, n: int, capacity: int) -> int:
    return int(load().i4d_bin_tiles_workspace_size(ctypes.byref(views), int(n), int(capacity)))


def i4d_bin_tiles(views: Views, n: int, proj, touched, capacity: int, ids, ranges, n_inst, status, ws, stream=None):
    check(load().i4d_bin_tiles(ctypes.byref(views), int(n), ptr(proj), ptr(touched), int(capacity), ptr(ids),
                               ptr(ranges), ptr(n_inst), ptr(status), ptr(ws), ws.numel() * ws.element_size(),
                               stream_ptr(stream)), "i4d_bin_tiles")


def i4d_render_fwd(views: Views, n: int, proj, ids, ranges, settings, tune, img, T_final, last, n_contrib,
                   stream=None):
    check(load().i4d_render_fwd(ctypes.byref(views), int(n), ptr(proj), ptr(ids), ptr(ranges), ctypes.byref(settings),
                                ctypes.byref(tune) if tune is not None else None, ptr(img), ptr(T_final), ptr(last),
                                ptr(n_contrib), stream_ptr(stream)), "i4d_render_fwd")


def i4d_render_bwd(g: Gaussians, views: Views, cams, settings, proj, touched, ids, ranges, T_final, last, dL_dimg,
                   grad2d, grads, stream=None):
    check(load().i4d_render_bwd(ctypes.byref(g), ctypes.byref(views), ptr(cams), ctypes.byref(settings), ptr(proj),
                                ptr(touched), ptr(ids), ptr(ranges), ptr(T_final), ptr(last), ptr(dL_dimg),
                                ptr(grad2d), ptr(grads), stream_ptr(stream)), "i4d_render_bwd")


def i4d_loss(img, target, kind: int, dL_dimg, loss_out, stream=None):
    check(load().i4d_loss(ptr(img), ptr(target), img.numel(), int(kind), ptr(dL_dimg), ptr(loss_out),
                          stream_ptr(stream)), "i4d_loss")


def i4d_adaptive_voxel_workspace_size(F: int) -> int:
    return int(load().i4d_adaptive_voxel_workspace_size(int(F)))


def i4d_adaptive_voxel(depth, cams, lambda_s: float, voxel_out, ws, stream=None):
    """depth: (F, H, W) float32 CUDA tensor; cams: (F, 20) camera tensor; voxel_out: 1 float."""
    F, H, W = depth.shape
    check(load().i4d_adaptive_voxel(ptr(depth), int(F), int(W), int(H), ptr(cams), float(lambda_s), ptr(voxel_out),
                                    ptr(ws), ws.numel() * ws.element_size(), stream_ptr(stream)), "i4d_adaptive_voxel")


def i4d_motion_masks_workspace_size(F: int) -> int:
    return int(load().i4d_motion_masks_workspace_size(int(F)))


def i4d_motion_masks(prob, W: int, H: int, mask, thresholds, ws, stream=None):
    """prob: (F, h, w) float32 CUDA tensor; mask: (F, H, W) uint8; thresholds: (F,) int32 or None."""
    F, h, w = prob.shape
    check(load().i4d_motion_masks(ptr(prob), int(F), int(w), int(h), int(W), int(H), ptr(mask), ptr(thresholds),
                                  ptr(ws), ws.numel() * ws.element_size(), stream_ptr(stream)), "i4d_motion_masks")


def i4d_photometric_loss_workspace_size(views: Views) -> int:
    return int(load().i4d_photometric_loss_workspace_size(ctypes.byref(views)))


def i4d_photometric_loss(views: Views, img, target, lambda_dssim: float, dL_dimg, loss_out, ssim_out, ws,
                         stream=None):
    check(load().i4d_photometric_loss(ctypes.byref(views), ptr(img), ptr(target), float(lambda_dssim), ptr(dL_dimg),
                                      ptr(loss_out), ptr(ssim_out), ptr(ws), ws.numel() * ws.element_size(),
                                      stream_ptr(stream)), "i4d_photometric_loss")


def i4d_psnr(img, target, psnr_out, stream=None):
    check(load().i4d_psnr(ptr(img), ptr(target), img.numel(), ptr(psnr_out), stream_ptr(stream)), "i4d_psnr")


def i4d_adam_step(params, grads, m, v, groups, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    arr = (AdamGroup * max(len(groups), 1))(*groups)
    check(load().i4d_adam_step(ptr(params), ptr(grads), ptr(m), ptr(v), params.numel(), arr, len(groups), ptr(step),
                               float(beta1), float(beta2), float(eps), stream_ptr(stream)), "i4d_adam_step")


def i4d_prune_workspace_size(n_points: int, table_slots: int) -> int:
    return int(load().i4d_prune_workspace_size(int(n_points), int(table_slots)))


def i4d_prune_points(depth, rgb, dyn, cams, F, W, H, voxel_static, voxel_dynamic, min_support, table_slots, capacity,
                     rep, count, xyz, rgb_out, t_out, flag, n_kept, status, ws, stream=None):
    check(load().i4d_prune_points(ptr(depth), ptr(rgb), ptr(dyn), ptr(cams), int(F), int(W), int(H),
                                  float(voxel_static), float(voxel_dynamic), int(min_support), int(table_slots),
                                  int(capacity), ptr(rep), ptr(count), ptr(xyz), ptr(rgb_out), ptr(t_out), ptr(flag),
                                  ptr(n_kept), ptr(status), ptr(ws), ws.numel() * ws.element_size(),
                                  stream_ptr(stream)), "i4d_prune_points")


def i4d_prune_points_xyz(xyz, rgb, t, dyn, voxel_static, voxel_dynamic, min_support, table_slots, capacity, rep,
                         count, xyz_out, rgb_out, t_out, flag, n_kept, status, ws, stream=None):
    check(load().i4d_prune_points_xyz(ptr(xyz), ptr(rgb), ptr(t), ptr(dyn), xyz.shape[0], float(voxel_static),
                                      float(voxel_dynamic), int(min_support), int(table_slots), int(capacity),
                                      ptr(rep), ptr(count), ptr(xyz_out), ptr(rgb_out), ptr(t_out), ptr(flag),
                                      ptr(n_kept), ptr(status), ptr(ws), ws.numel() * ws.element_size(),
                                      stream_ptr(stream)), "i4d_prune_points_xyz")


def i4d_init_heuristic(xyz, rgb, t, flag, n, sh_deg, spatial_scale, st_dynamic, st_static, opacity, params,
                       stream=None):
    check(load().i4d_init_heuristic(ptr(xyz), ptr(rgb), ptr(t), ptr(flag), int(n), int(sh_deg), float(spatial_scale),
                                    float(st_dynamic), float(st_static), float(opacity), ptr(params),
                                    stream_ptr(stream)), "i4d_init_heuristic")


def profile_enable(on: bool = True) -> None:
    load().i4d_profile_enable(1 if on else 0)


def profile_reset() -> None:
    load().i4d_profile_reset()


def i4d_measure_fp32_peak(blocks_per_sm: int = 8, iters: int = 20000, stream=None) -> float:
    """Measured FP32 FMA throughput of this GPU in TFLOP/s (packed-FMA chains; syncs the stream)."""
    out = ctypes.c_double()
    check(load().i4d_measure_fp32_peak(int(blocks_per_sm), int(iters), ctypes.byref(out), stream_ptr(stream)),
          "i4d_measure_fp32_peak")
    return float(out.value)


def profile_read() -> dict:
    """{kernel name: (total ms, launches)} of the launches recorded since the last reset (syncs)."""
    lib = load()
    out = {}
    for k in range(lib.i4d_profile_count()):
        name = ctypes.create_string_buffer(64)
        ms = ctypes.c_double()
        cnt = c_i64()
        check(lib.i4d_profile_read(k, name, 64, ctypes.byref(ms), ctypes.byref(cnt)), "i4d_profile_read")
        if cnt.value:
            out[name.value.decode()] = (ms.value, int(cnt.value))
    return out


def i4d_render_bwd_noalloc(g: Gaussians, views: Views, cams, settings, proj, touched, ids, ranges, T_final, last,
                           dL_dimg, grads, stream=None):
    """i4d_render_bwd without a scratch argument (the library's fixed scratch array is used)."""
    lib = load()
    rc = lib.i4d_render_bwd_noalloc(ctypes.byref(g), ctypes.byref(views), ptr(cams), ctypes.byref(settings),
                                    ptr(proj), ptr(touched), ptr(ids), ptr(ranges), ptr(T_final), ptr(last),
                                    ptr(dL_dimg), ptr(grads), stream_ptr(stream))
    if rc == -2:
        raise I4DError(f"i4d_render_bwd_noalloc: n_views * n = {views.n_views * g.n} exceeds the fixed scratch of "
                       f"{int(lib.i4d_render_bwd_noalloc_max_records())} records")
    check(rc, "i4d_render_bwd_noalloc")


def i4d_knn_workspace_size(n: int, table_slots: int) -> int:
    return int(load().i4d_knn_workspace_size(int(n), int(table_slots)))


def i4d_knn_features(xyz, rgb, t, flag, voxel, radius, ref_center, features, knn3, table_slots, status, ws,
                     stream=None):
    ref = (c_f * 3)(*[float(x) for x in ref_center])
    check(load().i4d_knn_features(ptr(xyz), ptr(rgb), ptr(t), ptr(flag), xyz.shape[0], float(voxel), int(radius), ref,
                                  ptr(features), ptr(knn3), int(table_slots), ptr(status), ptr(ws),
                                  ws.numel() * ws.element_size(), stream_ptr(stream)), "i4d_knn_features")


def i4d_mlp_weight_count() -> int:
    return int(load().i4d_mlp_weight_count())


def i4d_mlp_forward(features, weights, out, stream=None):
    check(load().i4d_mlp_forward(ptr(features), features.shape[0], ptr(weights), ptr(out), stream_ptr(stream)),
          "i4d_mlp_forward")


def i4d_mlp_grad_workspace_size(n: int) -> int:
    return int(load().i4d_mlp_grad_workspace_size(int(n)))


def i4d_mlp_grad(features, targets, weights, w_st, w_v, w_R, grads, loss_out, ws, stream=None):
    check(load().i4d_mlp_grad(ptr(features), ptr(targets), features.shape[0], ptr(weights), float(w_st), float(w_v),
                              float(w_R), ptr(grads), ptr(loss_out), ptr(ws), ws.numel() * ws.element_size(),
                              stream_ptr(stream)), "i4d_mlp_grad")


def i4d_init_learned(xyz, rgb, t, flag, spatial, mlp_out, n, sh_deg, st_dynamic, st_static, opacity, params,
                     fallbacks, stream=None):
    check(load().i4d_init_learned(ptr(xyz), ptr(rgb), ptr(t), ptr(flag), ptr(spatial), ptr(mlp_out), int(n),
                                  int(sh_deg), float(st_dynamic), float(st_static), float(opacity), ptr(params),
                                  ptr(fallbacks), stream_ptr(stream)), "i4d_init_learned")


def i4d_motion_targets(g: Gaussians, out, stream=None):
    check(load().i4d_motion_targets(ctypes.byref(g), ptr(out), stream_ptr(stream)), "i4d_motion_targets")
