"""Seeded synthetic inputs shaped like the paper's monocular-video workloads.

This module creates INPUTS only (Gaussian parameters, cameras, depth maps, images); it holds
none of the method's arithmetic, and both the CUDA path and the CPU oracle consume what it
returns.  All randomness is numpy PCG64 with an explicit seed.  Arrays are float32 (the
precision the GPU path stores); the oracle widens them to float64.

The public datasets the paper evaluates on (NVIDIA Dynamic Scene, DyCheck iPhone, DAVIS) are
not available here; these scenes stand in for them with the paper's shapes: ~200-frame
monocular videos, tens of millions of back-projected points pruned to ~1 M Gaussians, and
480x270 / 960x540-class frames.
"""
from __future__ import annotations

import math

import numpy as np

MODE_FULL, MODE_ISO_ROT, MODE_ISO_IDENTITY = 0, 1, 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------------------------------
# cameras (world->camera rotation R, translation t; OpenCV axes: x right, y down, z forward)
# ------------------------------------------------------------------------------------------
def camera(W: int, H: int, fov_x_deg: float = 60.0, R=None, t=None, time: float = 0.5) -> dict:
    """Pinhole camera, square pixels, principal point at the image centre, horizontal FOV."""
    fx = W / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return dict(R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                t=np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32),
                fx=np.float32(fx), fy=np.float32(fx), cx=np.float32(W / 2.0), cy=np.float32(H / 2.0),
                W=int(W), H=int(H), time=np.float32(time))


def look_at(eye, target, up=(0.0, -1.0, 0.0)):
    """World->camera (R, t) for a camera at `eye` looking at `target` (y down in the image)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(up, z)
    if np.linalg.norm(x) < 1e-9:
        x = np.cross((1.0, 0.0, 0.0), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    return R.astype(np.float32), (-R @ eye).astype(np.float32)


def arc_camera(k: int, n_frames: int = 200, W: int = 960, H: int = 540, fov_x_deg: float = 60.0,
               time: float = None, center=(0.0, 0.0, 3.0), radius: float = 3.0, yaw_deg: float = 20.0) -> dict:
    """Frame k of a smooth arc: eye at `radius` from `center`, yaw from -yaw_deg to +yaw_deg over
    the video, looking at `center`; frame time k / (n_frames - 1) unless `time` is given."""
    u = k / max(n_frames - 1, 1)
    yaw = math.radians(-yaw_deg + 2.0 * yaw_deg * u)
    c = np.asarray(center, np.float64)
    eye = c + radius * np.array([math.sin(yaw), 0.0, -math.cos(yaw)])
    R, t = look_at(eye, c)
    return camera(W, H, fov_x_deg, R, t, u if time is None else time)


# ------------------------------------------------------------------------------------------
# Gaussian scenes
# ------------------------------------------------------------------------------------------
def random_unit_quats(r: np.random.Generator, n: int) -> np.ndarray:
    q = r.normal(size=(n, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def _empty_sh(n: int, deg: int) -> np.ndarray:
    return np.zeros((n, (deg + 1) ** 2 - 1, 3), np.float32)


def gaussians_uniform(seed: int = 0, n: int = 2000, sh_deg: int = 0, mode: int = MODE_FULL) -> dict:
    """2,000-Gaussian render workload: means U[-1,1]^3 + (0,0,3), time centres U[0,1], spatial
    log-scales N(-3,0.5), temporal log-scale N(-1.5,0.3), two random unit quaternions, RGB U[0,1],
    opacity logit N(0,1)."""
    r = rng(seed)
    mean4 = np.zeros((n, 4), np.float32)
    mean4[:, :3] = r.uniform(-1.0, 1.0, size=(n, 3)) + np.array([0.0, 0.0, 3.0])
    mean4[:, 3] = r.uniform(0.0, 1.0, size=n)
    ls = np.zeros((n, 4), np.float32)
    ls[:, :3] = r.normal(-3.0, 0.5, size=(n, 3))
    ls[:, 3] = r.normal(-1.5, 0.3, size=n)
    g = dict(mean4=mean4, logscale4=ls, ql=random_unit_quats(r, n), qr=random_unit_quats(r, n),
             opacity=r.normal(0.0, 1.0, size=n).astype(np.float32),
             rgb=r.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32), sh_deg=sh_deg, mode=mode)
    g["sh"] = (r.normal(0.0, 0.1, size=(n, (sh_deg + 1) ** 2 - 1, 3)).astype(np.float32) if sh_deg > 0
               else _empty_sh(n, 0))
    return g


def velocity_quats(v: np.ndarray, s: np.ndarray, s_t: np.ndarray):
    """Left/right quaternions of the simple 4D rotation, in the plane of (v_hat, t), whose sliced
    mean moves with velocity v for an isotropic spatial scale s and temporal scale s_t.

    With q_l = q_r = cos(th/2) + sin(th/2) v_hat the time axis maps to (sin th v_hat, cos th), and
    the conditional mean moves by (s_t^2 - s^2) sin th cos th / (s^2 sin^2 th + s_t^2 cos^2 th)
    per unit time; tan th is the smaller root of k s^2 x^2 - (s_t^2 - s^2) x + k s_t^2 = 0 for
    speed k (clamped to the largest speed the scales allow)."""
    v = np.asarray(v, np.float64)
    k = np.linalg.norm(v, axis=1)
    vhat = np.where(k[:, None] > 0, v / np.maximum(k, 1e-30)[:, None], np.array([1.0, 0.0, 0.0]))
    s2, st2 = np.asarray(s, np.float64) ** 2, np.asarray(s_t, np.float64) ** 2
    a = st2 - s2
    kmax = np.maximum(a, 0.0) / (2.0 * np.sqrt(s2 * st2))
    kk = np.minimum(k, 0.999 * kmax)
    disc = np.maximum(a * a - 4.0 * kk * kk * s2 * st2, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        tan = np.where(kk > 0, (a - np.sqrt(disc)) / (2.0 * kk * s2), 0.0)
    th = np.arctan(tan)
    q = np.zeros((v.shape[0], 4))
    q[:, 0] = np.cos(th / 2.0)
    q[:, 1:] = np.sin(th / 2.0)[:, None] * vhat
    q = q.astype(np.float32)
    return q, q.copy()


def gaussians_surfaces(seed: int = 1, n_surf: int = 5, per_surf: int = 36000, n_sph: int = 3,
                       per_sph: int = 6667, sh_deg: int = 3) -> dict:
    """200k-Gaussian render workload: Gaussians drawn like the 2,000-Gaussian case but placed on
    5 random smooth surfaces (a plane through a point of [-1,1]^2 x [2,4] with a N(0,1) normal,
    displaced by three sinusoids of amplitude U[0,0.1] and frequency U[1,4]) plus 3 spheres
    (radius U[0.2,0.4]) moving with velocities N(0,0.3)^3; SH degree 3 (base U[0,1], the 45
    other coefficients N(0,0.1))."""
    r = rng(seed)
    pts, vel, is_sph = [], [], []
    for _ in range(n_surf):
        c = np.array([r.uniform(-1, 1), r.uniform(-1, 1), r.uniform(2, 4)])
        nrm = r.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        e1 = np.cross(nrm, [1.0, 0.0, 0.0] if abs(nrm[0]) < 0.9 else [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(nrm, e1)
        uv = r.uniform(-1.0, 1.0, size=(per_surf, 2))
        a = r.uniform(0.0, 0.1, size=3)
        w = r.uniform(1.0, 4.0, size=(3, 2))
        ph = r.uniform(0.0, 2 * np.pi, size=3)
        disp = sum(a[k] * np.sin(uv @ w[k] + ph[k]) for k in range(3))
        pts.append(c + uv[:, :1] * e1 + uv[:, 1:] * e2 + disp[:, None] * nrm)
        vel.append(np.zeros((per_surf, 3)))
        is_sph.append(np.zeros(per_surf, bool))
    for _ in range(n_sph):
        c0 = np.array([r.uniform(-1, 1), r.uniform(-1, 1), r.uniform(2, 4)])
        rad = r.uniform(0.2, 0.4)
        v = r.normal(0.0, 0.3, size=3)
        d = r.normal(size=(per_sph, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(c0 + rad * d)
        vel.append(np.tile(v, (per_sph, 1)))
        is_sph.append(np.ones(per_sph, bool))
    pts = np.concatenate(pts)
    vel = np.concatenate(vel)
    is_sph = np.concatenate(is_sph)
    n = pts.shape[0]
    mean4 = np.zeros((n, 4), np.float32)
    mean4[:, 3] = r.uniform(0.0, 1.0, size=n)
    # a sphere's surface point sits on the moving centre c0 + v (t - 0.5) at its own time centre
    mean4[:, :3] = pts + vel * (mean4[:, 3:4].astype(np.float64) - 0.5)
    ls = np.zeros((n, 4), np.float32)
    ls[:, :3] = r.normal(-3.0, 0.5, size=(n, 3))
    ls[:, 3] = r.normal(-1.5, 0.3, size=n)
    ql, qr = random_unit_quats(r, n), random_unit_quats(r, n)
    # moving Gaussians: isotropic spatial scale and a rotation in the (v, t) plane
    ls[is_sph, 1] = ls[is_sph, 0]
    ls[is_sph, 2] = ls[is_sph, 0]
    qv_l, qv_r = velocity_quats(vel[is_sph], np.exp(ls[is_sph, 0]), np.exp(ls[is_sph, 3]))
    ql[is_sph], qr[is_sph] = qv_l, qv_r
    g = dict(mean4=mean4, logscale4=ls, ql=ql, qr=qr, opacity=r.normal(0.0, 1.0, size=n).astype(np.float32),
             rgb=r.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32), sh_deg=sh_deg, mode=MODE_FULL)
    g["sh"] = r.normal(0.0, 0.1, size=(n, (sh_deg + 1) ** 2 - 1, 3)).astype(np.float32)
    g["velocity"] = vel.astype(np.float32)
    return g


def random_image(seed: int, W: int, H: int) -> np.ndarray:
    """Uniform [0,1] target image, (H, W, 3) float32."""
    return rng(seed).uniform(0.0, 1.0, size=(H, W, 3)).astype(np.float32)


def subset(g: dict, idx) -> dict:
    out = {}
    for k, v in g.items():
        out[k] = v[idx] if isinstance(v, np.ndarray) else v
    return out


# ------------------------------------------------------------------------------------------
# depth-map video (ray-cast analytic room with moving spheres)
# ------------------------------------------------------------------------------------------
# side walls, floor (+y) / ceiling, back wall; extents chosen so that pruning the 200-frame
# 640x360 video at a 0.01 voxel with minimum support 3 keeps about one million voxels
PRUNE_VOXEL = 0.01
PRUNE_MIN_SUPPORT = 3
ROOM = dict(x=(-0.812, 0.812), y=(-0.448, 0.448), z_back=3.98)


def room_colour(p: np.ndarray, kind: np.ndarray) -> np.ndarray:
    """Procedural texture of the room: colour of world point p on surface `kind` (1-5 planes,
    10+ spheres), in [0, 1]."""
    tex = 0.5 + 0.25 * np.sin(7.0 * p[..., 0]) * np.cos(5.0 * p[..., 1]) + 0.25 * np.sin(3.0 * p[..., 2])
    base = np.stack([0.3 + 0.1 * (kind % 3), 0.4 + 0.1 * (kind % 2), 0.5 + 0.05 * (kind % 5)], -1)
    return np.clip(base * (0.5 + tex[..., None]), 0.0, 1.0)


def room_spheres(seed: int, room: dict = None):
    """(centres at t = 0.5, radii, velocities) of the three moving spheres of the room video."""
    room = ROOM if room is None else room
    r = rng(seed)
    sx, sy, sz = 0.4 * room["x"][1], 0.4 * room["y"][1], room["z_back"]
    c0 = np.stack([r.uniform(-sx, sx, 3), r.uniform(-sy, sy, 3), r.uniform(0.45 * sz, 0.75 * sz, 3)], axis=1)
    rad = r.uniform(0.3, 0.5, 3) * (sz / 6.5)
    vel = r.normal(0.0, 0.3, size=(3, 3))
    return c0, rad, vel, r


def room_gaussians(seed: int = 1003, n: int = 200000, video_seed: int = 2, dyn_frac: float = 0.1,
                   n_frames: int = 200, room: dict = None) -> dict:
    """Hidden 4D Gaussian scene of the room video: static Gaussians on the planes seen by the arc
    cameras (temporal scale of the whole video) and dynamic Gaussians on the three moving spheres of
    the video with seed `video_seed` (velocity encoded in the 4D rotation, temporal scale of a few
    frames), coloured by the room texture; SH degree 0, isotropic spatial scale."""
    room = ROOM if room is None else room
    r = rng(seed)
    n_dyn = int(n * dyn_frac)
    n_st = n - n_dyn
    x0, x1 = room["x"]
    y0, y1 = room["y"]
    zb = room["z_back"]
    zlo = 0.8
    # planes with their areas inside the visible box
    planes = [(5, "z", zb, (x0, x1), (y0, y1)), (1, "x", x0, (y0, y1), (zlo, zb)), (2, "x", x1, (y0, y1), (zlo, zb)),
              (3, "y", y1, (x0, x1), (zlo, zb)), (4, "y", y0, (x0, x1), (zlo, zb))]
    areas = np.array([(a[1] - a[0]) * (b[1] - b[0]) for (_, _, _, a, b) in planes])
    which = r.choice(len(planes), size=n_st, p=areas / areas.sum())
    pts = np.zeros((n_st, 3))
    kind = np.zeros(n_st, np.int64)
    for k, (kd, ax, val, ra, rb) in enumerate(planes):
        m = which == k
        u = r.uniform(ra[0], ra[1], m.sum())
        v = r.uniform(rb[0], rb[1], m.sum())
        if ax == "z":
            pts[m] = np.c_[u, v, np.full(m.sum(), val)]
        elif ax == "x":
            pts[m] = np.c_[np.full(m.sum(), val), u, v]
        else:
            pts[m] = np.c_[u, np.full(m.sum(), val), v]
        kind[m] = kd
    c0, rad, vel, _ = room_spheres(video_seed, room)
    sph = r.integers(0, 3, n_dyn)
    d = r.normal(size=(n_dyn, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t_dyn = r.uniform(0.0, 1.0, n_dyn)
    dyn_pts = c0[sph] + rad[sph, None] * d + vel[sph] * (t_dyn[:, None] - 0.5)
    mean4 = np.zeros((n, 4), np.float32)
    mean4[:n_st, :3] = pts
    mean4[:n_st, 3] = 0.5
    mean4[n_st:, :3] = dyn_pts
    mean4[n_st:, 3] = t_dyn
    ls = np.zeros((n, 4), np.float32)
    spacing = math.sqrt(areas.sum() / max(n_st, 1))
    ls[:n_st, :3] = math.log(0.6 * spacing)
    ls[:n_st, 3] = math.log(1.0)
    s_dyn = 0.6 * math.sqrt(4 * math.pi * float(np.mean(rad ** 2)) / max(n_dyn / 3, 1)) * 3
    ls[n_st:, :3] = math.log(s_dyn)
    ls[n_st:, 3] = math.log(3.0 / max(n_frames - 1, 1))
    ql = np.zeros((n, 4), np.float32)
    ql[:, 0] = 1.0
    qr = ql.copy()
    qv_l, qv_r = velocity_quats(vel[sph], np.full(n_dyn, s_dyn), np.full(n_dyn, 3.0 / max(n_frames - 1, 1)))
    ql[n_st:], qr[n_st:] = qv_l, qv_r
    rgb = np.zeros((n, 3), np.float32)
    rgb[:n_st] = room_colour(pts, kind)
    rgb[n_st:] = room_colour(dyn_pts, 10 + sph)
    return dict(mean4=mean4, logscale4=ls, ql=ql, qr=qr, opacity=np.full(n, 2.0, np.float32), rgb=rgb,
                sh=np.zeros((n, 0, 3), np.float32), sh_deg=0, mode=MODE_FULL)


def depth_video(seed: int = 2, n_frames: int = 200, W: int = 640, H: int = 360, frames=None,
                noise: float = 0.01, fov_x_deg: float = 60.0, room: dict = None):
    """Depth maps of a room (floor, back wall, two side walls; z-depth clipped to [1, 10] m) with
    3 spheres moving linearly, seen from the arc camera, with multiplicative depth noise
    (1 + noise N(0,1)).  Returns dict(depth (F,H,W) f32, rgb (F,H,W,3) u8, dyn (F,H,W) u8, cams,
    times).  `frames` selects a subset of frame indices (same values as in the full video)."""
    room = ROOM if room is None else room
    sph_c0, sph_r, sph_v, r = room_spheres(seed, room)
    frames = list(range(n_frames)) if frames is None else list(frames)
    F = len(frames)
    depth = np.zeros((F, H, W), np.float32)
    rgb = np.zeros((F, H, W, 3), np.uint8)
    dyn = np.zeros((F, H, W), np.uint8)
    cams = []
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    for fi, k in enumerate(frames):
        cam = arc_camera(k, n_frames, W, H, fov_x_deg, center=(0.0, 0.0, 3.0), radius=3.0)
        cams.append(cam)
        R = cam["R"].astype(np.float64)
        t = cam["t"].astype(np.float64)
        eye = -R.T @ t
        dc = np.stack([(px - cam["cx"]) / cam["fx"], (py - cam["cy"]) / cam["fy"], np.ones_like(px)], -1)
        dw = dc @ R                       # world ray directions, scaled so that camera z = 1
        best = np.full((H, W), np.inf)
        hit_kind = np.zeros((H, W), np.int32)
        for axis, val, kind in ((0, room["x"][0], 1), (0, room["x"][1], 2), (1, room["y"][1], 3),
                                (1, room["y"][0], 4), (2, room["z_back"], 5)):
            with np.errstate(divide="ignore", invalid="ignore"):
                s = (val - eye[axis]) / dw[..., axis]
            ok = (s > 0) & (s < best)
            best = np.where(ok, s, best)
            hit_kind = np.where(ok, kind, hit_kind)
        u = k / max(n_frames - 1, 1)
        for j in range(3):
            c = sph_c0[j] + sph_v[j] * (u - 0.5)
            oc = eye - c
            a = np.sum(dw * dw, -1)
            b = 2.0 * np.sum(dw * oc, -1)
            cc = np.dot(oc, oc) - sph_r[j] ** 2
            disc = b * b - 4 * a * cc
            with np.errstate(invalid="ignore"):
                s = (-b - np.sqrt(np.maximum(disc, 0.0))) / (2 * a)
            ok = (disc > 0) & (s > 0) & (s < best)
            best = np.where(ok, s, best)
            hit_kind = np.where(ok, 10 + j, hit_kind)
        d = np.clip(best, 1.0, 10.0)  # ray scaled to camera z = 1: the hit parameter is the z-depth
        d = d * (1.0 + noise * r.normal(size=d.shape))
        depth[fi] = d.astype(np.float32)
        hit = eye + best[..., None] * dw
        rgb[fi] = (room_colour(hit, hit_kind) * 255.0 + 0.5).astype(np.uint8)
        dyn[fi] = (hit_kind >= 10).astype(np.uint8)
    times = np.array([k / max(n_frames - 1, 1) for k in frames], np.float32)
    return dict(depth=depth, rgb=rgb, dyn=dyn, cams=cams, times=times)


def motion_prob_maps(dyn: np.ndarray, factor: int = 8, noise: float = 0.12, seed: int = 0) -> np.ndarray:
    """Low-resolution motion-probability maps (F, ceil(H/factor), ceil(W/factor)) float32 in [0, 1],
    standing in for the SLAM network's per-frame maps: the fraction of moving pixels in each
    factor x factor cell of the dynamic mask, plus seeded Gaussian noise, clipped."""
    dyn = np.asarray(dyn, np.float32)
    F, H, W = dyn.shape
    h, w = -(-H // factor), -(-W // factor)
    pad = np.zeros((F, h * factor, w * factor), np.float32)
    pad[:, :H, :W] = dyn
    frac = pad.reshape(F, h, factor, w, factor).mean(axis=(2, 4))
    r = np.random.default_rng(seed)
    return np.clip(frac + r.normal(0.0, noise, size=frac.shape), 0.0, 1.0).astype(np.float32)
