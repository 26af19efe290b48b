"""Oracle of the two inputs of grid pruning that the paper derives from the video (test
infrastructure only): the adaptive voxel edge of Eq. 6 and the static / dynamic masks from
Otsu's thresholding of the motion-probability maps (Sec. 3.2 "Motion Probability Estimation").

Adaptive voxel edge (Eq. 6): S_v = lambda_s * (1/N) sum_i D_i / f_i, with D_i the mean depth of
frame i over its pixels with positive depth and f_i the frame's focal length (f_x).  The per-frame
depth sums are exact (each float32 depth is a multiple of 2^-32 in the depth range of a scene and
is summed as a 64-bit integer count of 2^-32 units); the rest is float64 in frame order, rounded
to float32 at the end.

Motion masks: each low-resolution probability map (h x w) is upsampled bilinearly to the frame
size (H x W) with pixel-centre alignment (source coordinate (x + 0.5) w / W - 0.5, clamped to the
map), every step a float32 operation; the upsampled values are binned into 256 bins
(bin = min(255, floor(256 p))), and Otsu's threshold is the bin t that maximises the between-class
variance w0 w1 (mu0 - mu1)^2 = (mu_T w0 - m(t))^2 / (w0 (1 - w0)) of the bin histogram (bins as
levels 0..255; the first maximum on ties; 0 where one class is empty).  A pixel is dynamic iff its
bin exceeds t.  One threshold per frame.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def adaptive_voxel(depth: np.ndarray, fx, lambda_s: float) -> np.float32:
    """depth: (F, H, W) float32; fx: focal length per frame (F,)."""
    depth = np.asarray(depth, np.float32)
    F = depth.shape[0]
    acc = 0.0
    for i in range(F):
        d = depth[i][depth[i] > 0].astype(np.float64)
        units = np.round(d * 2.0 ** 32).astype(np.int64)
        assert np.all(units.astype(np.float64) == d * 2.0 ** 32), "depth not a multiple of 2^-32"
        n = len(d)
        mean = float(int(units.sum())) / 2.0 ** 32 / n if n else 0.0
        acc += mean / float(np.float32(fx[i]))
    return np.float32(float(np.float32(lambda_s)) * (acc / F))


def upsample(prob: np.ndarray, H: int, W: int) -> np.ndarray:
    """Bilinear upsampling of one (h, w) float32 map to (H, W), float32 operation by operation."""
    prob = np.asarray(prob, np.float32)
    h, w = prob.shape
    sx_scale = f32(w) / f32(W)
    sy_scale = f32(h) / f32(H)
    out = np.empty((H, W), np.float32)
    xs = np.maximum((np.arange(W, dtype=np.float32) + f32(0.5)) * sx_scale - f32(0.5), f32(0))
    ys = np.maximum((np.arange(H, dtype=np.float32) + f32(0.5)) * sy_scale - f32(0.5), f32(0))
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    x1 = np.minimum(x0 + 1, w - 1)
    y1 = np.minimum(y0 + 1, h - 1)
    wx = (xs - x0.astype(np.float32)).astype(np.float32)
    wy = (ys - y0.astype(np.float32)).astype(np.float32)
    for j in range(H):
        a = prob[y0[j], x0]
        b = prob[y0[j], x1]
        c = prob[y1[j], x0]
        d = prob[y1[j], x1]
        top = (f32(1) - wx) * a + wx * b
        bot = (f32(1) - wx) * c + wx * d
        out[j] = (f32(1) - wy[j]) * top + wy[j] * bot
    return out


def bins(p: np.ndarray) -> np.ndarray:
    return np.minimum(np.floor(np.asarray(p, np.float32) * f32(256)).astype(np.int64), 255).clip(0, 255)


def otsu_threshold(hist: np.ndarray):
    """Returns (t, between-class variance per t) for a 256-bin histogram of counts."""
    c = np.asarray(hist, np.float64)
    N = c.sum()
    k = np.arange(256, dtype=np.float64)
    C = np.cumsum(c)                       # exact: integer counts
    M = np.cumsum(k * c)                   # exact: integers below 2^53
    muT = M[-1] / N
    w0 = C / N
    m = M / N
    sb = np.zeros(256)
    ok = (C > 0) & (C < N)
    sb[ok] = (muT * w0[ok] - m[ok]) ** 2 / (w0[ok] * (1.0 - w0[ok]))
    return int(np.argmax(sb)), sb


def otsu_masks(prob: np.ndarray, H: int, W: int):
    """prob: (F, h, w).  Returns (masks (F, H, W) uint8, thresholds (F,) int)."""
    F = prob.shape[0]
    masks = np.zeros((F, H, W), np.uint8)
    ts = np.zeros(F, np.int64)
    for i in range(F):
        b = bins(upsample(prob[i], H, W))
        t, _ = otsu_threshold(np.bincount(b.ravel(), minlength=256))
        ts[i] = t
        masks[i] = (b > t).astype(np.uint8)
    return masks, ts
