"""Oracle of the D-SSIM term of the photometric loss (test infrastructure only), in float64.

Sec. 4.1 trains with the loss weights of standard 3D Gaussian splatting, whose photometric loss is
(1 - lambda) L1 + lambda (1 - SSIM) with lambda = 0.2.  SSIM (Wang et al., 2004) is computed per
channel with an 11 x 11 Gaussian window of standard deviation 1.5 (weights normalised to sum 1),
windows centred on every pixel with zeros outside the image, C1 = 0.01^2, C2 = 0.03^2, and the
SSIM map averaged over pixels and channels:

    mu_x = w * x,  s_xx = w * x^2,  s_xy = w * (x y)        (windowed moments, zero padding)
    var_x = s_xx - mu_x^2,  cov = s_xy - mu_x mu_y
    S = (2 mu_x mu_y + C1)(2 cov + C2) / ((mu_x^2 + mu_y^2 + C1)(var_x + var_y + C2))

The gradient is written out from the chain rule through the moments: with
a = dS/dmu_x, b = dS/ds_xx, c = dS/ds_xy at each window centre q,
dS_mean/dx_p = (1/N) sum_q w(p - q) (a_q + 2 x_p b_q + y_p c_q).
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5


def window() -> np.ndarray:
    """The 11 x 11 Gaussian window (sum 1)."""
    x = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-x * x / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def _windowed(m: np.ndarray, w: np.ndarray) -> np.ndarray:
    """out[i, j] = sum_{u,v} w[u, v] m[i + u - R, j + v - R], zeros outside the image (the window is
    symmetric, so this is also the convolution)."""
    H, W = m.shape
    pad = np.zeros((H + 2 * RADIUS, W + 2 * RADIUS))
    pad[RADIUS:RADIUS + H, RADIUS:RADIUS + W] = m
    out = np.zeros((H, W))
    for u in range(2 * RADIUS + 1):
        for v in range(2 * RADIUS + 1):
            out += w[u, v] * pad[u:u + H, v:v + W]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray):
    """x, y: (H, W) one channel.  Returns (S map, (a, b, c) partial-derivative maps)."""
    w = window()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _windowed(x, w), _windowed(y, w)
    sxx, syy, sxy = _windowed(x * x, w), _windowed(y * y, w), _windowed(x * y, w)
    vx, vy, cov = sxx - mx * mx, syy - my * my, sxy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cov + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    S = A1 * A2 / (B1 * B2)
    # S as a function of (mu_x, s_xx, s_xy) with mu_y, s_yy fixed
    a = 2 * my * (A2 - A1) / (B1 * B2) - 2 * mx * S * (1.0 / B1 - 1.0 / B2)
    b = -S / B2
    c = 2 * A1 / (B1 * B2)
    return S, (a, b, c)


def ssim(img: np.ndarray, tgt: np.ndarray) -> float:
    """Mean SSIM of a (3, H, W) image against its target."""
    return float(np.mean([ssim_map(img[ch], tgt[ch])[0] for ch in range(img.shape[0])]))


def ssim_grad(img: np.ndarray, tgt: np.ndarray) -> np.ndarray:
    """d(mean SSIM)/d(img) for a (3, H, W) image (the target held fixed)."""
    w = window()
    n = img.size
    out = np.zeros(img.shape)
    for ch in range(img.shape[0]):
        _, (a, b, c) = ssim_map(img[ch], tgt[ch])
        x = np.asarray(img[ch], np.float64)
        y = np.asarray(tgt[ch], np.float64)
        out[ch] = (_windowed(a, w) + 2 * x * _windowed(b, w) + y * _windowed(c, w)) / n
    return out


def photometric_loss(imgs, tgts, lam: float = 0.2):
    """(1 - lam) L1 + lam (1 - SSIM) over a list of (3, H, W) views: L1 is the mean absolute error
    over every pixel and channel of all views; SSIM is each view's mean, weighted by its pixel count.
    Returns (loss, [dL/dimg per view]); d|e|/de = sign(e) (0 at 0)."""
    total = sum(im.size for im in imgs)
    l1 = sum(np.abs(np.asarray(im, np.float64) - t).sum() for im, t in zip(imgs, tgts)) / total
    s = sum(ssim(im, t) * im.size for im, t in zip(imgs, tgts)) / total
    grads = []
    for im, t in zip(imgs, tgts):
        g_l1 = np.sign(np.asarray(im, np.float64) - t) / total
        g_s = ssim_grad(im, t) * (im.size / total)
        grads.append((1 - lam) * g_l1 - lam * g_s)
    return (1 - lam) * l1 + lam * (1 - s), grads
