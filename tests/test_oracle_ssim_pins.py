"""Pins of the D-SSIM oracle (oracle/ssim.py) against facts outside it: scipy's Gaussian filter
for the windowed moments, closed forms of SSIM for identical, constant and affinely related
images, symmetry, and central finite differences of the gradient."""
import numpy as np
import pytest

from oracle import ssim as OS

ndi = pytest.importorskip("scipy.ndimage")


def _scipy_blur(m):
    # scipy's Gaussian kernel: exp(-x^2 / (2 sigma^2)) on |x| <= int(truncate sigma + 0.5), normalised
    return ndi.gaussian_filter(np.asarray(m, np.float64), sigma=OS.SIGMA, truncate=OS.RADIUS / OS.SIGMA,
                               mode="constant", cval=0.0)


def test_windowed_moments_match_scipy_gaussian_filter():
    r = np.random.default_rng(0)
    x = r.uniform(size=(23, 31))
    w = OS.window()
    assert w.shape == (11, 11) and w.sum() == pytest.approx(1.0, abs=1e-15)
    for m in (x, x * x, np.eye(23, 31)):
        np.testing.assert_allclose(OS._windowed(m, w), _scipy_blur(m), rtol=0, atol=1e-13)


def test_ssim_of_identical_images_is_one():
    x = np.random.default_rng(1).uniform(size=(3, 20, 17))
    assert OS.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(OS.ssim_grad(x, x), 0.0, atol=1e-12)


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.7, 0.2
    S, _ = OS.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    want = (2 * a * b + OS.C1) / (a * a + b * b + OS.C1)
    np.testing.assert_allclose(S[5:-5, 5:-5], want, rtol=1e-12)
    # at the border the zero padding lowers the window means, so SSIM differs there
    assert abs(S[0, 0] - want) > 1e-3


def test_affine_relation_closed_form_from_scipy_moments():
    """y = alpha x + beta: in the interior mu_y = alpha mu_x + beta, var_y = alpha^2 var_x,
    cov = alpha var_x, so SSIM follows from x's moments alone."""
    r = np.random.default_rng(2)
    x = r.uniform(size=(32, 28))
    alpha, beta = 0.6, 0.25
    y = alpha * x + beta
    S, _ = OS.ssim_map(x, y)
    mx = _scipy_blur(x)
    vx = _scipy_blur(x * x) - mx * mx
    my = alpha * mx + beta
    want = (2 * mx * my + OS.C1) * (2 * alpha * vx + OS.C2) / ((mx * mx + my * my + OS.C1) *
                                                                (vx * (1 + alpha * alpha) + OS.C2))
    np.testing.assert_allclose(S[5:-5, 5:-5], want[5:-5, 5:-5], rtol=1e-9)


def test_ssim_is_symmetric():
    r = np.random.default_rng(3)
    x, y = r.uniform(size=(3, 15, 19)), r.uniform(size=(3, 15, 19))
    assert OS.ssim(x, y) == pytest.approx(OS.ssim(y, x), abs=1e-14)


def test_ssim_gradient_matches_central_differences():
    r = np.random.default_rng(4)
    x, y = r.uniform(size=(3, 14, 13)), r.uniform(size=(3, 14, 13))
    g = OS.ssim_grad(x, y)
    h = 1e-6
    for _ in range(25):
        idx = (r.integers(3), r.integers(14), r.integers(13))
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (OS.ssim(xp, y) - OS.ssim(xm, y)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_photometric_loss_gradient_matches_central_differences():
    r = np.random.default_rng(5)
    imgs = [r.uniform(size=(3, 10, 12)), r.uniform(size=(3, 6, 8))]
    tgts = [r.uniform(size=(3, 10, 12)), r.uniform(size=(3, 6, 8))]
    loss, grads = OS.photometric_loss(imgs, tgts, 0.2)
    h = 1e-7
    for _ in range(20):
        v = int(r.integers(2))
        idx = tuple(int(r.integers(s)) for s in imgs[v].shape)
        if abs(imgs[v][idx] - tgts[v][idx]) < 1e-4:
            continue                                # the L1 kink
        p = [im.copy() for im in imgs]
        m = [im.copy() for im in imgs]
        p[v][idx] += h
        m[v][idx] -= h
        fd = (OS.photometric_loss(p, tgts, 0.2)[0] - OS.photometric_loss(m, tgts, 0.2)[0]) / (2 * h)
        assert grads[v][idx] == pytest.approx(fd, rel=1e-4, abs=1e-9)
