"""GPU <-> oracle parity of the photometric loss (1 - lambda) L1 + lambda (1 - SSIM) and its
gradient, through the C ABI, on ragged multi-view batches and at the training step's full size."""
import numpy as np
import pytest

from gpu_util import rel_l2
from oracle import ssim as OS

pytestmark = pytest.mark.gpu

LAM = 0.2


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _images(seed, sizes):
    """Images in [0, 1] with structure at several scales, and targets near them."""
    r = np.random.default_rng(seed)
    imgs, tgts = [], []
    for W, H in sizes:
        yy, xx = np.mgrid[0:H, 0:W]
        base = 0.5 * r.uniform(size=(3, H, W)) + \
            0.25 * (1 + np.sin(xx / 7.0 + r.uniform(0, 6)) * np.cos(yy / 5.0))[None]
        base = np.clip(base, 0, 1).astype(np.float32)
        imgs.append(base)
        tgts.append(np.clip(base + r.normal(0, 0.08, size=base.shape), 0, 1).astype(np.float32))
    return imgs, tgts


def _gpu(sizes, imgs, tgts, dev, lam=LAM):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    views = L.make_views(sizes, (16, 16))
    flat = lambda xs: torch.from_numpy(np.concatenate([x.ravel() for x in xs])).to(dev)
    img, tgt = flat(imgs), flat(tgts)
    dL = torch.full_like(img, 123.0)                       # overwritten, not accumulated
    loss = torch.zeros(1, device=dev)
    ssim = torch.zeros(1, device=dev)
    ws = torch.empty(L.i4d_photometric_loss_workspace_size(views), dtype=torch.uint8, device=dev)
    L.i4d_photometric_loss(views, img, tgt, lam, dL, loss, ssim, ws)
    out, off = [], 0
    g = dL.cpu().numpy().astype(np.float64)
    for W, H in sizes:
        out.append(g[off:off + 3 * W * H].reshape(3, H, W))
        off += 3 * W * H
    return float(loss.item()), float(ssim.item()), out


def _oracle(imgs, tgts, lam=LAM):
    imgs = [x.astype(np.float64) for x in imgs]
    tgts = [x.astype(np.float64) for x in tgts]
    loss, grads = OS.photometric_loss(imgs, tgts, lam)
    total = sum(im.size for im in imgs)
    s = sum(OS.ssim(im, t) * im.size for im, t in zip(imgs, tgts)) / total
    return loss, s, grads


@pytest.mark.parametrize("sizes", [[(37, 29)], [(64, 48), (33, 17), (16, 16)], [(5, 3)]])
def test_photometric_loss_matches_oracle_on_ragged_views(dev, sizes):
    imgs, tgts = _images(1, sizes)
    loss, s, g = _gpu(sizes, imgs, tgts, dev)
    want_loss, want_s, want_g = _oracle(imgs, tgts)
    assert loss == pytest.approx(want_loss, rel=1e-5)
    assert s == pytest.approx(want_s, abs=2e-5)
    got = np.concatenate([x.ravel() for x in g])
    want = np.concatenate([x.ravel() for x in want_g])
    assert rel_l2(got, want) < 1e-4
    # pixels whose L1 sign could flip in FP32 are left out of the element-wise check
    diff = np.abs(np.concatenate([(a.astype(np.float64) - b).ravel() for a, b in zip(imgs, tgts)]))
    ok = diff > 1e-6
    assert np.abs(got - want)[ok].max() < 1e-4 * np.abs(want).max()


def test_identical_images_give_zero_loss_and_unit_ssim(dev):
    sizes = [(40, 24), (17, 9)]
    imgs, _ = _images(2, sizes)
    loss, s, g = _gpu(sizes, imgs, imgs, dev)
    assert s == pytest.approx(1.0, abs=1e-5) and abs(loss) < 1e-5
    assert max(np.abs(x).max() for x in g) < 1e-8


def test_full_size_batch_matches_oracle(dev):
    """Full-size views of the training batch, 2 x 960x540 + 2 x 480x270 (the oracle sees every pixel)."""
    sizes = [(960, 540), (480, 270), (960, 540), (480, 270)]
    imgs, tgts = _images(3, sizes)
    loss, s, g = _gpu(sizes, imgs, tgts, dev)
    want_loss, want_s, want_g = _oracle(imgs, tgts)
    assert loss == pytest.approx(want_loss, rel=1e-5)
    assert s == pytest.approx(want_s, abs=2e-5)
    assert rel_l2(np.concatenate([x.ravel() for x in g]), np.concatenate([x.ravel() for x in want_g])) < 1e-4


def test_train_step_with_dssim_lowers_the_loss(dev):
    """Training steps with the L1 + D-SSIM loss on a small scene reduce the loss."""
    import synth
    from paper_2510_01119_gb300 import rasterizer as R
    from paper_2510_01119_gb300 import train as T
    g = synth.gaussians_uniform(0)
    hidden = synth.gaussians_uniform(1)
    sizes = [(128, 96), (64, 48)]
    cams = R.cameras_tensor([synth.camera(W, H, 60.0, time=0.5) for W, H in sizes], dev)
    hr = R.Rasterizer(2000, 0, 0, sizes)
    target = hr.forward(R.pack_params(hidden, dev), cams).clone()
    step = T.TrainStep(R.pack_params(g, dev), 2000, 0, 0, sizes, steps=100, dssim=T.DSSIM_LAMBDA)
    step.cams.copy_(cams)
    step.target.copy_(target)
    step.rast.forward(step.params, step.cams)
    losses = []
    for _ in range(30):
        step.run()
        losses.append(float(step.loss.item()))
    assert all(np.isfinite(losses)) and losses[-1] < losses[0]
    assert 0.0 < float(step.ssim.item()) <= 1.0
