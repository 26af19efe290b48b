"""Pins of the pruning-input oracle (oracle/prune_inputs.py): the adaptive voxel edge of Eq. 6 in
closed form, bilinear upsampling against torch's interpolate and a linear ramp, and Otsu's
threshold against a brute-force minimisation of the within-class variance."""
import numpy as np
import pytest

from oracle import prune_inputs as PI


def test_adaptive_voxel_closed_forms():
    F, H, W = 4, 6, 5
    d = np.full((F, H, W), 3.0, np.float32)
    assert PI.adaptive_voxel(d, np.full(F, 500.0), 1.5) == pytest.approx(1.5 * 3.0 / 500.0, rel=1e-7)
    # frames with different depths and focal lengths: the mean of D_i / f_i
    d2 = np.stack([np.full((H, W), v, np.float32) for v in (1.0, 2.0, 4.0, 8.0)])
    f = np.array([100.0, 200.0, 100.0, 400.0])
    assert PI.adaptive_voxel(d2, f, 1.0) == pytest.approx(np.mean([0.01, 0.01, 0.04, 0.02]), rel=1e-7)
    # pixels without depth do not count
    d3 = d.copy()
    d3[:, :3] = 0.0
    d3[:, 3:] = 5.0
    assert PI.adaptive_voxel(d3, np.full(F, 500.0), 1.0) == pytest.approx(5.0 / 500.0, rel=1e-7)
    # depth scaled by two (exactly) scales the edge by two
    r = np.random.default_rng(0)
    d4 = r.uniform(1, 10, size=(F, H, W)).astype(np.float32)
    assert PI.adaptive_voxel(2 * d4, f, 1.0) == 2 * PI.adaptive_voxel(d4, f, 1.0)


def test_upsample_matches_torch_interpolate():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(1)
    for (h, w, H, W) in ((5, 7, 40, 56), (45, 80, 360, 640), (3, 3, 7, 11)):
        m = r.uniform(size=(h, w)).astype(np.float32)
        want = torch.nn.functional.interpolate(torch.from_numpy(m)[None, None], size=(H, W), mode="bilinear",
                                               align_corners=False)[0, 0].numpy()
        np.testing.assert_allclose(PI.upsample(m, H, W), want, atol=2e-7)


def test_upsample_reproduces_a_linear_ramp():
    h, w, H, W = 6, 9, 48, 72
    m = np.tile((np.arange(w, dtype=np.float32) / (w - 1))[None], (h, 1))
    up = PI.upsample(m, H, W).astype(np.float64)
    sx = np.clip((np.arange(W) + 0.5) * w / W - 0.5, 0, w - 1)
    np.testing.assert_allclose(up, np.tile(sx / (w - 1), (H, 1)), atol=1e-6)


def _within_class_argmin(b):
    best, arg = np.inf, 0
    for t in range(256):
        lo, hi = b[b <= t].astype(np.float64), b[b > t].astype(np.float64)
        if len(lo) == 0 or len(hi) == 0:
            continue
        wv = len(lo) * lo.var() + len(hi) * hi.var()
        if best == np.inf or wv < best - 1e-9 * max(best, 1.0):
            best, arg = wv, t
    return arg


def test_otsu_maximum_is_the_within_class_minimum():
    r = np.random.default_rng(2)
    for seed in range(4):
        p = np.clip(np.concatenate([r.normal(0.2 + 0.1 * seed, 0.08, 3000), r.normal(0.75, 0.1, 1200)]), 0, 1)
        b = PI.bins(p.astype(np.float32))
        t, _ = PI.otsu_threshold(np.bincount(b, minlength=256))
        assert t == _within_class_argmin(b)


def test_otsu_masks_separate_two_clusters():
    r = np.random.default_rng(3)
    F, h, w = 2, 8, 10
    prob = np.clip(r.normal(0.1, 0.03, size=(F, h, w)), 0, 1).astype(np.float32)
    prob[:, 2:5, 3:7] = np.clip(r.normal(0.9, 0.03, size=(F, 3, 4)), 0, 1)
    masks, ts = PI.otsu_masks(prob, 64, 80)
    up = np.stack([PI.upsample(prob[i], 64, 80) for i in range(F)])
    assert np.all(masks[up > 0.8] == 1) and np.all(masks[up < 0.2] == 0)
    assert np.all((ts > 0.2 * 256) & (ts < 0.8 * 256))
