"""GPU <-> oracle parity of the fused Adam update, the loss/PSNR reductions and grid pruning,
through the C ABI."""
import math

import numpy as np
import pytest

import synth
from gpu_util import assert_prune_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _group(L, begin, end, lr0, lr1=None, decay=0):
    g = L.AdamGroup()
    g.begin, g.end = begin, end
    lr1 = lr0 if lr1 is None else lr1
    for k in range(4):
        g.lr_init[k] = lr0[k] if hasattr(lr0, "__len__") else lr0
        g.lr_final[k] = lr1[k] if hasattr(lr1, "__len__") else lr1
    g.decay_steps = decay
    return g


def test_adam_matches_oracle_with_groups_and_schedule(dev, orc):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    r = np.random.default_rng(1)
    n = 4 * 5003
    p0 = r.normal(size=n).astype(np.float32)
    groups = [_group(L, 0, 4000, 1e-3, 1e-5, decay=7),           # log-linear decay
              _group(L, 4000, 12000, [5e-2, 2.5e-3, 2.5e-3, 2.5e-3]),  # per-lane rates
              _group(L, 12000, 20000, 1e-4)]                     # floats beyond 20000: untouched
    p = torch.from_numpy(p0).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    step = torch.zeros(1, dtype=torch.int32, device=dev)
    ref = (p0.astype(np.float64), np.zeros(n), np.zeros(n))
    for s in range(1, 11):
        gr = r.normal(size=n).astype(np.float32)
        L.i4d_adam_step(p, torch.from_numpy(gr).to(dev), m, v, groups, step, 0.9, 0.999, 1e-15)
        lr = np.zeros(n)
        frac = min(s / 7, 1.0)
        lr[0:4000] = math.exp((1 - frac) * math.log(1e-3) + frac * math.log(1e-5))
        lr[4000:12000] = np.tile([5e-2, 2.5e-3, 2.5e-3, 2.5e-3], 2000)
        lr[12000:20000] = 1e-4
        # the betas as the float32 values the kernel receives (0.999 is not exact in float32)
        pn, mn, vn = orc.adam_step(ref[0], gr, ref[1], ref[2], lr, s, beta1=float(np.float32(0.9)),
                                   beta2=float(np.float32(0.999)), eps=float(np.float32(1e-15)))
        keep = np.arange(n) >= 20000
        pn[keep], mn[keep], vn[keep] = ref[0][keep], ref[1][keep], ref[2][keep]
        ref = (pn, mn, vn)
    assert int(step.item()) == 10
    got = p.cpu().numpy()
    assert np.allclose(got, ref[0], rtol=0, atol=2e-6)
    assert np.allclose(m.cpu().numpy(), ref[1], atol=1e-6)
    assert np.allclose(v.cpu().numpy(), ref[2], rtol=1e-5, atol=1e-9)
    assert np.array_equal(got[20000:], p0[20000:])


@pytest.mark.parametrize("kind", [0, 1])
def test_loss_and_gradient(dev, kind):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    r = np.random.default_rng(2)
    count = 3 * 1000 * 517 + 7
    a = r.uniform(size=count).astype(np.float32)
    b = r.uniform(size=count).astype(np.float32)
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    g = torch.empty_like(ta)
    out = torch.zeros(1, device=dev)
    L.i4d_loss(ta, tb, kind, g, out)
    d = a.astype(np.float64) - b
    if kind == 0:
        want, wg = np.abs(d).mean(), np.sign(d) / count
    else:
        want, wg = (d * d).mean(), 2 * d / count
    assert float(out.item()) == pytest.approx(want, rel=1e-5)
    assert np.allclose(g.cpu().numpy(), wg, rtol=1e-6, atol=1e-12)
    L.i4d_psnr(ta, tb, out)
    assert float(out.item()) == pytest.approx(10 * math.log10(1 / (d * d).mean()), abs=1e-4)


def _prune_gpu(xyz, rgb, t, dyn, vs, vd, k, slots=1 << 20):
    import torch
    from paper_2510_01119_gb300.prune import Pruner
    pr = Pruner(xyz.shape[0], slots)
    f = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pr.prune_xyz(f(xyz), f(rgb), f(t), f(dyn), vs, vd, k)
    return pr.result()


@pytest.mark.parametrize("min_support", [1, 2, 5])
def test_prune_xyz_kept_set_bit_exact(dev, orc, min_support):
    r = np.random.default_rng(50 + min_support)
    n = 200000
    xyz = (r.normal(size=(n, 3)) * 0.4).astype(np.float32)
    rgb = r.uniform(size=(n, 3)).astype(np.float32)
    t = r.uniform(size=n).astype(np.float32)
    dyn = (r.uniform(size=n) < 0.25).astype(np.uint8)
    got = _prune_gpu(xyz, rgb, t, dyn, 0.02, 0.05, min_support)
    want = orc.prune(xyz, 0.02, 0.05, min_support, rgb=rgb, t=t, dyn=dyn)
    assert np.array_equal(got["rep"].astype(np.int64), want["rep"].astype(np.int64))
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["flag"], want["flag"])
    assert np.allclose(got["xyz"], want["centroid"], rtol=1e-6, atol=1e-7)
    assert np.allclose(got["rgb"], want["rgb"], atol=1e-6)
    assert np.allclose(got["t"], want["t"], atol=1e-6)


@pytest.mark.parametrize("variant", ["full", "lite"])
def test_prune_variants_bit_exact(dev, orc, variant):
    """The Full model (dynamic points unpruned, voxel_dynamic = 0) and the Lite model (one coarse
    voxel for both flags): kept set, counts and flags bit-exact, centroids to float rounding."""
    r = np.random.default_rng(60)
    n = 150000
    xyz = (r.normal(size=(n, 3)) * 0.4).astype(np.float32)
    rgb = r.uniform(size=(n, 3)).astype(np.float32)
    t = r.uniform(size=n).astype(np.float32)
    dyn = (r.uniform(size=n) < 0.2).astype(np.uint8)
    vs, vd, k = (0.01, 0.0, 3) if variant == "full" else (0.04, 0.04, 2)
    got = _prune_gpu(xyz, rgb, t, dyn, vs, vd, k, slots=1 << 18)
    want = orc.prune(xyz, vs, vd, k, rgb=rgb, t=t, dyn=dyn)
    assert np.array_equal(got["rep"].astype(np.int64), want["rep"].astype(np.int64))
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["flag"], want["flag"])
    assert np.allclose(got["xyz"], want["centroid"], rtol=1e-6, atol=1e-7)
    assert np.allclose(got["t"], want["t"], atol=1e-6)
    if variant == "full":
        assert int(got["flag"].sum()) == int(dyn.sum())


def _prune_video_oracle(orc, vid, vs, vd, k):
    """The oracle's pruning of a depth video: the float32 reading of Eq. 5, then the group-by."""
    F, H, W = vid["depth"].shape
    pts = orc.backproject_video_f32(vid)
    rgb = vid["rgb"].reshape(-1, 3).astype(np.float32) / np.float32(255.0)
    t = np.repeat(np.asarray(vid["times"], np.float32), H * W)
    return orc.prune(pts, vs, vd, k, rgb=rgb, t=t, dyn=vid["dyn"].reshape(-1))


@pytest.mark.parametrize("min_support", [1, 3])
def test_prune_depth_video_bit_exact(dev, orc, min_support):
    """Depth maps -> fused back-projection (Eq. 5) + pruning, against the oracle on the same float32
    reading of Eq. 5: the kept set, counts and flags are equal, with no exclusions."""
    import torch
    from paper_2510_01119_gb300.prune import Pruner
    from paper_2510_01119_gb300.rasterizer import cameras_tensor
    vid = synth.depth_video(2, n_frames=200, W=160, H=90, frames=list(range(0, 200, 20)))
    F = len(vid["cams"])
    S = 0.02
    pr = Pruner(F * 160 * 90, 1 << 19)
    pr.prune_depth(torch.from_numpy(vid["depth"]).cuda(), torch.from_numpy(vid["rgb"]).cuda(),
                   torch.from_numpy(vid["dyn"]).cuda(), cameras_tensor(vid["cams"]), S, S, min_support)
    got = pr.result()
    want = _prune_video_oracle(orc, vid, S, S, min_support)
    assert len(want["rep"]) > 10000
    assert_prune_equal(got, want)


def test_fp32_peak_probe_is_plausible(dev):
    """The measured FP32 FMA throughput (the compositing roofline's denominator) lies between half
    and 1.1x of SMs x 128 lanes x 2 FLOP x the fastest clock a GB300 runs (2.1 GHz)."""
    import torch
    from paper_2510_01119_gb300 import _lib as L
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = sms * 128 * 2 * 2.1e9 / 1e12
    peak = L.i4d_measure_fp32_peak()
    assert 0.5 * nominal < peak < 1.1 * nominal, (peak, nominal)
