"""GPU <-> FP64 oracle parity of slice/project, tile binning, compositing and the backward,
through the C ABI (libi4d.so)."""
import numpy as np
import pytest

import synth
from gpu_util import (FLAG_MARGIN, GRAD_TOL, IMG_TOL, check_tile_lists, compare_images, flagged_gaussians,
                      gpu_records, oracle_views, rel_l2)

pytestmark = pytest.mark.gpu

GRAD_KEYS = ("mean4", "logscale4", "ql", "qr", "opacity", "rgb", "sh")


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _gpu_render(g, cams, tile=(16, 16), settings=None, capacity=None):
    from paper_2510_01119_gb300 import rasterizer as R
    rast = R.Rasterizer(g["mean4"].shape[0], g["sh_deg"], g.get("mode", 0), [(c["W"], c["H"]) for c in cams],
                        tile=tile, settings=settings, capacity=capacity)
    params = R.pack_params(g)
    camt = R.cameras_tensor(cams)
    rast.forward(params, camt)
    return rast, params, camt


def _oracle_grads(orc, g, cams, gimgs, settings=None):
    tot = None
    for cam, gi in zip(cams, gimgs):
        _, gr = orc.render_bwd(g, cam, gi.reshape(-1, 3), settings=settings)
        tot = gr if tot is None else {k: tot[k] + gr[k] for k in tot}
    return tot


def _compare_grads(rast, g, want):
    from paper_2510_01119_gb300 import rasterizer as R
    got = R.unpack_params(rast.grads, g["mean4"].shape[0], g["sh_deg"])
    got["opacity"] = got["opacity"]
    errs = {}
    for k in GRAD_KEYS:
        if k == "sh" and g["sh_deg"] == 0:
            continue
        if np.linalg.norm(want[k]) == 0 and np.linalg.norm(got[k]) == 0:
            continue
        errs[k] = rel_l2(got[k], want[k])
    return errs


def _settings_dict(orc_settings_over):
    return orc_settings_over


# --------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode,deg", [(0, 0), (1, 0), (2, 0), (0, 3)])
def test_slice_project_records_match_oracle(dev, orc, mode, deg):
    g = synth.gaussians_uniform(0, sh_deg=deg, mode=mode)
    cam = synth.camera(128, 96, 60.0, time=0.5)
    rast, _, _ = _gpu_render(g, [cam])
    n = g["mean4"].shape[0]
    rec = gpu_records(rast)
    touched = rast.touched[:n].cpu().numpy()
    P = orc.project(g, cam)
    C = orc.P
    vis = P[:, C["visible"]] != 0
    sus = flagged_gaussians(orc, [P])[0]
    ok = np.array([i not in sus for i in range(n)])
    # a Gaussian with a tile that holds a blendable pixel centre is binned, on at least that many
    # tiles; one the oracle culls is not binned (decisions within FLAG_MARGIN excepted)
    wt, wi, ws = orc.tile_lists(P, cam)
    need = np.bincount(wi[ws == 1], minlength=n)
    assert np.all(touched[ok] >= need[ok])
    assert np.all(touched[ok & ~vis] == 0)
    print(f"records: {int(ok.sum())} compared, {int((~ok).sum())} flagged")
    assert (~ok).sum() < 0.02 * n
    vis = vis & (touched > 0)
    m = vis & ok
    assert m.sum() > 500
    u, v, ca, cb, cc, ot = (rec[k][m] for k in ("u", "v", "ca", "cb", "cc", "ot"))
    r, gg, b, depth, radius = (rec[k][m] for k in ("r", "g", "b", "depth", "radius"))
    # the kept test's exponent threshold: kFalloff min(q_max, 2 ln(o_t / alpha_min))
    mthr = np.minimum(9.0, 2 * np.log(P[m, C["ot"]] * 255.0)) * (-0.5 / np.log(2.0))
    assert np.allclose(rec["m_thr"][m], mthr, rtol=0, atol=1e-4)
    assert np.allclose(u, P[m, C["u"]], rtol=0, atol=2e-3)
    assert np.allclose(v, P[m, C["v"]], rtol=0, atol=2e-3)
    assert np.allclose(depth, P[m, C["depth"]], rtol=2e-6)
    assert np.allclose(ot, P[m, C["ot"]], rtol=2e-5, atol=1e-7)
    scale = np.maximum(np.abs(P[m][:, [C["ca"], C["cb"], C["cc"]]]).max(axis=1), 1e-12)
    for got, col in ((ca, "ca"), (cb, "cb"), (cc, "cc")):
        assert np.all(np.abs(got - P[m, C[col]]) <= 2e-4 * scale)
    for got, col in ((r, "r"), (gg, "g"), (b, "b")):
        assert np.allclose(got, P[m, C[col]], atol=2e-6)
    assert np.array_equal(radius, P[m, C["radius"]])


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_tile_lists_match_oracle(dev, orc, tile):
    """The sorted (tile, id) list against the oracle's binning: every tile holding a blendable pixel
    centre listed, every other listed tile within the documented slack of the blendable box, no
    duplicate, depth order inside each tile (near-equal depths in either order)."""
    g = synth.gaussians_uniform(0)
    cams = [synth.camera(128, 96, 60.0, time=0.5), synth.camera(75, 41, 55.0, time=0.3)]
    rast, _, _ = _gpu_render(g, cams, tile=tile)
    tiles, ids = rast.tile_lists()
    Ps = [orc.project(g, c) for c in cams]
    rep = check_tile_lists(orc, tiles, ids, Ps, cams, tile)
    print("tile lists:", rep)
    assert rep["flagged_needed_pairs"] < 0.01 * rep["needed"]
    assert rep["gpu"] <= 1.5 * rep["needed"]


def test_tile_order_is_longest_first_and_stable(dev):
    """The order in which the compositing kernels take tiles: a permutation of all tiles, by
    decreasing octave of list length (floor(log2(length + 1))), tile index order inside an octave
    (over more than one 1024-tile chunk of the ordering kernel)."""
    g = synth.gaussians_uniform(0)
    cams = [synth.camera(320, 240, 60.0, time=0.5), synth.camera(75, 41, 55.0, time=0.3)]
    rast, _, _ = _gpu_render(g, cams, tile=(8, 8))
    T = rast.total_tiles
    assert T > 1024
    rg = rast.ranges[:3 * T].cpu().numpy().astype(np.int64)
    length, order = rg[1:2 * T:2] - rg[0:2 * T:2], rg[2 * T:]
    assert np.array_equal(np.sort(order), np.arange(T))
    f = np.log2(length[order] + 1.0)
    b = np.floor(f)
    near = np.abs(f - np.round(f)) < 1e-4           # float32 log2 may put these in either bucket
    loose = near[:-1] | near[1:]
    d = np.diff(b)
    assert np.all((d <= 0) | loose)
    assert np.all(np.diff(order)[(d == 0) & ~loose] > 0)
    assert len(np.unique(b)) > 3
    # every tile with a non-empty list comes before every empty one
    assert np.all(np.diff((length[order] == 0).astype(int)) >= 0)


@pytest.mark.parametrize("mode,deg", [(0, 0), (1, 0), (2, 0), (0, 3)])
def test_render_forward_matches_oracle(dev, orc, mode, deg):
    g = synth.gaussians_uniform(0, sh_deg=deg, mode=mode)
    cams = [synth.camera(128, 96, 60.0, time=0.5)]
    rast, _, _ = _gpu_render(g, cams)
    ov = oracle_views(orc, g, cams)
    gimg = [x.cpu().numpy() for x in rast.split_images()]
    bad, unchecked, worst = compare_images(gimg, ov)
    print(f"forward: {bad} bad, {unchecked} unchecked of {128 * 96}, worst {worst:.2e}")
    assert bad == 0, (bad, unchecked, worst)
    assert unchecked < 0.02 * 128 * 96
    T = rast.split_pixels(rast.T_final)[0].cpu().numpy()
    nc = rast.split_pixels(rast.n_contrib)[0].cpu().numpy()
    fl = ov[0][4] < FLAG_MARGIN
    assert np.abs(T - ov[0][2])[~fl].max() < IMG_TOL
    assert np.array_equal(nc[~fl], ov[0][3][~fl])


def test_render_backward_matches_oracle(dev, orc):
    """MSE against a uniform-random target (the 2,000-Gaussian workload), dL/dimg from the oracle's
    image and zeroed at flagged pixels (both sides get the same upstream gradient)."""
    g = synth.gaussians_uniform(0)
    cam = synth.camera(128, 96, 60.0, time=0.5)
    rast, params, camt = _gpu_render(g, [cam])
    ov = oracle_views(orc, g, [cam])
    img = ov[0][1]
    tgt = synth.random_image(0, 128, 96)
    gimg = 2.0 * (img - tgt) / img.size
    gimg[ov[0][4] < FLAG_MARGIN] = 0.0
    import torch
    dl = torch.from_numpy(gimg.transpose(2, 0, 1).astype(np.float32).reshape(-1)).to(dev)
    rast.backward(params, camt, dl)
    want = _oracle_grads(orc, g, [cam], [gimg])
    errs = _compare_grads(rast, g, want)
    assert all(e < GRAD_TOL for e in errs.values()), errs


@pytest.mark.parametrize("mode,deg", [(1, 0), (2, 0), (0, 3)])
def test_render_backward_modes_and_sh(dev, orc, mode, deg):
    g = synth.gaussians_uniform(4, n=1500, sh_deg=deg, mode=mode)
    cam = synth.camera(96, 80, 60.0, time=0.42)
    rast, params, camt = _gpu_render(g, [cam])
    ov = oracle_views(orc, g, [cam])
    gimg = np.random.default_rng(9).normal(size=ov[0][1].shape) * 1e-3
    gimg[ov[0][4] < FLAG_MARGIN] = 0.0
    import torch
    dl = torch.from_numpy(gimg.transpose(2, 0, 1).astype(np.float32).reshape(-1)).to(dev)
    rast.backward(params, camt, dl)
    errs = _compare_grads(rast, g, _oracle_grads(orc, g, [cam], [gimg]))
    assert all(e < GRAD_TOL for e in errs.values()), errs


def test_multiview_single_launch_matches_per_view_oracle(dev, orc):
    """Views at different timestamps and resolutions (ragged sizes) in one launch."""
    g = synth.gaussians_uniform(0)
    cams = [synth.camera(128, 96, 60.0, time=0.5), synth.camera(77, 45, 50.0, time=0.1),
            synth.arc_camera(40, 200, 100, 60), synth.camera(33, 129, 40.0, time=0.9)]
    rast, params, camt = _gpu_render(g, cams)
    ov = oracle_views(orc, g, cams)
    gimg = [x.cpu().numpy() for x in rast.split_images()]
    bad, flagged, worst = compare_images(gimg, ov)
    assert bad == 0, (bad, flagged, worst)
    rng = np.random.default_rng(3)
    ups = []
    for v in ov:
        u = rng.normal(size=v.img.shape) * 1e-3
        u[v.flag < FLAG_MARGIN] = 0.0
        ups.append(u)
    import torch
    dl = torch.from_numpy(np.concatenate([u.transpose(2, 0, 1).reshape(-1) for u in ups]).astype(np.float32)).to(dev)
    rast.backward(params, camt, dl)
    errs = _compare_grads(rast, g, _oracle_grads(orc, g, cams, ups))
    assert all(e < GRAD_TOL for e in errs.values()), errs


@pytest.mark.parametrize("tile", [(8, 8), (16, 8), (32, 8), (32, 16)])
def test_image_is_tile_size_invariant(dev, orc, tile):
    g = synth.gaussians_uniform(0)
    cams = [synth.camera(128, 96, 60.0, time=0.5)]
    r16, _, _ = _gpu_render(g, cams)
    rt, _, _ = _gpu_render(g, cams, tile=tile)
    a = r16.img.cpu().numpy()
    b = rt.img.cpu().numpy()
    ov = oracle_views(orc, g, cams)
    bad, _, _ = compare_images([x.cpu().numpy() for x in rt.split_images()], ov)
    assert bad == 0
    assert np.abs(a - b).max() < 1e-5


def test_empty_and_fully_culled_scenes(dev, orc):
    g = synth.gaussians_uniform(0, n=50)
    g["mean4"][:, 2] = -5.0                      # every Gaussian behind the camera
    cams = [synth.camera(40, 30, time=0.5)]
    rast, params, camt = _gpu_render(g, cams)
    assert int(rast.n_inst.item()) == 0
    img = rast.img.cpu().numpy()
    assert np.all(img == 0.0) and np.all(rast.T_final.cpu().numpy() == 1.0)
    import torch
    rast.backward(params, camt, torch.ones_like(rast.img))
    assert np.all(rast.grads.cpu().numpy() == 0.0)


def test_capacity_overflow_is_reported_and_recovered(dev, orc):
    import torch
    from paper_2510_01119_gb300 import rasterizer as R
    g = synth.gaussians_uniform(0)
    cams = [synth.camera(128, 96, 60.0, time=0.5)]
    rast = R.Rasterizer(2000, 0, 0, [(128, 96)], capacity=1000)
    params = R.pack_params(g)
    camt = R.cameras_tensor(cams)
    rast.project(params, camt)
    rast.bin()
    torch.cuda.synchronize()
    assert int(rast.status.item()) == -2 and int(rast.n_inst.item()) > 1000
    rast.forward(params, camt)                    # regrows the bins
    assert rast.capacity >= int(rast.n_inst.item())
    bad, _, _ = compare_images([x.cpu().numpy() for x in rast.split_images()], oracle_views(orc, g, cams))
    assert bad == 0


def test_autograd_function_matches_oracle(dev, orc):
    import torch
    from paper_2510_01119_gb300 import rasterizer as R
    g = synth.gaussians_uniform(6, n=800)
    cam = synth.camera(64, 48, 60.0, time=0.55)
    rast = R.Rasterizer(800, 0, 0, [(64, 48)])
    params = R.pack_params(g).requires_grad_(True)
    camt = R.cameras_tensor([cam])
    img = R.render(params, camt, rast)
    w = torch.from_numpy(np.random.default_rng(2).normal(size=img.shape[0]).astype(np.float32)).to(dev)
    ov = oracle_views(orc, g, [cam])
    fl = ov[0][4] < FLAG_MARGIN
    wnp = w.cpu().numpy().reshape(3, 48, 64)
    wnp[:, fl] = 0.0
    w = torch.from_numpy(wnp.reshape(-1)).to(dev)
    (img * w).sum().backward()
    want = _oracle_grads(orc, g, [cam], [wnp.transpose(1, 2, 0).astype(np.float64)])
    got = R.unpack_params(params.grad, 800, 0)
    for k in ("mean4", "logscale4", "ql", "qr", "opacity", "rgb"):
        assert rel_l2(got[k], want[k]) < GRAD_TOL, k
