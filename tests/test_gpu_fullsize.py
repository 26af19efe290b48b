"""GPU <-> oracle parity at the full workload sizes, in the launch configuration the bench uses, on
sampled outputs the oracle computes one by one: sampled pixels of the forward, and the gradient of
a loss that lives only on those pixels (both sides get the same sparse upstream gradient)."""
import numpy as np
import pytest

import synth
from gpu_util import (DEPTH_MARGIN, FLAG_MARGIN, GRAD_TOL, IMG_TOL, IMPACT_MIN, assert_init_equal,
                      assert_prune_equal, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _sampled_parity(orc, g, cams, n_pix, seed, dev, grad_keys, min_checked=0.95, tile_check=False):
    """Forward: every sampled pixel matches the oracle to IMG_TOL; a pixel with a decision that
    float32 may take either way (a threshold, the T stop, the order of near-equal depths) must match
    one of its valid colours, and only pixels with too many such branches to list go unchecked
    (fewer than 1 - min_checked).  Backward: the gradient of a loss on the sampled pixels without
    such decisions, against the oracle's.  With tile_check, the whole (tile, id) list of the batch
    is also checked against the oracle's binning."""
    import torch
    from gpu_util import MAX_ALT, match_alternatives
    from paper_2510_01119_gb300 import rasterizer as R
    n = g["mean4"].shape[0]
    rast = R.Rasterizer(n, g["sh_deg"], g.get("mode", 0), [(c["W"], c["H"]) for c in cams])
    params = R.pack_params(g)
    camt = R.cameras_tensor(cams)
    rast.forward(params, camt)
    imgs = [x.cpu().numpy() for x in rast.split_images()]
    rng = np.random.default_rng(seed)
    upstream, Ps = [], []
    want = None
    bad = unchecked = by_alt = 0
    worst = 0.0
    for v, cam in enumerate(cams):
        W, H = cam["W"], cam["H"]
        pix = np.sort(rng.choice(W * H, n_pix, replace=False)).astype(np.int32)
        P = orc.project(g, cam)
        Ps.append(P)
        oimg, T, nc, mg, dmg = orc.render(P, cam, pix=pix, depth_margin=True, impact_min=IMPACT_MIN)
        fl = (mg < FLAG_MARGIN) | (dmg < DEPTH_MARGIN)
        got = imgs[v].reshape(3, -1)[:, pix].T
        err = np.abs(got - oimg).max(axis=1)
        if fl.any():
            alt, n_alt = orc.render_alternatives(P, cam, pix[fl], FLAG_MARGIN, DEPTH_MARGIN, IMPACT_MIN, MAX_ALT)
            err[fl] = match_alternatives(got[fl], [alt[k, :m] if m > 0 else None for k, m in enumerate(n_alt)])
            by_alt += int((n_alt > 0).sum())
        skip = np.isnan(err)
        bad += int(((err > IMG_TOL) & ~skip).sum())
        unchecked += int(skip.sum())
        worst = max(worst, float(err[~skip].max()))
        up = rng.normal(size=(n_pix, 3)) * 1e-2
        up[fl] = 0.0
        dense = np.zeros((3, W * H), np.float32)
        dense[:, pix] = up.T
        upstream.append(dense.reshape(-1))
        _, gr = orc.render_bwd(g, cam, up, pix=pix)
        want = gr if want is None else {k: want[k] + gr[k] for k in want}
    total = n_pix * len(cams)
    print(f"sampled pixels: {total}, checked against their valid colours {by_alt}, unchecked {unchecked}, "
          f"worst {worst:.2e}")
    assert bad == 0, (bad, unchecked, by_alt)
    assert total - unchecked >= min_checked * total, (unchecked, by_alt)
    if tile_check:
        from gpu_util import check_tile_lists
        tiles, ids = rast.tile_lists()
        rep = check_tile_lists(orc, tiles, ids, Ps, cams)
        print("tile lists:", rep)
        assert rep["flagged_needed_pairs"] < 1e-3 * rep["needed"]
    rast.backward(params, camt, torch.from_numpy(np.concatenate(upstream)).to(dev))
    got = R.unpack_params(rast.grads, n, g["sh_deg"])
    errs = {k: rel_l2(got[k], want[k]) for k in grad_keys}
    assert all(e < GRAD_TOL for e in errs.values()), errs
    return total - unchecked


def _gpu_knn3_matches(xyz, want, dev):
    """The neighbourhood kernel's 3-NN scale over all ~1.13M kept points equals the oracle's."""
    import torch
    from paper_2510_01119_gb300 import _lib as L
    n = xyz.shape[0]
    slots = 1 << int(np.ceil(np.log2(2 * n)))
    x = torch.from_numpy(xyz).to(dev)
    feats = torch.empty(n, 64, device=dev)
    knn3 = torch.empty(n, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(L.i4d_knn_workspace_size(n, slots), dtype=torch.uint8, device=dev)
    L.i4d_knn_features(x, None, None, None, synth.PRUNE_VOXEL, 2, (0.0, 0.0, 0.0), feats, knn3, slots, status, ws)
    assert int(status.item()) == 0
    np.testing.assert_allclose(knn3.cpu().numpy(), want, rtol=2e-6, atol=0)
    del feats, ws


def test_surfaces_200k_sh3_960x540_sampled(dev, orc):
    """The 200k-Gaussian surfaces workload (SH degree 3) in one 960x540 arc view."""
    g = synth.gaussians_surfaces(1)
    cams = [synth.arc_camera(57, 200, 960, 540, time=0.37)]
    _sampled_parity(orc, g, cams, 1500, 11, dev, ("mean4", "logscale4", "ql", "qr", "opacity", "rgb", "sh"),
                    tile_check=True)


@pytest.fixture(scope="module")
def room(orc):
    """The bench's room video (200 frames of 640x360, 46.08 M points) and the oracle's pruning of it
    (float32 reading of Eq. 5, voxel 0.01, support 3)."""
    vid = synth.depth_video(2)
    F, H, W = vid["depth"].shape
    pts = orc.backproject_video_f32(vid)
    res = orc.prune(pts, synth.PRUNE_VOXEL, synth.PRUNE_VOXEL, synth.PRUNE_MIN_SUPPORT,
                    rgb=vid["rgb"].reshape(-1, 3).astype(np.float32) / np.float32(255.0),
                    t=np.repeat(np.asarray(vid["times"], np.float32), H * W), dyn=vid["dyn"].reshape(-1))
    del pts
    return vid, res


def test_prune_room_video_bit_exact_full_size(dev, room):
    """The bench's pruning call (46.08 M back-projected points, 2^22 table slots, one launch of
    each kernel) keeps exactly the oracle's voxels: representatives, counts and flags equal."""
    import torch
    from paper_2510_01119_gb300.prune import Pruner
    from paper_2510_01119_gb300.rasterizer import cameras_tensor
    vid, want = room
    F, H, W = vid["depth"].shape
    pr = Pruner(F * W * H, 1 << 22, capacity=1 << 22, device=dev)
    pr.prune_depth(torch.from_numpy(vid["depth"]).to(dev), torch.from_numpy(vid["rgb"]).to(dev),
                   torch.from_numpy(vid["dyn"]).to(dev), cameras_tensor(vid["cams"], dev), synth.PRUNE_VOXEL,
                   synth.PRUNE_VOXEL, synth.PRUNE_MIN_SUPPORT)
    got = pr.result()
    assert len(want["rep"]) > 1_000_000
    assert_prune_equal(got, want)
    del pr
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def room_knn3(room):
    """The oracle's 3-NN spatial scale of every kept voxel of the room (the bench's initialisation)."""
    from oracle import learned as OL
    _, res = room
    return OL.knn3_scale(res["centroid"].astype(np.float32), synth.PRUNE_VOXEL, radius=2)


def test_init_and_motion_targets_full_size(dev, room, room_knn3):
    """The bench's initialisation call (i4d_init_learned without proposals, per-point 3-NN scale)
    on the ~1.13M kept voxels, the same call with MLP-shaped proposals (some degenerate), and the
    motion targets of the result: element by element against the oracle."""
    import torch
    from oracle import learned as OL
    from paper_2510_01119_gb300 import _lib as L
    from paper_2510_01119_gb300 import rasterizer as R
    _, res = room
    n = len(res["rep"])
    pr = dict(res, centroid=res["centroid"].astype(np.float32), rgb=res["rgb"].astype(np.float32),
              t=res["t"].astype(np.float32))
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    xyz, rgb, t, flag = f(pr["centroid"]), f(pr["rgb"]), f(pr["t"]), f(pr["flag"])
    spatial = room_knn3.astype(np.float32)
    r = np.random.default_rng(13)
    y = r.normal(size=(n, 12)).astype(np.float32)
    y[:, 0] = r.normal(-3.5, 1.0, n)
    y[r.choice(n, 1000, replace=False), 4:8] = 0.0
    params = torch.empty(5 * n * 4, device=dev)
    fb = torch.zeros(1, dtype=torch.int32, device=dev)
    for proposals in (None, y):
        L.i4d_init_learned(xyz, rgb, t, flag, f(spatial), None if proposals is None else f(proposals), n, 0,
                           2.0 / 199, 1.0, 0.1, params, fb)
        g, nfb = OL.init_learned(pr, spatial, proposals, 2.0 / 199, 1.0, 0.1)
        assert int(fb.item()) == nfb
        assert_init_equal(params.cpu().numpy().reshape(5, n, 4), g, n, 0)
    out = torch.empty(n, 20, device=dev)
    gs = L.Gaussians()
    gs.params, gs.n, gs.sh_deg, gs.mode, gs.sch_terms = params.data_ptr(), n, 0, 0, 0
    L.i4d_motion_targets(gs, out)
    got = out.cpu().numpy()
    want = OL.motion_targets(R.unpack_params(params, n, 0))
    Rm = want[:, 4:20].reshape(n, 4, 4)
    s = np.exp(params.cpu().numpy().reshape(5, n, 4)[1].astype(np.float64))
    Sig = np.einsum("nik,nk,njk->nij", Rm, s * s, Rm)
    scale = np.sqrt(np.stack([Sig[:, a, a] for a in range(3)], 1) / Sig[:, 3, 3][:, None]) + np.abs(want[:, 1:4])
    assert np.all(np.abs(got[:, 1:4] - want[:, 1:4]) <= 2e-5 * scale)
    np.testing.assert_allclose(got[:, 4:20], want[:, 4:20], rtol=0, atol=2e-6)
    assert np.array_equal(got[:, 0], want[:, 0].astype(np.float32))
    del params, out
    torch.cuda.empty_cache()


def test_training_batch_1M_eight_views_sampled(dev, orc, room, room_knn3):
    """The training step's batch: ~1.13M Gaussians pruned from the 200-frame room video (by the
    oracle), 4 x 960x540 + 4 x 480x270 views at distinct times, one launch of each kernel."""
    _, res = room
    # the bench's initialisation: per-point spatial scale = mean distance to the 3 nearest kept points
    xyz = res["centroid"].astype(np.float32)
    knn3 = room_knn3
    _gpu_knn3_matches(xyz, knn3, dev)
    g = orc.init_heuristic(res, knn3, 2.0 / 199, 1.0)
    g = {k: (v.astype(np.float32) if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    frames = [3, 61, 122, 190, 17, 88, 140, 170]
    cams = [synth.arc_camera(f, 200, 960, 540) for f in frames[:4]] + \
           [synth.arc_camera(f, 200, 480, 270) for f in frames[4:]]
    # voxel centroids on the walls give many near-equal depths among the high-weight fragments, and
    # the 3-NN spatial scale overlaps ~15 of them per pixel: about 45% of the sampled pixels have
    # more than one valid order, and are checked against the colours of all of them.  The whole
    # batch's tile list (two tile-sort passes over ~10,200 tiles, a depth sort over ~7.6 M visible
    # records) is checked against the oracle's binning.
    _sampled_parity(orc, g, cams, 1000, 12, dev, ("mean4", "logscale4", "ql", "qr", "opacity", "rgb"),
                    tile_check=True)
