"""Shared helpers of the GPU parity tests (comparison protocol against the FP64 oracle)."""
from typing import NamedTuple

import numpy as np

# A pixel whose oracle decisions (q <= 9, alpha >= 1/255, the T stop, o_t cull, near plane, depth
# order) sit within this relative margin of a threshold may legitimately differ between the FP32
# GPU and the FP64 oracle; every other pixel must match to IMG_TOL.
FLAG_MARGIN = 1e-4
# Two fragments whose depths differ by less than this relative gap may swap order (FP32 depth is
# good to ~2e-7 relative here).
DEPTH_MARGIN = 2e-6
IMG_TOL = 1e-4        # max-abs on rendered images
# only decisions whose flip could move the pixel by more than this are flagged
IMPACT_MIN = 0.5 * IMG_TOL
GRAD_TOL = 1e-3       # relative L2 on gradients


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class OView(NamedTuple):
    """The oracle's render of one view.  flag < FLAG_MARGIN: a decision of the pixel (a threshold,
    the T stop or the order of near-equal depths) may go either way in float32; alt: for those
    pixels, every valid colour (render_alternatives), or None when there are too many branches."""
    P: np.ndarray
    img: np.ndarray
    T: np.ndarray
    nc: np.ndarray
    flag: np.ndarray
    alt: dict


MAX_ALT = 1024


def oracle_views(orc, g, cams, settings=None, bg=(0, 0, 0)):
    """Oracle render of each view (list of OView)."""
    out = []
    for cam in cams:
        P = orc.project(g, cam, settings=settings)
        img, T, nc, mg, dmg = orc.render(P, cam, bg=bg, settings=settings, depth_margin=True, impact_min=IMPACT_MIN)
        W, H = int(cam["W"]), int(cam["H"])
        # one flag value per pixel: below FLAG_MARGIN means "may differ"
        flag = np.minimum(mg, dmg * (FLAG_MARGIN / DEPTH_MARGIN))
        flagged = np.nonzero(flag < FLAG_MARGIN)[0]
        alt = {}
        if len(flagged):
            a, na = orc.render_alternatives(P, cam, flagged, FLAG_MARGIN, DEPTH_MARGIN, IMPACT_MIN, MAX_ALT, bg=bg,
                                            settings=settings)
            alt = {int(p): (a[k, :na[k]] if na[k] > 0 else None) for k, p in enumerate(flagged)}
        out.append(OView(P, img.reshape(H, W, 3), T.reshape(H, W), nc.reshape(H, W), flag.reshape(H, W), alt))
    return out


def match_alternatives(got, alt):
    """Max-abs error of each pixel of `got` (m, 3) against the closest of its valid colours (alt:
    list of (k, 3) arrays or None); NaN where the alternatives were too many to list."""
    err = np.full(len(got), np.nan)
    for j, cols in enumerate(alt):
        if cols is not None:
            err[j] = np.abs(cols - got[j]).max(axis=1).min()
    return err


def compare_images(gpu_imgs, orc_views, what=""):
    """gpu_imgs: list of (3,H,W) numpy.  Every pixel must match the oracle to IMG_TOL; a pixel with
    a decision that float32 may take either way must match one of its valid colours.  Returns
    (n_bad, n_unchecked (too many branches to list), max_err)."""
    bad = unchecked = 0
    worst = 0.0
    for gi, ov in zip(gpu_imgs, orc_views):
        got = gi.transpose(1, 2, 0).reshape(-1, 3)
        err = np.abs(got - ov.img.reshape(-1, 3)).max(axis=1)
        if ov.alt:
            ps = np.fromiter(ov.alt.keys(), np.int64)
            err[ps] = match_alternatives(got[ps], list(ov.alt.values()))
        skip = np.isnan(err)
        unchecked += int(skip.sum())
        worst = max(worst, float(err[~skip].max()) if (~skip).any() else 0.0)
        bad += int(((err > IMG_TOL) & ~skip).sum())
    return bad, unchecked, worst


# exp(-q/2) = 2^(KFALLOFF q): the records carry the conic scaled by it (the record layout of i4d.h)
KFALLOFF = -0.5 / np.log(2.0)


def gpu_records(rast):
    """The projected records of a Rasterizer as float64 columns (the 64-byte record layout of
    i4d.h: box | u, v, sa, sb2 | sc, o_t, m_thr, r | g, b, depth, radius), conic unscaled."""
    rec = rast.proj.view(-1, 4, 4).cpu().numpy().astype(np.float64)
    k = KFALLOFF
    return dict(box=rec[:, 0], u=rec[:, 1, 0], v=rec[:, 1, 1], ca=rec[:, 1, 2] / k, cb=rec[:, 1, 3] / (2 * k),
                cc=rec[:, 2, 0] / k, ot=rec[:, 2, 1], m_thr=rec[:, 2, 2], r=rec[:, 2, 3], g=rec[:, 3, 0],
                b=rec[:, 3, 1], depth=rec[:, 3, 2], radius=rec[:, 3, 3])


def tile_lists_oracle(orc, views_P, cams, tile=(16, 16)):
    """The oracle's tile lists of a batch of views with the GPU's tile numbering (views
    concatenated): (tiles, ids, status), status 1 = needed, 2 = near a threshold."""
    tiles, ids, sts, off = [], [], [], 0
    for P, cam in zip(views_P, cams):
        t, i, st = orc.tile_lists(P, cam, tile=tile, tile_offset=off, margin=FLAG_MARGIN)
        tiles.append(t.astype(np.int64))
        ids.append(i.astype(np.int64))
        sts.append(st)
        tx = (int(cam["W"]) + tile[0] - 1) // tile[0]
        ty = (int(cam["H"]) + tile[1] - 1) // tile[1]
        off += tx * ty
    return np.concatenate(tiles), np.concatenate(ids), np.concatenate(sts)


# Extra (tile, Gaussian) pairs the GPU may list beyond the oracle's: binning uses the box of the
# ellipse q <= min(q_max, 2 ln(o_t / alpha_min)) + 1e-3 widened by 1% + 0.01 px, in float32.  A pair
# is within slack when its tile holds a pixel centre of the box of the ellipse q <= q_lim + 2e-3,
# half-widths sqrt(q Sigma2) widened by 2% + 1e-6 cond + 0.05 px (cond = the 2D covariance's
# condition number: the float32 conic's relative error grows with it).
SLACK_Q, SLACK_REL, SLACK_COND, SLACK_PX = 2e-3, 0.02, 1e-6, 0.05


def _view_of_tiles(cams, tile):
    offs = [0]
    for cam in cams:
        offs.append(offs[-1] + ((int(cam["W"]) + tile[0] - 1) // tile[0]) * ((int(cam["H"]) + tile[1] - 1) // tile[1]))
    return np.asarray(offs, np.int64)


def check_tile_lists(orc, gpu_tiles, gpu_ids, views_P, cams, tile=(16, 16)):
    """Compare the GPU's sorted (tile, id) list with the oracle's definition of the binning, for a
    batch of views.  Asserts: (1) every needed oracle pair of a Gaussian whose culls are not within
    FLAG_MARGIN of their thresholds is listed; (2) every other listed pair is within the slack box
    above (and belongs to a Gaussian the oracle keeps, unless flagged); (3) no pair is listed twice;
    (4) inside each tile the order is by depth (up to DEPTH_MARGIN relative, where either order is
    valid).  Returns counts for the report."""
    C = orc.P
    gpu_tiles = np.asarray(gpu_tiles, np.int64)
    gpu_ids = np.asarray(gpu_ids, np.int64)
    wt, wi, ws = tile_lists_oracle(orc, views_P, cams, tile)
    offs = _view_of_tiles(cams, tile)
    n = views_P[0].shape[0]
    view_g = np.searchsorted(offs, gpu_tiles, side="right") - 1
    view_w = np.searchsorted(offs, wt, side="right") - 1
    allP = np.concatenate(views_P)
    # per (view, Gaussian) flags: a cull decision within FLAG_MARGIN
    flagged = allP[:, C["margin"]] < FLAG_MARGIN
    key_g = gpu_tiles * n + gpu_ids
    key_w = wt * n + wi
    assert len(np.unique(key_g)) == len(key_g), "a pair is listed twice"
    listed = np.isin(key_w, key_g)
    need = (ws == 1) & ~flagged[view_w * n + wi]
    missing = int((need & ~listed).sum())
    assert missing == 0, f"{missing} needed pairs missing"
    extra = ~np.isin(key_g, key_w)
    ev, ei = view_g[extra], gpu_ids[extra]
    et = gpu_tiles[extra] - offs[ev]
    recs = allP[ev * n + ei]
    fl = flagged[ev * n + ei]
    ok_vis = (recs[:, C["visible"]] != 0) | fl
    assert ok_vis.all(), f"{int((~ok_vis).sum())} pairs of culled Gaussians"
    worst = 0.0
    if len(recs):
        ca, cb, cc, ot = recs[:, C["ca"]], recs[:, C["cb"]], recs[:, C["cc"]], recs[:, C["ot"]]
        det = ca * cc - cb * cb
        tr = ca + cc
        disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0))
        cond = (tr / 2 + disc) / np.maximum(tr / 2 - disc, 1e-300)
        with np.errstate(divide="ignore", invalid="ignore"):
            qlim = np.minimum(9.0, np.maximum(2 * np.log(ot * 255.0), 0.0)) + SLACK_Q
        grow = 1.0 + SLACK_REL + SLACK_COND * cond
        hx = np.sqrt(qlim * cc / det) * grow + SLACK_PX
        hy = np.sqrt(qlim * ca / det) * grow + SLACK_PX
        Ws = np.array([int(c["W"]) for c in cams])[ev]
        Hs = np.array([int(c["H"]) for c in cams])[ev]
        tx = (Ws + tile[0] - 1) // tile[0]
        cx, cy = et % tx, et // tx
        xlo, xhi = cx * tile[0] + 0.5, np.minimum((cx + 1) * tile[0], Ws) - 0.5
        ylo, yhi = cy * tile[1] + 0.5, np.minimum((cy + 1) * tile[1], Hs) - 0.5
        dx = np.abs(np.clip(recs[:, C["u"]], xlo, xhi) - recs[:, C["u"]])
        dy = np.abs(np.clip(recs[:, C["v"]], ylo, yhi) - recs[:, C["v"]])
        ratio = np.maximum((dx - SLACK_PX) / (hx - SLACK_PX), (dy - SLACK_PX) / (hy - SLACK_PX))
        worst = float(ratio[~fl].max()) if (~fl).any() else 0.0
        inside = ((dx <= hx) & (dy <= hy)) | fl
        assert inside.all(), f"{int((~inside).sum())} extra pairs beyond the slack box (worst {worst})"
    # order inside each tile: non-decreasing oracle depth, near-equal depths in either order
    depth = allP[view_g * n + gpu_ids, C["depth"]]
    same = gpu_tiles[1:] == gpu_tiles[:-1]
    bad_order = same & (depth[:-1] > depth[1:] * (1 + DEPTH_MARGIN))
    assert not bad_order.any(), f"{int(bad_order.sum())} pairs out of depth order"
    return dict(gpu=len(key_g), needed=int((ws == 1).sum()), near=int((ws == 2).sum()), extra=int(extra.sum()),
                extra_worst_box_fraction=worst, flagged_records=int(flagged.sum()),
                flagged_needed_pairs=int(((ws == 1) & flagged[view_w * n + wi]).sum()))


def flagged_gaussians(orc, views_P):
    """Per view, ids whose culls, radius or depth order sit within FLAG_MARGIN of a flip."""
    C = orc.P
    out = []
    for P in views_P:
        s = set(np.nonzero((P[:, C["radius_margin"]] < FLAG_MARGIN) | (P[:, C["margin"]] < FLAG_MARGIN))[0].tolist())
        vis = np.nonzero(P[:, C["visible"]] != 0)[0]
        d = P[vis, C["depth"]]
        order = np.argsort(d, kind="stable")
        ds = d[order]
        close = np.nonzero(np.diff(ds) / ds[:-1] < DEPTH_MARGIN)[0] if len(ds) > 1 else []
        for k in close:
            s.add(int(vis[order[k]]))
            s.add(int(vis[order[k + 1]]))
        out.append(s)
    return out


def assert_prune_equal(got, want):
    """Kept set, counts and flags bit-exact; averaged attributes to float32 rounding (the GPU sums
    in 64-bit fixed point, the oracle in float64)."""
    assert np.array_equal(got["rep"].astype(np.int64), want["rep"].astype(np.int64))
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["flag"], want["flag"])
    assert np.allclose(got["xyz"], want["centroid"], rtol=1e-6, atol=1e-6)
    assert np.allclose(got["rgb"], want["rgb"], atol=1e-6)
    assert np.allclose(got["t"], want["t"], atol=1e-6)


def assert_init_equal(P, g, n, deg):
    """GPU parameter planes against an oracle Gaussian dict: copies exact, logarithms to float32
    rounding of the log (device logf is within 1 ulp), SH planes zero."""
    assert np.array_equal(P[0], np.c_[g["mean4"]].astype(np.float32))
    np.testing.assert_allclose(P[1], g["logscale4"], rtol=0, atol=2e-6)
    np.testing.assert_allclose(P[2], g["ql"], rtol=0, atol=0)
    np.testing.assert_allclose(P[3], g["qr"], rtol=0, atol=0)
    np.testing.assert_allclose(P[4, :, 0], g["opacity"], rtol=0, atol=1e-6)
    assert np.array_equal(P[4, :, 1:], np.asarray(g["rgb"], np.float32))
    assert not P[5:].any()
