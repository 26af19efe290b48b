"""Shared helpers of the GPU parity tests (comparison protocol against the FP64 oracle)."""
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


def oracle_views(orc, g, cams, tile=(16, 16), settings=None, bg=(0, 0, 0)):
    """Oracle render of each view: list of (proj, img (H,W,3), T, nc, margin)."""
    out = []
    for cam in cams:
        P = orc.project(g, cam, tile=tile, settings=settings)
        img, T, nc, mg, dmg = orc.render(P, cam, bg=bg, settings=settings, depth_margin=True, impact_min=IMPACT_MIN)
        W, H = int(cam["W"]), int(cam["H"])
        # one flag value per pixel: below FLAG_MARGIN means "may differ"
        flag = np.minimum(mg, dmg * (FLAG_MARGIN / DEPTH_MARGIN))
        out.append((P, img.reshape(H, W, 3), T.reshape(H, W), nc.reshape(H, W), flag.reshape(H, W)))
    return out


def compare_images(gpu_imgs, orc_views, what=""):
    """gpu_imgs: list of (3,H,W) numpy.  Returns (n_bad_unflagged, n_flagged, max_err_unflagged)."""
    bad = flagged = 0
    worst = 0.0
    for gi, (P, img, T, nc, mg) in zip(gpu_imgs, orc_views):
        err = np.abs(gi.transpose(1, 2, 0) - img).max(axis=2)
        fl = mg < FLAG_MARGIN
        flagged += int(fl.sum())
        worst = max(worst, float(err[~fl].max()) if (~fl).any() else 0.0)
        bad += int(((err > IMG_TOL) & ~fl).sum())
    return bad, flagged, worst


def tile_pairs_oracle(orc, views_P, cams, tile=(16, 16)):
    tiles, ids, off = [], [], 0
    for P, cam in zip(views_P, cams):
        t, i = orc.tile_pairs(P, cam, tile=tile, tile_offset=off)
        tiles.append(t.astype(np.int64))
        ids.append(i.astype(np.int64))
        tx = (int(cam["W"]) + tile[0] - 1) // tile[0]
        ty = (int(cam["H"]) + tile[1] - 1) // tile[1]
        off += tx * ty
    return np.concatenate(tiles), np.concatenate(ids)


def suspicious_gaussians(orc, views_P):
    """Per view, ids whose rectangle, visibility or depth order sits within FLAG_MARGIN of a flip."""
    C = orc.P
    out = []
    for P in views_P:
        s = set(np.nonzero((P[:, C["rect_margin"]] < FLAG_MARGIN) | (P[:, C["margin"]] < FLAG_MARGIN))[0].tolist())
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
