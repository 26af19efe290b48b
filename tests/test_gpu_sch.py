"""GPU <-> FP64 oracle parity of the SCH appearance variant (the 4DGS colour model of Sec. 3.1:
SH times temporal Fourier terms): records, rendered images and every gradient, including the SCH
coefficients', over views at different frame times."""
import numpy as np
import pytest

import synth
from gpu_util import FLAG_MARGIN, GRAD_TOL, compare_images, gpu_records, oracle_views, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _scene(seed, deg, nt, n=1500):
    g = synth.gaussians_uniform(seed, n=n, sh_deg=deg)
    g["sch_terms"] = nt
    g["sch"] = np.random.default_rng(seed + 100).normal(0, 0.08, (n, nt - 1, (deg + 1) ** 2, 3))
    return g


@pytest.mark.parametrize("deg,nt", [(0, 2), (0, 4), (2, 3), (3, 2)])
def test_sch_forward_and_backward_match_oracle(dev, orc, deg, nt):
    import torch
    from paper_2510_01119_gb300 import rasterizer as R
    g = _scene(7 + deg, deg, nt)
    cams = [synth.camera(96, 80, 60.0, time=0.21), synth.camera(64, 48, 55.0, time=0.77)]
    rast = R.Rasterizer(g["mean4"].shape[0], deg, 0, [(c["W"], c["H"]) for c in cams], sch_terms=nt)
    params = R.pack_params(g, dev)
    camt = R.cameras_tensor(cams, dev)
    rast.forward(params, camt)
    ov = oracle_views(orc, g, cams)
    bad, flagged, worst = compare_images([x.cpu().numpy() for x in rast.split_images()], ov)
    assert bad == 0, (bad, flagged, worst)
    # records: the colour columns carry the SCH terms (records on no tile are not written)
    n = g["mean4"].shape[0]
    rec = gpu_records(rast)
    touched = rast.touched[:len(cams) * n].cpu().numpy()
    C = orc.P
    for v, cam in enumerate(cams):
        P = ov[v][0]
        vis = (P[:, C["visible"]] != 0) & (touched[v * n:(v + 1) * n] > 0)
        assert vis.sum() > 100
        got = np.c_[rec["r"], rec["g"], rec["b"]][v * n:(v + 1) * n]
        want = P[:, [C["r"], C["g"], C["b"]]]
        assert np.abs(got[vis] - want[vis]).max() < 2e-6
    # backward, summed over both views
    rng = np.random.default_rng(deg * 10 + nt)
    ups, want = [], None
    for v, cam in enumerate(cams):
        gi = rng.normal(size=ov[v][1].shape) * 1e-3
        gi[ov[v][4] < FLAG_MARGIN] = 0.0
        ups.append(gi.transpose(2, 0, 1).reshape(-1))
        _, gr = orc.render_bwd(g, cam, gi.reshape(-1, 3))
        want = gr if want is None else {k: want[k] + gr[k] for k in want}
    rast.backward(params, camt, torch.from_numpy(np.concatenate(ups).astype(np.float32)).to(dev))
    got = R.unpack_params(rast.grads, n, deg, nt)
    keys = ["mean4", "logscale4", "ql", "qr", "opacity", "rgb", "sch"] + (["sh"] if deg > 0 else [])
    errs = {}
    for k in keys:
        w = want[k][:, :(deg + 1) ** 2 - 1] if k == "sh" else want[k]
        errs[k] = rel_l2(got[k], w)
    assert all(e < GRAD_TOL for e in errs.values()), errs


def test_sch_with_one_term_is_the_plain_colour(dev, orc):
    """sch_terms = 1 leaves the parameter layout and every output of the plain colour model unchanged."""
    from paper_2510_01119_gb300 import rasterizer as R
    g = synth.gaussians_uniform(3, n=800, sh_deg=1)
    cams = [synth.camera(64, 48, 60.0, time=0.6)]
    a = R.Rasterizer(800, 1, 0, [(64, 48)])
    b = R.Rasterizer(800, 1, 0, [(64, 48)], sch_terms=1)
    p = R.pack_params(g, dev)
    c = R.cameras_tensor(cams, dev)
    assert np.array_equal(a.forward(p, c).cpu().numpy(), b.forward(p, c).cpu().numpy())
