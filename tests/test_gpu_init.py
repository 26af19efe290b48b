"""GPU <-> oracle parity of the initialisation kernels (Sec. 4.1; Sec. 3.3 "Motion-Aware Gaussian")
and of the motion targets (velocity b / c of Eq. 7, the 4D rotation), element by element, through
the C ABI."""
import numpy as np
import pytest

from gpu_util import assert_init_equal
from oracle import learned as OL

pytestmark = pytest.mark.gpu

ST_DYN, ST_STATIC = 2.0 / 199, 1.0


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _pruned(n, seed):
    r = np.random.default_rng(seed)
    return dict(rep=np.arange(n, dtype=np.uint32), count=np.ones(n, np.int32),
                centroid=r.normal(size=(n, 3)).astype(np.float32), t=r.uniform(size=n).astype(np.float32),
                rgb=r.uniform(size=(n, 3)).astype(np.float32), flag=(r.uniform(size=n) < 0.3).astype(np.uint8))


def _planes(params, n, deg):
    from paper_2510_01119_gb300 import rasterizer as R
    return params.cpu().numpy().reshape(R.n_planes(deg), n, 4)


@pytest.mark.parametrize("deg", [0, 3])
def test_init_heuristic_matches_oracle(dev, orc, deg):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    from paper_2510_01119_gb300 import rasterizer as R
    n = 100003
    pr = _pruned(n, 70 + deg)
    params = torch.full((R.n_planes(deg) * n * 4,), float("nan"), device=dev)
    L.i4d_init_heuristic(_t(pr["centroid"], dev), _t(pr["rgb"], dev), _t(pr["t"], dev), _t(pr["flag"], dev), n, deg,
                         0.012, ST_DYN, ST_STATIC, 0.1, params)
    g = orc.init_heuristic(pr, 0.012, ST_DYN, ST_STATIC, 0.1)
    assert_init_equal(_planes(params, n, deg), g, n, deg)


@pytest.mark.parametrize("with_mlp", [False, True])
def test_init_learned_matches_oracle(dev, with_mlp):
    """Per-point spatial scale, proposals from an MLP output with ~6% degenerate rows (non-finite,
    zero quaternion, log s_t out of range) that fall back to the heuristic, and the NULL-proposal
    call the bench initialises with."""
    import torch
    from paper_2510_01119_gb300 import _lib as L
    n = 120007
    pr = _pruned(n, 80)
    r = np.random.default_rng(81)
    spatial = np.exp(r.normal(-4.5, 0.4, n)).astype(np.float32)
    y = None
    if with_mlp:
        y = r.normal(size=(n, 12)).astype(np.float32)
        y[:, 0] = r.normal(-3, 1, n)
        bad = r.choice(n, 7500, replace=False)
        y[bad[:2500], r.integers(0, 12, 2500)] = np.nan
        y[bad[2500:5000], 4:8] = 0.0
        y[bad[5000:], 0] = 7.0
    params = torch.full((5 * n * 4,), float("nan"), device=dev)
    fb = torch.full((1,), -1, dtype=torch.int32, device=dev)
    L.i4d_init_learned(_t(pr["centroid"], dev), _t(pr["rgb"], dev), _t(pr["t"], dev), _t(pr["flag"], dev),
                       _t(spatial, dev), None if y is None else _t(y, dev), n, 0, ST_DYN, ST_STATIC, 0.1, params, fb)
    g, nfb = OL.init_learned(pr, spatial, y, ST_DYN, ST_STATIC, 0.1)
    assert int(fb.item()) == nfb
    if with_mlp:
        assert nfb == 7500
    P = _planes(params, n, 0)
    np.testing.assert_allclose(P[1, :, :3], g["logscale4"][:, :3], rtol=0, atol=2e-6)
    assert_init_equal(P, g, n, 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_motion_targets_match_oracle(dev, mode):
    """log s_t, velocity b / c and R of every Gaussian.  The velocity is a ratio of float32 dot
    products: its error is a few ulp of sqrt(Sigma_aa / c) + |v_a| (Cauchy-Schwarz on b_a), so each
    component is held to 2e-5 of that scale; R entries to 2e-6."""
    import torch
    from paper_2510_01119_gb300 import _lib as L
    n = 200003
    r = np.random.default_rng(90 + mode)
    g = dict(mean4=r.normal(size=(n, 4)), logscale4=np.c_[r.normal(-3, 0.5, (n, 3)), r.normal(-1.5, 0.3, n)],
             ql=r.normal(size=(n, 4)), qr=r.normal(size=(n, 4)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
             sh=np.zeros((n, 0, 3)), sh_deg=0, mode=mode)
    g = {k: (v.astype(np.float32) if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    from paper_2510_01119_gb300 import rasterizer as R
    params = R.pack_params(g, dev)
    out = torch.empty(n, 20, device=dev)
    gs = L.Gaussians()
    gs.params, gs.n, gs.sh_deg, gs.mode, gs.sch_terms = params.data_ptr(), n, 0, mode, 0
    L.i4d_motion_targets(gs, out)
    got = out.cpu().numpy()
    want = OL.motion_targets(g)
    assert np.array_equal(got[:, 0], g["logscale4"][:, 3])
    s = np.exp(np.asarray(g["logscale4"], np.float64))
    if mode:
        s[:, 1] = s[:, 2] = s[:, 0]
    Rm = want[:, 4:20].reshape(n, 4, 4)
    Sig = np.einsum("nik,nk,njk->nij", Rm, s * s, Rm)
    scale = np.sqrt(np.stack([Sig[:, a, a] for a in range(3)], 1) / Sig[:, 3, 3][:, None]) + np.abs(want[:, 1:4])
    err = np.abs(got[:, 1:4] - want[:, 1:4])
    assert np.all(err <= 2e-5 * scale), float((err / scale).max())
    np.testing.assert_allclose(got[:, 4:20], want[:, 4:20], rtol=0, atol=2e-6)
