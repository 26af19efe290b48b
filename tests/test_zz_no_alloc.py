"""i4d_render_bwd_noalloc against i4d_render_bwd through the C ABI.

The no-allocation entry point serves callers that may not allocate device memory when they run
the backward; it keeps its 2D-gradient scratch in a fixed array inside the library.  This file is
collected last so that a failure here does not stop the other GPU tests; it passes alone in a fresh
process as well as after them."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import GRAD_TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def test_noalloc_backward_matches_existing_entry_point(dev):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    from paper_2510_01119_gb300 import rasterizer as R
    g = synth.gaussians_uniform(0, sh_deg=1)
    cams = [synth.camera(128, 96, 60.0, time=0.5), synth.camera(77, 45, 50.0, time=0.2)]
    rast = R.Rasterizer(2000, 1, 0, [(c["W"], c["H"]) for c in cams])
    params = R.pack_params(g)
    camt = R.cameras_tensor(cams)
    rast.forward(params, camt)
    rng = np.random.default_rng(5)
    for call in range(2):                      # two calls in a row reuse the shared scratch
        dl = torch.from_numpy(rng.normal(size=rast.img.numel()).astype(np.float32) * 1e-3).to(dev)
        want = rast.backward(params, camt, dl).clone()
        got = torch.full_like(want, float("nan"))
        L.i4d_render_bwd_noalloc(rast.gaussians(params), rast.views, camt, rast.settings, rast.proj, rast.touched,
                                 rast.ids, rast.ranges, rast.T_final, rast.last, dl, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert rel_l2(a, b) < GRAD_TOL, (call, rel_l2(a, b))


def test_noalloc_rejects_sizes_beyond_its_scratch(dev):
    import torch
    from paper_2510_01119_gb300 import _lib as L
    from paper_2510_01119_gb300 import rasterizer as R
    lib = L.load()
    cap = int(lib.i4d_render_bwd_noalloc_max_records())
    assert cap == 1 << 19
    rast = R.Rasterizer(100, 0, 0, [(32, 32)] * 2)
    params = torch.zeros(5 * 100 * 4, device=dev)
    g = rast.gaussians(params)
    g.n = cap // 2 + 1                         # 2 views x n records > cap: rejected before any launch
    with pytest.raises(L.I4DError, match="exceeds the fixed scratch"):
        L.i4d_render_bwd_noalloc(g, rast.views, torch.zeros(2, 20, device=dev), rast.settings, rast.proj,
                                 rast.touched, rast.ids, rast.ranges, rast.T_final, rast.last, rast.img, rast.grads)


def test_noalloc_at_full_capacity_on_a_side_stream(dev):
    """2 views x 262,144 Gaussians fill the fixed scratch exactly; the call runs on a stream other
    than the default one and matches i4d_render_bwd."""
    import torch
    from paper_2510_01119_gb300 import _lib as L
    from paper_2510_01119_gb300 import rasterizer as R
    lib = L.load()
    n = int(lib.i4d_render_bwd_noalloc_max_records()) // 2
    g = synth.gaussians_uniform(3, n=n)
    cams = [synth.camera(160, 120, 60.0, time=0.5), synth.camera(96, 64, 50.0, time=0.3)]
    rast = R.Rasterizer(n, 0, 0, [(c["W"], c["H"]) for c in cams])
    params = R.pack_params(g)
    camt = R.cameras_tensor(cams)
    rast.forward(params, camt)
    dl = torch.from_numpy(np.random.default_rng(6).normal(size=rast.img.numel()).astype(np.float32) * 1e-3).to(dev)
    want = rast.backward(params, camt, dl).clone()
    got = torch.full_like(want, float("nan"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    L.i4d_render_bwd_noalloc(rast.gaussians(params), rast.views, camt, rast.settings, rast.proj, rast.touched,
                             rast.ids, rast.ranges, rast.T_final, rast.last, dl, got, stream=side)
    side.synchronize()
    a, b = got.cpu().numpy(), want.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert rel_l2(a, b) < GRAD_TOL
