"""Parity of the whole training step (Sec. 3.3 optimisation with the Sec. 4.1 loss and optimiser):
the CUDA-graph replay against the same calls launched eagerly, and one step against the oracle
chain render -> (1 - 0.2) L1 + 0.2 D-SSIM -> backward -> Adam."""
import numpy as np
import pytest

import synth
from gpu_util import FLAG_MARGIN, GRAD_TOL, oracle_views, rel_l2

pytestmark = pytest.mark.gpu

SIZES = [(128, 96), (96, 72), (80, 64)]
TIMES = [0.5, 0.31, 0.77]


@pytest.fixture(scope="module")
def dev():
    import torch
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    _lib.load()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _cams():
    return [synth.camera(W, H, 60.0, time=t) for (W, H), t in zip(SIZES, TIMES)]


def _targets():
    return [synth.random_image(40 + k, W, H) for k, (W, H) in enumerate(SIZES)]


def _step(params, n, dev, cams, tgts):
    import torch
    from paper_2510_01119_gb300 import train as T
    from paper_2510_01119_gb300 import rasterizer as R
    st = T.TrainStep(params, n, 0, 0, SIZES, steps=100, dssim=T.DSSIM_LAMBDA)
    st.cams.copy_(R.cameras_tensor(cams, dev))
    st.target.copy_(torch.from_numpy(np.concatenate([t.transpose(2, 0, 1).reshape(-1) for t in tgts])).to(dev))
    return st


def test_captured_step_replays_the_eager_step(dev):
    """Three replays of the captured step against three eager steps on a copy of the parameters:
    the first loss is bit-identical (the forward has no atomics); afterwards the two runs differ only
    by the order of the backward's float atomics, so losses agree to 1e-6 and the parameter updates
    to 1e-5 relative L2; the Adam step counter reads 3 on both."""
    import torch
    from paper_2510_01119_gb300 import rasterizer as R
    g = synth.gaussians_uniform(0)
    n = g["mean4"].shape[0]
    cams, tgts = _cams(), _targets()
    p0 = R.pack_params(g, dev)
    pe, pg = p0.clone(), p0.clone()
    se, sg = _step(pe, n, dev, cams, tgts), _step(pg, n, dev, cams, tgts)
    sg.capture(warmup=0)
    torch.cuda.synchronize()
    assert torch.equal(pg, p0)                     # capturing enqueues nothing
    for k in range(3):
        se.run()
        sg.replay()
        torch.cuda.synchronize()
        le, lg = float(se.loss.item()), float(sg.loss.item())
        if k == 0:
            assert le == lg
        assert lg == pytest.approx(le, rel=1e-6)
    assert int(se.step_count.item()) == 3 and int(sg.step_count.item()) == 3
    assert rel_l2((pg - p0).cpu().numpy(), (pe - p0).cpu().numpy()) < 1e-5
    assert rel_l2(sg.m.cpu().numpy(), se.m.cpu().numpy()) < 1e-5
    assert rel_l2(sg.v.cpu().numpy(), se.v.cpu().numpy()) < 1e-5


def test_one_step_matches_the_oracle_chain(dev, orc):
    """One training step of the 2,000-Gaussian scene over three views of different sizes and times:
    the loss, the gradient of every parameter group and Adam's moments against the oracle's chain
    render -> (1 - 0.2) L1 + 0.2 D-SSIM -> analytic backward -> Adam.  At the first step Adam moves
    each parameter by -lr sign(g); the move is checked where the oracle's gradient is clear of zero
    (|g| > 1e-2 of its group's RMS), where a float32 gradient cannot take the other sign."""
    import torch
    from oracle import ssim as OS
    from paper_2510_01119_gb300 import rasterizer as R
    from paper_2510_01119_gb300 import train as T
    g = synth.gaussians_uniform(0)
    n = g["mean4"].shape[0]
    cams, tgts = _cams(), _targets()
    p0 = R.pack_params(g, dev)
    st = _step(p0.clone(), n, dev, cams, tgts)
    st.run()
    torch.cuda.synchronize()
    # the oracle chain
    ov = oracle_views(orc, g, cams)
    imgs = [v.img.transpose(2, 0, 1) for v in ov]
    loss, dL = OS.photometric_loss(imgs, [t.transpose(2, 0, 1).astype(np.float64) for t in tgts], T.DSSIM_LAMBDA)
    want = None
    for cam, d in zip(cams, dL):
        _, gr = orc.render_bwd(g, cam, d.transpose(1, 2, 0).reshape(-1, 3))
        want = gr if want is None else {k: want[k] + gr[k] for k in want}
    flagged = sum(int((v.flag < FLAG_MARGIN).sum()) for v in ov)
    print(f"pixels with a near-threshold decision: {flagged} of {sum(W * H for W, H in SIZES)}")
    assert float(st.loss.item()) == pytest.approx(loss, rel=1e-5)
    got = R.unpack_params(st.rast.grads, n, 0)
    errs = {k: rel_l2(got[k], want[k]) for k in ("mean4", "logscale4", "ql", "qr", "opacity", "rgb")}
    print("gradient rel L2 per group:", errs)
    assert all(e < GRAD_TOL for e in errs.values()), errs
    # Adam: the oracle's moments and the sign step, group by group
    gflat = R.pack_params(dict(g, **{k: want[k] for k in ("mean4", "logscale4", "ql", "qr", "opacity", "rgb")}),
                          "cpu").numpy().astype(np.float64)
    lr = np.zeros(gflat.size)
    for grp in st.groups:
        for k in range(4):
            lr[grp.begin + k:grp.end:4] = grp.lr_init[k]
    # the first update uses step 1 of the schedule (decaying groups move from lr_init by one step)
    for grp in st.groups:
        if grp.decay_steps > 0:
            for k in range(4):
                lr[grp.begin + k:grp.end:4] = T.log_lr(grp.lr_init[k], grp.lr_final[k], 1.0 / grp.decay_steps)
    p_o, m_o, v_o = orc.adam_step(p0.cpu().numpy(), gflat, np.zeros_like(gflat), np.zeros_like(gflat), lr, 1,
                                  beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                                  eps=float(np.float32(1e-15)))
    assert rel_l2(st.m.cpu().numpy(), m_o) < GRAD_TOL
    assert rel_l2(st.v.cpu().numpy(), v_o) < 2 * GRAD_TOL
    dp = st.params.cpu().numpy().astype(np.float64) - p0.cpu().numpy()
    for grp in st.groups:
        sl = slice(grp.begin, grp.end)
        gg = gflat[sl]
        clear = np.abs(gg) > 1e-2 * np.sqrt(np.mean(gg * gg))
        np.testing.assert_allclose(dp[sl][clear], (p_o - p0.cpu().numpy())[sl][clear], rtol=1e-3,
                                   atol=1e-6 * np.abs(p0.cpu().numpy()[sl][clear]).max())
