"""Pins of the learned-initialisation oracle (CPU only): bfloat16 rounding and GELU against torch,
the MLP backward against torch autograd with straight-through rounding, the rotation-loss
gradient against central differences, and the neighbourhood features against scipy's k-d tree."""
import numpy as np
import pytest

from oracle import learned as OL

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    r = np.random.default_rng(0)
    x = np.concatenate([r.normal(size=5000) * 10.0 ** r.integers(-8, 8, 5000), [0.0, -0.0, 1.0, 3.0e38]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OL.bf16(x), want)


def test_gelu_matches_torch():
    z = np.linspace(-8, 8, 1001)
    want = torch.nn.functional.gelu(torch.from_numpy(z)).numpy()
    assert np.allclose(OL.gelu(z), want, atol=1e-14)
    h = 1e-6
    assert np.allclose(OL.gelu_grad(z), (OL.gelu(z + h) - OL.gelu(z - h)) / (2 * h), atol=1e-8)


def test_mlp_forward_backward_match_torch_autograd():
    r = np.random.default_rng(1)
    w = OL.init_weights(3).astype(np.float64) + r.normal(0, 0.05, OL.weight_count())
    w = w.astype(np.float32)
    x = r.normal(size=(40, 64)).astype(np.float32)
    y, cache = OL.forward(w, x)
    dy = r.normal(size=y.shape)
    g = OL.backward(w, cache, dy, operands="exact")

    def st(t):  # straight-through bfloat16 rounding
        return t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()

    wt = torch.from_numpy(w.astype(np.float64)).requires_grad_(True)
    off, layers = 0, []
    for o, i in OL.LAYER_SHAPES:
        W = wt[off:off + o * i].view(o, i)
        off += o * i
        b = wt[off:off + o]
        off += o
        layers.append((st(W), b))
    h = st(torch.from_numpy(x.astype(np.float64)))
    for k, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = st(torch.nn.functional.gelu(z)) if k < 2 else z
    assert np.allclose(h.detach().numpy(), y, rtol=1e-12, atol=1e-12)
    (h * torch.from_numpy(dy)).sum().backward()
    assert np.allclose(wt.grad.numpy(), g, rtol=1e-10, atol=1e-12)


class _RoundGrad(torch.autograd.Function):
    """Identity forward; the backward rounds the incoming gradient to bfloat16."""

    @staticmethod
    def forward(ctx, t):
        return t.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def _torch_mlp_grad(w, x, dy, round_grads):
    def st(t):  # straight-through bfloat16 rounding of the forward operands
        return t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()

    wt = torch.from_numpy(w.astype(np.float64)).requires_grad_(True)
    off, layers = 0, []
    for o, i in OL.LAYER_SHAPES:
        W = wt[off:off + o * i].view(o, i)
        off += o * i
        b = wt[off:off + o]
        off += o
        layers.append((st(W), b))
    h = st(torch.from_numpy(x.astype(np.float64)))
    for k, (W, b) in enumerate(layers):
        m = h @ W.T
        z = (_RoundGrad.apply(m) if round_grads else m) + b
        h = st(torch.nn.functional.gelu(z)) if k < 2 else z
    (h * torch.from_numpy(dy)).sum().backward()
    return wt.grad.numpy()


def test_mlp_bf16_operand_backward_matches_torch_autograd():
    """The training kernels' reading: the gradient entering each matrix product is rounded to
    bfloat16 (biases take the unrounded sums).  Autograd places that rounding between each product
    and its bias add; the oracle's backward must agree to float64 rounding, and differ from the
    exact gradient by about the bfloat16 precision."""
    r = np.random.default_rng(11)
    w = (OL.init_weights(5).astype(np.float64) + r.normal(0, 0.05, OL.weight_count())).astype(np.float32)
    x = r.normal(size=(50, 64)).astype(np.float32)
    y, cache = OL.forward(w, x)
    dy = r.normal(size=y.shape) * 1e-3
    g = OL.backward(w, cache, dy)
    want = _torch_mlp_grad(w, x, dy, round_grads=True)
    assert np.allclose(g, want, rtol=1e-10, atol=1e-15)
    exact = OL.backward(w, cache, dy, operands="exact")
    assert np.allclose(exact, _torch_mlp_grad(w, x, dy, round_grads=False), rtol=1e-10, atol=1e-15)
    d = np.linalg.norm(g - exact) / np.linalg.norm(exact)
    assert 1e-5 < d < 1e-2, d
    # the biases sum unrounded values: the output-layer bias gradient is the same in both
    nb3 = OL.LAYER_SHAPES[2][0]
    assert np.array_equal(g[-nb3:], exact[-nb3:])


def test_rotation_loss_gradient_matches_central_differences():
    r = np.random.default_rng(2)
    y = r.normal(size=(6, 12))
    tgt = np.zeros((6, 20))
    tgt[:, :4] = r.normal(size=(6, 4))
    for i in range(6):
        tgt[i, 4:] = OL.rotation(r.normal(size=4), r.normal(size=4)).ravel()
    _, dy = OL.loss_and_grad(y, tgt, 0.7, 1.3, 2.0)
    h = 1e-6
    for i in range(6):
        for j in range(12):
            yp, ym = y.copy(), y.copy()
            yp[i, j] += h
            ym[i, j] -= h
            fd = (OL.loss_and_grad(yp, tgt, 0.7, 1.3, 2.0)[0] - OL.loss_and_grad(ym, tgt, 0.7, 1.3, 2.0)[0]) / (2 * h)
            assert abs(fd - dy[i, j]) < 1e-7 * max(1.0, abs(fd))


def test_rotation_is_orthogonal_and_conjugate_pair_fixes_time():
    r = np.random.default_rng(4)
    q = r.normal(size=4)
    R = OL.rotation(q, r.normal(size=4))
    assert np.allclose(R @ R.T, np.eye(4), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)
    R = OL.rotation(q, q * np.array([1, -1, -1, -1]))
    assert np.allclose(R[3], [0, 0, 0, 1], atol=1e-14) and np.allclose(R[:, 3], [0, 0, 0, 1], atol=1e-14)


def test_knn_features_match_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    r = np.random.default_rng(5)
    n, voxel = 1500, 0.05
    xyz = r.uniform(0, 0.4, size=(n, 3)).astype(np.float32)
    rgb = r.uniform(size=(n, 3))
    t = r.uniform(size=n)
    flag = (r.uniform(size=n) < 0.2).astype(np.uint8)
    feats, knn3, idx = OL.knn_features(xyz, rgb, t, flag, voxel, (0.5, 0.5, -2.0), radius=2)
    tree = spatial.cKDTree(xyz.astype(np.float64))
    d, j = tree.query(xyz.astype(np.float64), k=17)
    # where the 16th neighbour lies well inside the +-2-voxel window, the window search is exact
    inside = d[:, 16] < 1.5 * voxel
    assert inside.sum() > 200
    for i in np.nonzero(inside)[0]:
        assert set(idx[i].tolist()) == set(j[i, 1:].tolist())
        assert knn3[i] == pytest.approx(d[i, 1:4].mean(), rel=1e-12)
    assert np.allclose(feats[:, 49:52], rgb) and np.allclose(feats[:, 52], t)
    assert np.allclose(feats[:, 48], np.linalg.norm(xyz.astype(np.float64) - [0.5, 0.5, -2.0], axis=1))


def test_knn3_scale_matches_brute_force_window_search():
    """The k-d tree 3-NN scale equals the brute-force window search, including sparse points with
    fewer than 3 neighbours in the window, neighbours cut off by the window and duplicate points."""
    pytest.importorskip("scipy.spatial")
    r = np.random.default_rng(8)
    voxel = 0.05
    dense = r.uniform(0, 0.3, size=(600, 3))
    sparse = r.uniform(1.0, 3.0, size=(60, 3))           # mostly isolated: fewer than 3 in the window
    dup = dense[:20] + 0.0                               # exact duplicates: zero distances
    xyz = np.concatenate([dense, sparse, dup]).astype(np.float32)
    n = xyz.shape[0]
    _, want, _ = OL.knn_features(xyz, np.zeros((n, 3)), np.zeros(n), np.zeros(n, np.uint8), voxel, (0, 0, 0), radius=2)
    got = OL.knn3_scale(xyz, voxel, radius=2, k0=4)      # small first query exercises the widening
    assert np.sum(want == voxel) >= 10                   # the fallback case is covered
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_bf16_margin_locates_rounding_boundaries():
    """bf16_margin is 0 exactly where bfloat16 rounding changes value (checked with torch's
    float32 -> bfloat16 cast on both sides of the boundary) and 0.5 on bfloat16 values."""
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(4)
    v = r.normal(size=2000).astype(np.float32)
    b = torch.from_numpy(v).to(torch.bfloat16).float().numpy()
    assert np.allclose(OL.bf16_margin(b), 0.5)
    # the midpoint above each bfloat16 value: half a bfloat16 spacing (16 low bits = 0x8000)
    mid = (b.view(np.uint32) | np.uint32(0x8000)).view(np.float32)
    assert np.all(OL.bf16_margin(mid) == 0.0)
    lo = np.nextafter(mid, np.float32(0)).astype(np.float32)
    hi = np.nextafter(mid, np.float32(np.inf) * np.sign(mid)).astype(np.float32)
    rl = torch.from_numpy(lo).to(torch.bfloat16).float().numpy()
    rh = torch.from_numpy(hi).to(torch.bfloat16).float().numpy()
    assert np.all(rl != rh)
