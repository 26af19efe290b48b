"""Oracle of the learned initialisation (test infrastructure only): neighbourhood features,
the 3-layer GELU MLP with BF16-rounded operands, its loss and its analytic backward, in float64.

The paper initialises temporal scale, rotation and motion by a heuristic (Sec. 4.1, Sec. 3.3
"Motion-Aware Gaussian"); the learned initialisation is an addition that proposes those values
from each pruned point's voxel neighbourhood.  Definitions:

features (64 per point): the 16 nearest other points among those whose voxel cell lies within
+-radius cells of the point's cell on every axis, ordered by (squared distance, index); their
offsets (neighbour - point) / voxel (48 values, zeros for missing slots); the distance to a
reference centre (the mean camera centre of the video); the colour (3); the time; the number of
neighbours found / 16; the dynamic flag; the least-squares velocity of the neighbourhood,
sum_k dt_k o_k / (sum_k dt_k^2 + 1e-6) with o_k the offsets in voxels and dt_k the neighbours' time
minus the point's, divided by 16 (3); the RMS of dt_k (1); zeros to 64.  The 3-NN scale is the mean distance to the
3 nearest neighbours (the voxel edge when fewer than 3 exist).

MLP: h1 = gelu(W1 bf(x) + b1), h2 = gelu(W2 bf(h1) + b2), y = W3 bf(h2) + b3 with bf() rounding to
bfloat16 (round to nearest even) and W* rounded to bfloat16; gelu(z) = z Phi(z) with the exact
normal CDF.  y = (log s_t, v_x, v_y, v_z, q_l (4), q_r (4)).

loss (mean over points): w_st (y0 - log s_t*)^2 + w_v |v - v*|^2 + w_R ||R(q_l, q_r) - R*||_F^2 with
R(q_l, q_r) the 4D rotation v -> q_l v q_r of the normalised quaternions (sign-free target).

Backward: bfloat16 operands with float32 accumulation, like the forward: the gradient entering
each layer's matrix product is rounded to bfloat16 before the two products that use it (see
backward()); the exact straight-through gradient is kept beside it for the pins.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYER_SHAPES = [(64, 64), (64, 64), (12, 64)]


def weight_count() -> int:
    return sum(o * i + o for o, i in LAYER_SHAPES)


def unpack_weights(w: np.ndarray):
    out, off = [], 0
    for o, i in LAYER_SHAPES:
        W = w[off:off + o * i].reshape(o, i)
        off += o * i
        b = w[off:off + o]
        off += o
        out.append((W, b))
    return out


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((u >> 16) & 1)
    r = ((u + rounding) >> 16) << 16
    r = np.where(np.isnan(a), u, r)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def knn_features(xyz, rgb, t, flag, voxel: float, ref_center, radius: int = 2, k: int = 16):
    """Brute-force neighbourhood features of every point (O(n^2); small n only)."""
    xyz = np.asarray(xyz, np.float64)
    n = xyz.shape[0]
    cell = np.floor(np.asarray(xyz, np.float32) * np.float32(1.0 / np.float32(voxel))).astype(np.int64)
    feats = np.zeros((n, 64))
    knn3 = np.zeros(n)
    nbr_idx = np.full((n, k), -1, np.int64)
    for i in range(n):
        near = np.all(np.abs(cell - cell[i]) <= radius, axis=1)
        near[i] = False
        js = np.nonzero(near)[0]
        d2 = np.sum((xyz[js] - xyz[i]) ** 2, axis=1)
        order = np.lexsort((js, d2))
        js, d2 = js[order][:k], d2[order][:k]
        nbr_idx[i, :len(js)] = js
        feats[i, :3 * len(js)] = ((xyz[js] - xyz[i]) / voxel).reshape(-1)
        feats[i, 48] = np.linalg.norm(xyz[i] - np.asarray(ref_center, np.float64))
        feats[i, 49:52] = rgb[i]
        feats[i, 52] = t[i]
        feats[i, 53] = len(js) / k
        feats[i, 54] = float(flag[i])
        if len(js):
            dt = np.asarray(t, np.float64)[js] - float(t[i])
            o = (xyz[js] - xyz[i]) / voxel
            feats[i, 55:58] = (dt[:, None] * o).sum(0) / (np.sum(dt * dt) + 1e-6) / 16.0
            feats[i, 58] = math.sqrt(np.mean(dt * dt))
        knn3[i] = np.sqrt(d2[:3]).mean() if len(js) >= 3 else voxel
    return feats, knn3, nbr_idx


def knn3_scale(xyz, voxel: float, radius: int = 2, k0: int = 16) -> np.ndarray:
    """The 3-NN spatial scale of every point (same definition as knn_features' second output) for
    large point sets: candidates in distance order from a k-d tree, filtered to the +-radius cell
    window, the first 3 survivors averaged; the query widens for points whose candidates ran out."""
    from scipy.spatial import cKDTree
    x64 = np.asarray(xyz, np.float64)
    n = x64.shape[0]
    cell = np.floor(np.asarray(xyz, np.float32) * np.float32(1.0 / np.float32(voxel))).astype(np.int64)
    tree = cKDTree(x64)
    out = np.full(n, float(voxel))
    todo = np.arange(n)
    k = k0
    while len(todo):
        kk = min(k, n)
        d, j = tree.query(x64[todo], k=kk, workers=-1)
        d, j = d.reshape(len(todo), kk), j.reshape(len(todo), kk)
        ok = (j != todo[:, None]) & np.all(np.abs(cell[j] - cell[todo][:, None, :]) <= radius, axis=2)
        # ties in distance are ordered by index, as in the brute-force definition
        order = np.lexsort((j, d), axis=1)
        d, ok = np.take_along_axis(d, order, 1), np.take_along_axis(ok, order, 1)
        cnt = np.cumsum(ok, axis=1)
        three = cnt[:, -1] >= 3
        first3 = ok & (cnt <= 3)
        s = np.where(first3, d, 0.0).sum(axis=1)
        out[todo[three]] = s[three] / 3.0
        done = three | (kk >= n)
        todo = todo[~done]
        k *= 4
    return out


def forward(w: np.ndarray, x: np.ndarray):
    """Returns (y, cache) for the backward."""
    (W1, b1), (W2, b2), (W3, b3) = unpack_weights(np.asarray(w, np.float64))
    W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
    x0 = bf16(x)
    z1 = x0 @ W1.T + b1
    h1 = bf16(gelu(z1))
    z2 = h1 @ W2.T + b2
    h2 = bf16(gelu(z2))
    y = h2 @ W3.T + b3
    return y, (x0, z1, h1, z2, h2, W1, W2, W3)


def bf16_margin(x: np.ndarray) -> np.ndarray:
    """Distance of float32 values from the nearest bfloat16 rounding boundary (the midpoint between
    two neighbouring bfloat16 values), as a fraction of the bfloat16 spacing there (0 = on the
    boundary, 0.5 = on a bfloat16 value)."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    low = (a.view(np.uint32) & 0xFFFF).astype(np.float64)
    return np.abs(low - 32768.0) / 65536.0


def forward_margins(w: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Per point, the smallest bf16_margin of the two hidden activations before their bfloat16
    rounding: a float32 evaluation that lands within its rounding error of a boundary may round the
    other way there (the inputs are float32 values, identical on every side)."""
    _, (x0, z1, h1, z2, h2, W1, W2, W3) = forward(w, x)
    g1 = gelu(z1)
    g2 = gelu(z2)
    return np.minimum(bf16_margin(g1).min(axis=1), bf16_margin(g2).min(axis=1))


def _left(p):
    a, b, c, d = p
    return np.array([[a, -d, c, b], [d, a, -b, c], [-c, b, a, d], [-b, -c, -d, a]])


def _right(q):
    e, f, g, h = q
    return np.array([[e, h, -g, f], [-h, e, f, g], [g, -f, e, h], [-f, -g, -h, e]])


def rotation(ql, qr):
    """4D rotation matrix of v -> q_l v q_r (vector (x,y,z,t) <-> quaternion t + xi + yj + zk)."""
    ql = np.asarray(ql, np.float64) / np.linalg.norm(ql)
    qr = np.asarray(qr, np.float64) / np.linalg.norm(qr)
    return _left(ql) @ _right(qr)


def _rotation_grad(ql, qr, G):
    """Gradient of <G, R(q_l, q_r)> with respect to the unnormalised quaternions: R = L(ql_hat)
    Rr(qr_hat) is linear in each quaternion, dR/dql_hat_j = L(e_j) Rr, dR/dqr_hat_j = L Rr(e_j), then
    through q_hat = q / |q|."""
    nl, nr = np.linalg.norm(ql), np.linalg.norm(qr)
    qlh, qrh = np.asarray(ql, np.float64) / nl, np.asarray(qr, np.float64) / nr
    Lm, Rm = _left(qlh), _right(qrh)
    E = np.eye(4)
    gl = np.array([np.sum(G * (_left(E[j]) @ Rm)) for j in range(4)])
    gr = np.array([np.sum(G * (Lm @ _right(E[j]))) for j in range(4)])
    gl = (gl - qlh * (qlh @ gl)) / nl
    gr = (gr - qrh * (qrh @ gr)) / nr
    return gl, gr


def loss_and_grad(y: np.ndarray, target: np.ndarray, w_st=1.0, w_v=1.0, w_R=1.0):
    """target: (n, 20) = (log s_t, v (3), R (16, row-major)).  Returns (loss, dL/dy)."""
    n = y.shape[0]
    dy = np.zeros_like(y, dtype=np.float64)
    loss = 0.0
    for i in range(n):
        e0 = y[i, 0] - target[i, 0]
        ev = y[i, 1:4] - target[i, 1:4]
        eR = rotation(y[i, 4:8], y[i, 8:12]) - target[i, 4:20].reshape(4, 4)
        loss += w_st * e0 * e0 + w_v * ev @ ev + w_R * np.sum(eR * eR)
        dy[i, 0] = 2 * w_st * e0
        dy[i, 1:4] = 2 * w_v * ev
        gl, gr = _rotation_grad(y[i, 4:8], y[i, 8:12], 2 * w_R * eR)
        dy[i, 4:8] = gl
        dy[i, 8:12] = gr
    return loss / n, dy / n


def backward(w: np.ndarray, cache, dy: np.ndarray, operands: str = "bf16") -> np.ndarray:
    """Gradient of sum(dy * y) with respect to the float32 master weights (straight through the
    bfloat16 rounding of the weights and activations), in the packed weight layout.

    operands="bf16" (the training kernels' arithmetic: bfloat16 operands, float32 accumulation):
    the gradient flowing into each layer's matrix product, dL/d(W h) (dy for the output layer,
    dz2 and dz1 for the hidden ones), is rounded to bfloat16 before it multiplies the bfloat16
    activations (weight gradients) and the bfloat16 weights (gradient of the layer below); the
    bias gradients sum the unrounded values.  operands="exact": no rounding in the backward, the
    exact gradient of the forward with straight-through rounding."""
    if operands not in ("bf16", "exact"):
        raise ValueError(operands)
    r = bf16 if operands == "bf16" else (lambda a: np.asarray(a, np.float64))
    x0, z1, h1, z2, h2, W1, W2, W3 = cache
    dyr = r(dy)
    dW3 = dyr.T @ h2
    db3 = dy.sum(0)
    dh2 = dyr @ W3
    dz2 = dh2 * gelu_grad(z2)
    dz2r = r(dz2)
    dW2 = dz2r.T @ h1
    db2 = dz2.sum(0)
    dh1 = dz2r @ W2
    dz1 = dh1 * gelu_grad(z1)
    dW1 = r(dz1).T @ x0
    db1 = dz1.sum(0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def init_weights(seed: int) -> np.ndarray:
    r = np.random.default_rng(seed)
    parts = []
    for o, i in LAYER_SHAPES:
        parts.append(r.normal(0.0, 1.0 / math.sqrt(i), size=o * i))
        parts.append(np.zeros(o))
    w = np.concatenate(parts).astype(np.float32)
    # start the quaternion heads at the identity rotation (a + 0i + 0j + 0k)
    off = 64 * 64 + 64 + 64 * 64 + 64 + 12 * 64
    w[off + 4] = 1.0
    w[off + 8] = 1.0
    return w


def rotation_batch(ql, qr) -> np.ndarray:
    """rotation() of many quaternion pairs at once -> (n, 4, 4): L(q_l / |q_l|) Rr(q_r / |q_r|)."""
    ql = np.asarray(ql, np.float64)
    qr = np.asarray(qr, np.float64)
    a, b, c, d = (ql / np.linalg.norm(ql, axis=1, keepdims=True)).T
    e, f, g, h = (qr / np.linalg.norm(qr, axis=1, keepdims=True)).T
    L = np.stack([np.stack([a, -d, c, b], -1), np.stack([d, a, -b, c], -1),
                  np.stack([-c, b, a, d], -1), np.stack([-b, -c, -d, a], -1)], 1)
    M = np.stack([np.stack([e, h, -g, f], -1), np.stack([-h, e, f, g], -1),
                  np.stack([g, -f, e, h], -1), np.stack([-f, -g, -h, e], -1)], 1)
    return L @ M


def motion_targets(g: dict) -> np.ndarray:
    """Per Gaussian (n, 20): (log s_t, velocity v = b / c, R row-major), the values the learned
    initialisation is trained to propose.  Sigma = R diag(s^2) R^T (Sec. 3.3) partitioned as
    [[A, b], [b^T, c]]; by Eq. 7 the conditional mean moves as mu_xyz + b (t - mu_t) / c, so b / c is
    the Gaussian's velocity.  ISO modes tie s_x = s_y = s_z to the first log-scale; ISO_IDENTITY
    fixes R = I."""
    ls = np.asarray(g["logscale4"], np.float64)
    n = ls.shape[0]
    mode = int(g.get("mode", 0))
    s = np.exp(ls)
    if mode != 0:
        s[:, 1] = s[:, 2] = s[:, 0]
    if mode == 2:
        R = np.broadcast_to(np.eye(4), (n, 4, 4)).copy()
    else:
        R = rotation_batch(g["ql"], g["qr"])
    Sig = np.einsum("nik,nk,njk->nij", R, s * s, R)
    out = np.zeros((n, 20))
    out[:, 0] = ls[:, 3]
    out[:, 1:4] = Sig[:, 0:3, 3] / Sig[:, 3, 3][:, None]
    out[:, 4:20] = R.reshape(n, 16)
    return out


def proposal_ok(y: np.ndarray) -> np.ndarray:
    """The learned proposal y = (log s_t, v, q_l, q_r) of a point is used only when every value is
    finite, both quaternions have squared norm above 1e-8 and -20 < log s_t < 5; otherwise the point
    falls back to the heuristic.  Decided on the float32 values, in float32."""
    y = np.asarray(y, np.float32)
    fin = np.all(np.isfinite(y), axis=1)
    with np.errstate(over="ignore", invalid="ignore"):
        nl = np.sum(y[:, 4:8] * y[:, 4:8], axis=1, dtype=np.float32)
        nr = np.sum(y[:, 8:12] * y[:, 8:12], axis=1, dtype=np.float32)
    return fin & (nl > np.float32(1e-8)) & (nr > np.float32(1e-8)) & (y[:, 0] > -20) & (y[:, 0] < 5)


def init_learned(pruned: dict, spatial, mlp_out, st_dynamic: float, st_static: float = 1.0,
                 opacity: float = 0.1):
    """4D Gaussians from pruned voxels with a per-point spatial scale and, where the proposal passes
    proposal_ok(), the proposed temporal log-scale and quaternions; every other point takes the
    heuristic of Sec. 4.1 (s_t by the dynamic flag, q_l = q_r = 1).  mlp_out None: the heuristic for
    every point.  Returns (gaussians dict, number of fallbacks)."""
    n = len(pruned["rep"])
    mean4 = np.c_[np.asarray(pruned["centroid"], np.float64), np.asarray(pruned["t"], np.float64)]
    ls = np.zeros((n, 4))
    ls[:, :3] = np.log(np.asarray(spatial, np.float64)).reshape(-1, 1)
    ls[:, 3] = np.where(np.asarray(pruned["flag"]) != 0, math.log(st_dynamic), math.log(st_static))
    ql = np.zeros((n, 4))
    ql[:, 0] = 1.0
    qr = ql.copy()
    fallbacks = 0
    if mlp_out is not None:
        y = np.asarray(mlp_out, np.float32)
        ok = proposal_ok(y)
        fallbacks = int((~ok).sum())
        ls[ok, 3] = y[ok, 0]
        ql[ok] = y[ok, 4:8]
        qr[ok] = y[ok, 8:12]
    g = dict(mean4=mean4, logscale4=ls, ql=ql, qr=qr,
             opacity=np.full(n, math.log(opacity / (1.0 - opacity))),
             rgb=np.asarray(pruned["rgb"], np.float64), sh=np.zeros((n, 0, 3)), sh_deg=0, mode=0)
    return g, fallbacks
