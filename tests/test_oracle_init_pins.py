"""Pins of the oracle's initialisation (Sec. 4.1; Sec. 3.3 "Motion-Aware Gaussian") and of its
motion targets (velocity b / c of Eq. 7, the 4D rotation), against closed forms and against the C
oracle's independent slicing and covariance code (CPU only)."""
import math

import numpy as np
import pytest

from oracle import learned as OL

F = 200                      # frames of the video; time normalised to [0, 1], one frame = 1 / (F - 1)
ST_DYN, ST_STATIC = 2.0 / (F - 1), 1.0


def _pruned():
    """Five hand-made voxels: centroids, mean times, colours and flags."""
    return dict(rep=np.arange(5, dtype=np.uint32), count=np.ones(5, np.int32),
                centroid=np.array([[0.0, 0.0, 3.0], [0.3, -0.2, 2.5], [-0.4, 0.1, 4.0], [0.05, 0.2, 3.3],
                                   [0.2, 0.25, 2.0]]),
                t=np.array([0.5, 0.25, 0.8, 0.1, 0.95]),
                rgb=np.array([[0.2, 0.4, 0.6], [1.0, 0.0, 0.5], [0.1, 0.9, 0.3], [0.5, 0.5, 0.5], [0.0, 0.2, 1.0]]),
                flag=np.array([1, 0, 1, 0, 1], np.uint8))


def _cam(time):
    return dict(R=np.eye(3), t=np.zeros(3), fx=400.0, fy=400.0, cx=200.0, cy=150.0, W=400, H=300, time=time)


def test_init_heuristic_covariance_is_diagonal_with_paper_temporal_scales(orc):
    """R = I (q_l = q_r = 1) and the scales of Sec. 4.1: the C oracle's 4D covariance of each
    initial Gaussian is diag(s^2, s^2, s^2, s_t^2) with s_t two frames (dynamic) or the video
    length (static)."""
    pr = _pruned()
    g = orc.init_heuristic(pr, 0.01, ST_DYN, ST_STATIC)
    for i in range(5):
        Sig = orc.cov4(g["logscale4"][i], g["ql"][i], g["qr"][i])
        st = ST_DYN if pr["flag"][i] else ST_STATIC
        assert np.allclose(Sig, np.diag([1e-4, 1e-4, 1e-4, st * st]), rtol=1e-12, atol=1e-18)


def test_init_heuristic_temporal_opacity_and_static_position(orc):
    """Sliced k frames away from its mean time, a dynamic initial Gaussian keeps o_t = 0.1
    exp(-k^2 / 8) (two-frame temporal scale, opacity 0.1), a static one 0.1 exp(-(k / (F - 1))^2 / 2);
    with R = I the sliced mean stays at the voxel centroid (no motion), and the colour is the mean
    colour of the voxel."""
    pr = _pruned()
    g = orc.init_heuristic(pr, 0.01, ST_DYN, ST_STATIC)
    C = orc.P
    for i in range(5):
        gi = {k: (v[i:i + 1] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
        for k in (0, 1, 3):
            t = pr["t"][i] + k / (F - 1)
            P = orc.project(gi, _cam(t))
            want = 0.1 * (math.exp(-k * k / 8.0) if pr["flag"][i] else math.exp(-0.5 * (k / (F - 1)) ** 2))
            assert P[0, C["ot"]] == pytest.approx(want, rel=1e-12)
            assert np.allclose(P[0, [C["m3x"], C["m3y"], C["m3z"]]], pr["centroid"][i], atol=1e-15)
            assert np.allclose(P[0, [C["r"], C["g"], C["b"]]], pr["rgb"][i], atol=1e-15)


def test_init_learned_uses_valid_proposals_and_falls_back_otherwise(orc):
    """Per point: a valid proposal sets log s_t and both quaternions; a non-finite, zero-quaternion
    or out-of-range proposal falls back to the heuristic; without proposals init_learned equals
    init_heuristic with the per-point spatial scale."""
    pr = _pruned()
    spatial = np.array([0.01, 0.02, 0.015, 0.03, 0.005])
    g0, fb0 = OL.init_learned(pr, spatial, None, ST_DYN, ST_STATIC)
    assert fb0 == 0
    for i in range(5):
        gh = orc.init_heuristic({k: v[i:i + 1] for k, v in pr.items()}, spatial[i], ST_DYN, ST_STATIC)
        for k in ("mean4", "logscale4", "ql", "qr", "opacity", "rgb"):
            assert np.allclose(g0[k][i], gh[k][0], rtol=1e-15, atol=0), k
    y = np.zeros((5, 12), np.float32)
    y[:, 0] = -2.5
    y[:, 1:4] = 0.1
    y[:, 4] = y[:, 8] = 0.8
    y[:, 5] = y[:, 10] = 0.6
    y[1, 4:8] = 0.0              # zero quaternion
    y[2, 3] = np.inf             # not finite (anywhere in the proposal)
    y[3, 0] = 6.0                # log s_t out of range
    g, fb = OL.init_learned(pr, spatial, y, ST_DYN, ST_STATIC)
    assert fb == 3
    ok = np.array([True, False, False, False, True])
    assert np.allclose(g["logscale4"][ok, 3], -2.5)
    assert np.allclose(g["ql"][ok], y[ok, 4:8]) and np.allclose(g["qr"][ok], y[ok, 8:12])
    assert np.array_equal(g["logscale4"][~ok, 3], g0["logscale4"][~ok, 3])
    assert np.allclose(g["ql"][~ok], [1, 0, 0, 0]) and np.allclose(g["qr"][~ok], [1, 0, 0, 0])
    assert np.array_equal(g["mean4"], g0["mean4"]) and np.array_equal(g["logscale4"][:, :3], g0["logscale4"][:, :3])


def _random_gaussians(n, seed, mode=0):
    r = np.random.default_rng(seed)
    return dict(mean4=r.normal(size=(n, 4)), logscale4=np.c_[r.normal(-3, 0.5, (n, 3)), r.normal(-1.5, 0.3, n)],
                ql=r.normal(size=(n, 4)), qr=r.normal(size=(n, 4)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
                sh=np.zeros((n, 0, 3)), sh_deg=0, mode=mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_motion_targets_match_c_covariance_and_precision_conditioning(orc, mode):
    """The targets' R diag(s^2) R^T equals the C oracle's 4D covariance, and the velocity b / c
    equals -Lambda_xx^-1 Lambda_xt of the precision matrix Lambda = Sigma^-1 (the textbook form of
    the conditional mean's slope)."""
    g = _random_gaussians(40, 5 + mode, mode)
    tg = OL.motion_targets(g)
    for i in range(40):
        Sig = orc.cov4(g["logscale4"][i], g["ql"][i], g["qr"][i], mode=mode)
        R = tg[i, 4:20].reshape(4, 4)
        s = np.exp(g["logscale4"][i])
        if mode:
            s[1] = s[2] = s[0]
        assert np.allclose(R @ np.diag(s * s) @ R.T, Sig, rtol=1e-10, atol=1e-16)
        Lam = np.linalg.inv(Sig)
        v = -np.linalg.solve(Lam[:3, :3], Lam[:3, 3])
        assert np.allclose(tg[i, 1:4], v, rtol=1e-8, atol=1e-12)
        assert tg[i, 0] == g["logscale4"][i, 3]
    if mode == 2:
        assert np.allclose(tg[:, 1:4], 0.0) and np.allclose(tg[:, 4:20], np.eye(4).reshape(16))


def test_motion_targets_velocity_is_slope_of_sliced_mean(orc):
    """Eq. 7: the C oracle's sliced mean at two frame times moves by (b / c) dt."""
    g = _random_gaussians(30, 9)
    g["mean4"][:, 2] = 3.0 + np.abs(g["mean4"][:, 2])
    g["mean4"][:, 3] = 0.5
    g["logscale4"][:, 3] = 0.0     # wide temporal support: visible at both times
    tg = OL.motion_targets(g)
    C = orc.P
    P0, P1 = orc.project(g, _cam(0.45)), orc.project(g, _cam(0.55))
    m0 = P0[:, [C["m3x"], C["m3y"], C["m3z"]]]
    m1 = P1[:, [C["m3x"], C["m3y"], C["m3z"]]]
    vis = (P0[:, C["visible"]] != 0) & (P1[:, C["visible"]] != 0)
    assert vis.sum() > 10
    assert np.allclose((m1 - m0)[vis] / 0.1, tg[vis, 1:4], rtol=1e-9, atol=1e-12)


def test_motion_targets_plane_rotation_closed_form():
    """Isotropic spatial scale s, temporal scale s_t, and q_l = q_r = cos(th/2) + sin(th/2) u (a
    simple rotation by th in the plane of e_t and the spatial unit vector u): Sigma = s^2 I +
    (s_t^2 - s^2) e e^T with e = R e_t, so |b / c| = (s_t^2 - s^2) sin th cos th / (s^2 + (s_t^2 -
    s^2) cos^2 th) along u, and a conjugate pair (q_r = conj q_l) gives no motion."""
    s, st = 0.05, 0.4
    u = np.array([2.0, -1.0, 0.5])
    u /= np.linalg.norm(u)
    for th in (0.1, 0.6, 1.2):
        q = np.r_[math.cos(th / 2), math.sin(th / 2) * u]
        g = dict(logscale4=np.log([[s, s, s, st]]), ql=q[None], qr=q[None], mode=0)
        v = OL.motion_targets(g)[0, 1:4]
        want = (st * st - s * s) * math.sin(th) * math.cos(th) / (s * s + (st * st - s * s) * math.cos(th) ** 2)
        assert abs(np.dot(v, u)) == pytest.approx(want, rel=1e-12)
        assert np.allclose(np.cross(v, u), 0.0, atol=1e-14)
        qc = q * np.array([1, -1, -1, -1])
        g2 = dict(logscale4=np.log([[s, s, s, st]]), ql=q[None], qr=qc[None], mode=0)
        assert np.allclose(OL.motion_targets(g2)[0, 1:4], 0.0, atol=1e-15)
