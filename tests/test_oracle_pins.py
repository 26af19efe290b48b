"""Pins of the FP64 oracle against closed forms, textbook identities, library routines and finite
differences -- facts that do not come from the oracle itself (CPU only)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _rot3_textbook(q):
    """Rotation matrix of the unit quaternion (w, x, y, z) (standard formula for v -> q v q*)."""
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _one(mean4, ls4, ql, qr, opacity=0.0, rgb=(0.5, 0.5, 0.5), mode=0):
    return dict(mean4=np.array([mean4], np.float64), logscale4=np.array([ls4], np.float64),
                ql=np.array([ql], np.float64), qr=np.array([qr], np.float64),
                opacity=np.array([opacity], np.float64), rgb=np.array([rgb], np.float64),
                sh=np.zeros((1, 0, 3)), sh_deg=0, mode=mode)


# ---------------------------------------------------------------------------------------------
# 4D covariance and the rotation parameterisation
# ---------------------------------------------------------------------------------------------
def test_cov4_spectrum_is_scales_squared(orc):
    r = np.random.default_rng(11)
    for _ in range(20):
        ls = r.normal(-2, 0.5, 4)
        S = orc.cov4(ls, r.normal(size=4), r.normal(size=4))
        assert np.allclose(S, S.T, atol=1e-15)
        ev = np.sort(np.linalg.eigvalsh(S))
        assert np.allclose(ev, np.sort(np.exp(2 * ls)), rtol=1e-10)


def test_cov4_conjugate_pair_is_3d_rotation(orc):
    """q_r = conj(q_l): the 4D rotation fixes t and rotates xyz by the textbook matrix of q_l."""
    r = np.random.default_rng(12)
    for _ in range(10):
        q = r.normal(size=4)
        qc = q * np.array([1, -1, -1, -1])
        ls = r.normal(-2, 0.5, 4)
        S = orc.cov4(ls, q, qc)
        R3 = _rot3_textbook(q)
        assert np.allclose(S[:3, :3], R3 @ np.diag(np.exp(2 * ls[:3])) @ R3.T, atol=1e-14)
        assert np.allclose(S[:3, 3], 0.0, atol=1e-15)
        assert S[3, 3] == pytest.approx(math.exp(2 * ls[3]), rel=1e-13)


def test_cov4_plane_rotation_closed_form(orc):
    """q_l = q_r = cos(th/2) + sin(th/2) i rotates the (x, t) plane by th:
    S_xx = sx^2 cos^2 + st^2 sin^2, S_xt = (st^2 - sx^2) sin cos, S_tt = sx^2 sin^2 + st^2 cos^2."""
    th = 0.7
    q = np.array([math.cos(th / 2), math.sin(th / 2), 0, 0])
    ls = np.log([0.1, 0.2, 0.3, 0.5])
    S = orc.cov4(ls, q, q)
    sx2, sy2, sz2, st2 = np.exp(2 * ls)
    c, s = math.cos(th), math.sin(th)
    assert S[0, 0] == pytest.approx(sx2 * c * c + st2 * s * s, rel=1e-13)
    assert S[0, 3] == pytest.approx((st2 - sx2) * s * c, rel=1e-13)
    assert S[3, 3] == pytest.approx(sx2 * s * s + st2 * c * c, rel=1e-13)
    assert S[1, 1] == pytest.approx(sy2, rel=1e-13) and S[2, 2] == pytest.approx(sz2, rel=1e-13)
    assert abs(S[0, 1]) < 1e-15 and abs(S[1, 3]) < 1e-15


def test_cov4_isotropic_modes(orc):
    r = np.random.default_rng(13)
    ls = np.array([-2.0, 5.0, 5.0, -1.0])  # y, z ignored in the isotropic modes
    S = orc.cov4(ls, r.normal(size=4), r.normal(size=4), mode=orc.MODE_ISO_IDENTITY)
    assert np.allclose(S, np.diag(np.exp(2 * ls[[0, 0, 0, 3]])), atol=1e-15)
    S = orc.cov4(ls, r.normal(size=4), r.normal(size=4), mode=orc.MODE_ISO_ROT)
    assert np.allclose(np.sort(np.linalg.eigvalsh(S)), np.sort(np.exp(2 * ls[[0, 0, 0, 3]])), rtol=1e-10)


# ---------------------------------------------------------------------------------------------
# Eq. 7-8 conditioning and the temporal opacity
# ---------------------------------------------------------------------------------------------
def test_slice_matches_precision_matrix_conditioning(orc):
    """Conditional mean/covariance of a Gaussian from the precision matrix L = S^-1:
    cov3|t = (L_xx)^-1, mean3|t = mu - (L_xx)^-1 L_xt (t - mu_t)."""
    g = synth.gaussians_uniform(5, n=50)
    cam = synth.camera(64, 48, time=0.37)
    P = orc.project(g, cam)
    C = orc.P
    for i in range(50):
        S = orc.cov4(g["logscale4"][i], g["ql"][i], g["qr"][i])
        L = np.linalg.inv(S)
        cov3 = np.linalg.inv(L[:3, :3])
        mu = g["mean4"][i].astype(np.float64)
        mean3 = mu[:3] - cov3 @ L[:3, 3] * (float(cam["time"]) - mu[3])
        got_m = P[i, [C["m3x"], C["m3y"], C["m3z"]]]
        got_c = P[i, [C["s3xx"], C["s3xy"], C["s3xz"], C["s3yy"], C["s3yz"], C["s3zz"]]]
        want_c = cov3[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
        assert np.allclose(got_m, mean3, rtol=1e-11, atol=1e-13)
        assert np.allclose(got_c, want_c, rtol=1e-9, atol=1e-15)


def test_temporal_opacity_is_marginal_over_peak(orc):
    """o_t / sigmoid(o) equals the xyz-marginal of the 4D density at t divided by its value at
    t = mu_t (quadrature of the 4D density on a grid)."""
    from scipy.stats import multivariate_normal
    r = np.random.default_rng(14)
    ls = np.array([-1.0, -1.2, -0.9, -1.3])
    ql, qr = r.normal(size=4), r.normal(size=4)
    S = orc.cov4(ls, ql, qr)
    mu = np.array([0.0, 0.0, 4.0, 0.5])
    rv = multivariate_normal(mean=mu, cov=S)
    sd = np.sqrt(np.diag(S))
    axes = [np.linspace(mu[k] - 7 * sd[k], mu[k] + 7 * sd[k], 41) for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")

    def marginal(t):
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel(), np.full(X.size, t)], -1)
        return rv.pdf(pts).sum()

    for t in (0.35, 0.62):
        ratio = marginal(t) / marginal(mu[3])
        g = _one(mu, ls, ql, qr, opacity=0.3)
        P = orc.project(g, synth.camera(64, 48, time=t))
        sig = 1 / (1 + math.exp(-0.3))
        assert P[0, orc.P["ot"]] / sig == pytest.approx(ratio, rel=1e-6)


# ---------------------------------------------------------------------------------------------
# EWA projection against Monte-Carlo projected samples
# ---------------------------------------------------------------------------------------------
def test_ewa_covariance_matches_projected_samples(orc):
    r = np.random.default_rng(15)
    ls = np.log([0.002, 0.001, 0.0015, 0.3])
    ql, qr = synth.random_unit_quats(r, 1)[0], synth.random_unit_quats(r, 1)[0]
    mu = np.array([0.9, -0.55, 3.0, 0.5])
    R, t = synth.look_at([0.2, 0.1, -0.3], [0.3, 0.0, 3.0])
    cam = synth.camera(256, 192, 60.0, R, t, time=0.5)
    g = _one(mu, ls, ql, qr)
    P = orc.project(g, cam, settings=orc.settings_array(dilation=0.0))
    C = orc.P
    m3 = P[0, [C["m3x"], C["m3y"], C["m3z"]]]
    c3 = P[0, [C["s3xx"], C["s3xy"], C["s3xz"], C["s3yy"], C["s3yz"], C["s3zz"]]]
    cov3 = np.array([[c3[0], c3[1], c3[2]], [c3[1], c3[3], c3[4]], [c3[2], c3[4], c3[5]]])
    x = r.multivariate_normal(m3, cov3, size=200000)
    xc = x @ np.asarray(R, np.float64).T + np.asarray(t, np.float64)
    u = cam["fx"] * xc[:, 0] / xc[:, 2] + cam["cx"]
    v = cam["fy"] * xc[:, 1] / xc[:, 2] + cam["cy"]
    emp = np.cov(np.stack([u, v]))
    conic = np.array([[P[0, C["ca"]], P[0, C["cb"]]], [P[0, C["cb"]], P[0, C["cc"]]]])
    cov2 = np.linalg.inv(conic)
    assert abs(u.mean() - P[0, C["u"]]) < 0.02 and abs(v.mean() - P[0, C["v"]]) < 0.02
    assert np.allclose(cov2, emp, rtol=0.02, atol=0.02 * np.abs(emp).max())
    assert abs(cov2[0, 1]) > 0.1 * np.sqrt(cov2[0, 0] * cov2[1, 1])  # the test exercises a tilted ellipse


# ---------------------------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------------------------
def test_single_gaussian_closed_form(orc):
    g = _one([0.05, -0.03, 2.5, 0.5], np.log([0.08, 0.05, 0.06, 0.4]), [1, 0.1, 0.2, 0], [1, -0.1, -0.2, 0],
             opacity=1.5, rgb=(0.9, 0.2, 0.4))
    cam = synth.camera(40, 30, time=0.6)
    bg = np.array([0.2, 0.3, 0.4])
    P = orc.project(g, cam)
    img, T, nc, _ = orc.render(P, cam, bg=bg)
    C = orc.P
    u, v, ot = P[0, C["u"]], P[0, C["v"]], P[0, C["ot"]]
    a_, b_, c_ = P[0, C["ca"]], P[0, C["cb"]], P[0, C["cc"]]
    for p in range(40 * 30):
        dx, dy = p % 40 + 0.5 - u, p // 40 + 0.5 - v
        q = a_ * dx * dx + 2 * b_ * dx * dy + c_ * dy * dy
        al = min(0.99, ot * math.exp(-0.5 * q))
        if q > 9 or al < 1 / 255:
            al = 0.0
        assert np.allclose(img[p], al * np.array([0.9, 0.2, 0.4]) + (1 - al) * bg, atol=1e-14)
        assert T[p] == pytest.approx(1 - al, abs=1e-14)
        assert nc[p] == (1 if al > 0 else 0)
    assert nc.sum() > 20


def test_front_to_back_order_and_occlusion(orc):
    """The nearer Gaussian is blended first: C = a1 c1 + (1 - a1) a2 c2."""
    near = _one([0, 0, 2.0, 0.5], np.log([0.3, 0.3, 0.3, 10]), [1, 0, 0, 0], [1, 0, 0, 0], opacity=3.0, rgb=(1, 0, 0))
    far = _one([0, 0, 3.0, 0.5], np.log([0.3, 0.3, 0.3, 10]), [1, 0, 0, 0], [1, 0, 0, 0], opacity=3.0, rgb=(0, 0, 1))
    both = {k: (np.concatenate([far[k], near[k]]) if isinstance(far[k], np.ndarray) else far[k]) for k in far}
    cam = synth.camera(16, 16, time=0.5)
    P = orc.project(both, cam)
    img, T, nc, _ = orc.render(P, cam, pix=[8 * 16 + 8])
    a1 = min(0.99, P[1, orc.P["ot"]] * math.exp(-0.5 * _q(P[1], 8.5, 8.5)))
    a2 = min(0.99, P[0, orc.P["ot"]] * math.exp(-0.5 * _q(P[0], 8.5, 8.5)))
    assert img[0] == pytest.approx([a1, 0, (1 - a1) * a2], abs=1e-14)
    assert T[0] == pytest.approx((1 - a1) * (1 - a2), abs=1e-14)


def test_render_alternatives_enumerate_near_equal_depths(orc):
    """Three Gaussians at depths within 1e-7 of each other cover the pixel: every one of the 3! orders
    is a valid result, and each equals the closed-form front-to-back sum of that order; far apart
    (1e-3) only the (depth, id) order is; the first listed colour is render()'s."""
    import itertools
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    cam = synth.camera(16, 16, time=0.5)
    for gap, want_n in ((1e-7, 6), (1e-3, 1)):
        gs = [_one([0, 0, 3.0 + k * gap, 0.5], np.log([0.3, 0.3, 0.3, 10]), [1, 0, 0, 0], [1, 0, 0, 0],
                   opacity=0.5 - 0.4 * k, rgb=cols[k]) for k in range(3)]
        g = {k: (np.concatenate([x[k] for x in gs]) if isinstance(gs[0][k], np.ndarray) else gs[0][k]) for k in gs[0]}
        P = orc.project(g, cam)
        alt, n_alt = orc.render_alternatives(P, cam, [8 * 16 + 8], 1e-4, 2e-6, 5e-5)
        assert n_alt[0] == want_n
        img, _, _, _ = orc.render(P, cam, pix=[8 * 16 + 8])
        assert np.allclose(alt[0, 0], img[0], atol=1e-15)
        a = [min(0.99, P[k, orc.P["ot"]] * math.exp(-0.5 * _q(P[k], 8.5, 8.5))) for k in range(3)]
        want = set()
        for perm in itertools.permutations(range(3)) if want_n == 6 else [(0, 1, 2)]:
            C, T = np.zeros(3), 1.0
            for k in perm:
                C += T * a[k] * np.asarray(cols[k], float)
                T *= 1 - a[k]
            want.add(tuple(np.round(C, 12)))
        got = {tuple(np.round(c, 12)) for c in alt[0, :n_alt[0]]}
        assert got == want


def test_render_alternatives_branch_on_near_threshold_decisions(orc):
    """A fragment whose alpha sits 1e-7 (relative) above alpha_min may be blended or not, and a
    blend that takes T to within 1e-6 of T_min may stop the pixel or not: both colours are valid,
    each in closed form; the same cases 1% away from the thresholds have one colour."""
    cam = synth.camera(17, 17, time=0.5)      # principal point (8.5, 8.5): pixel (8, 8)'s centre
    px = 8 * 17 + 8
    C = orc.P
    # one Gaussian facing the camera, centred on the pixel centre (q = 0): alpha = o_t
    for rel, want_n in ((1e-7, 2), (1e-2, 1)):
        ot = (1 / 255) * (1 + rel)
        g = _one([0, 0, 3.0, 0.5], np.log([0.3, 0.3, 0.3, 1e6]), [1, 0, 0, 0], [1, 0, 0, 0],
                 opacity=math.log(ot / (1 - ot)), rgb=(0.2, 0.5, 0.9))
        P = orc.project(g, cam)
        a = P[0, C["ot"]] * math.exp(-0.5 * _q(P[0], 8.5, 8.5))
        alt, n_alt = orc.render_alternatives(P, cam, [px], 1e-4, 2e-6, 1e-6)
        assert a == pytest.approx(ot, rel=1e-12)
        assert n_alt[0] == want_n
        want = {tuple(np.round(a * np.array([0.2, 0.5, 0.9]), 12))} | ({(0.0, 0.0, 0.0)} if want_n == 2 else set())
        assert {tuple(np.round(c, 12)) for c in alt[0, :want_n]} == want
    # a stack of alpha-0.9 Gaussians: T = 0.1, 0.01, 1e-3, 1e-4 (1 + rel) after the fourth
    for rel, want_n in ((1e-6, 2), (1e-2, 1)):
        T4 = 1e-4 * (1 + rel)
        al = 1 - T4 ** 0.25
        gs = [_one([0, 0, 3.0 + 0.01 * k, 0.5], np.log([0.3, 0.3, 0.3, 1e6]), [1, 0, 0, 0], [1, 0, 0, 0],
                   opacity=math.log(al / (1 - al)), rgb=(1.0, 1.0, 1.0)) for k in range(4)]
        g = {k: (np.concatenate([x[k] for x in gs]) if isinstance(gs[0][k], np.ndarray) else gs[0][k]) for k in gs[0]}
        P = orc.project(g, cam)
        alt, n_alt = orc.render_alternatives(P, cam, [px], 1e-4, 2e-6, 1e-6)
        assert n_alt[0] == want_n
        ak = [P[k, C["ot"]] * math.exp(-0.5 * _q(P[k], 8.5, 8.5)) for k in range(4)]
        T3 = np.prod([1 - x for x in ak[:3]])
        full = 1 - T3 * (1 - ak[3])           # white: C = 1 - T after four blends
        stopped = 1 - T3                      # the fourth stops the pixel
        got = sorted(round(c[0], 12) for c in alt[0, :want_n])
        want = sorted({round(full, 12), round(stopped, 12)}) if want_n == 2 else [round(full if rel > 0 else stopped, 12)]
        assert got == want


def _q(rec, x, y):
    C = {k: i for i, k in enumerate(
        ["visible", "u", "v", "depth", "ot", "ca", "cb", "cc"])}
    dx, dy = x - rec[C["u"]], y - rec[C["v"]]
    return rec[C["ca"]] * dx * dx + 2 * rec[C["cb"]] * dx * dy + rec[C["cc"]] * dy * dy


def test_transmittance_stop_rule(orc):
    """Stacked Gaussians of alpha 0.95: T = 0.05, 0.0025, 1.25e-4; the 4th would take T below
    1e-4 and ends the walk, so exactly three are blended."""
    n = 6
    g = dict(mean4=np.array([[0, 0, 2.0 + 0.1 * k, 0.5] for k in range(n)]),
             logscale4=np.tile(np.log([1.0, 1.0, 1.0, 10.0]), (n, 1)),
             ql=np.tile([1.0, 0, 0, 0], (n, 1)), qr=np.tile([1.0, 0, 0, 0], (n, 1)),
             opacity=np.full(n, math.log(0.95 / 0.05)), rgb=np.tile([1.0, 1.0, 1.0], (n, 1)),
             sh=np.zeros((n, 0, 3)), sh_deg=0, mode=0)
    cam = synth.camera(17, 17, time=0.5)  # the centre pixel's centre is the principal point: q = 0
    P = orc.project(g, cam)
    img, T, nc, _ = orc.render(P, cam, pix=[8 * 17 + 8])
    assert nc[0] == 3
    assert T[0] == pytest.approx(0.05 ** 3, rel=1e-6)


def test_partition_of_unity_and_transmittance_bounds(orc):
    g = synth.gaussians_uniform(0)
    g["rgb"] = np.ones_like(g["rgb"])
    cam = synth.camera(128, 96, time=0.5)
    img, T, nc, _ = orc.render(orc.project(g, cam), cam)
    assert np.allclose(img + T[:, None], 1.0, atol=1e-12)
    assert np.all(T <= 1.0) and np.all(T >= 1e-4 * 0.01 - 1e-15)
    assert np.all((T < 1.0) == (nc > 0))


# ---------------------------------------------------------------------------------------------
# infinite temporal scale reduces to 3D Gaussian splatting
# ---------------------------------------------------------------------------------------------
def _render_3dgs_numpy(mu3, scales3, quats, opac, rgb, cam, settings):
    """Plain 3D Gaussian splatting, written independently of the 4D oracle (vectorised numpy)."""
    alpha_max, alpha_min, T_min, q_max, _, z_near, dil, fovc = settings
    W, H = cam["W"], cam["H"]
    R = np.asarray(cam["R"], np.float64)
    tt = np.asarray(cam["t"], np.float64)
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    n = mu3.shape[0]
    recs = []
    for i in range(n):
        Rq = _rot3_textbook(quats[i])
        cov = Rq @ np.diag(scales3[i] ** 2) @ Rq.T
        m = R @ mu3[i] + tt
        o = 1.0 / (1.0 + math.exp(-opac[i]))
        if m[2] <= z_near or o < 1 / 255:
            continue
        limx, limy = fovc * 0.5 * W / fx, fovc * 0.5 * H / fy
        rx = np.clip(m[0] / m[2], -limx, limx)
        ry = np.clip(m[1] / m[2], -limy, limy)
        J = np.array([[fx / m[2], 0, -fx * rx / m[2]], [0, fy / m[2], -fy * ry / m[2]]])
        c2 = J @ R @ cov @ R.T @ J.T + dil * np.eye(2)
        recs.append((m[2], i, fx * m[0] / m[2] + cx, fy * m[1] / m[2] + cy, np.linalg.inv(c2), o))
    recs.sort(key=lambda r: (r[0], r[1]))
    img = np.zeros((H * W, 3))
    Ts = np.ones(H * W)
    ys, xs = np.divmod(np.arange(H * W), W)
    done = np.zeros(H * W, bool)
    for depth, i, u, v, Q, o in recs:
        dx, dy = xs + 0.5 - u, ys + 0.5 - v
        q = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
        a = np.minimum(alpha_max, o * np.exp(-0.5 * q))
        use = (~done) & (q <= q_max) & (a >= alpha_min)
        Tn = Ts * (1 - a)
        stop = use & (Tn < T_min)
        done |= stop
        use &= ~stop
        img[use] += (Ts[use] * a[use])[:, None] * rgb[i]
        Ts = np.where(use, Tn, Ts)
    return img, Ts


def test_infinite_temporal_scale_is_3dgs(orc):
    g = synth.gaussians_uniform(3, n=150)
    g = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    g["mean4"][:, :2] *= 0.4
    g["logscale4"][:, 3] = 30.0                                   # s_t -> infinity
    g["qr"] = g["ql"] * np.array([1, -1, -1, -1])                 # q_r = conj(q_l): R fixes t
    cam = synth.camera(48, 36, time=0.83)
    S = orc.settings_array()
    img, T, _, _ = orc.render(orc.project(g, cam, settings=S), cam, settings=S)
    ref, Tref = _render_3dgs_numpy(g["mean4"][:, :3], np.exp(g["logscale4"][:, :3]), g["ql"], g["opacity"],
                                   g["rgb"], cam, S)
    assert np.abs(img - ref).max() < 1e-12
    assert np.abs(T - Tref).max() < 1e-12
    assert (T < 1).sum() > 200


# ---------------------------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------------------------
def test_sh_orthonormal_by_quadrature(orc):
    zs, wz = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * 2 * np.pi / 32
    G = np.zeros((15, 15))
    for z, w in zip(zs, wz):
        for ph in phis:
            s = math.sqrt(1 - z * z)
            Y = orc.sh_basis(np.array([s * math.cos(ph), s * math.sin(ph), z]))
            G += w * (2 * np.pi / 32) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(15), atol=1e-12)


def test_sh_matches_scipy_real_form(orc):
    """Real SH from scipy's complex Y_l^m: m>0: sqrt2 (-1)^m Re Y_l^m, m<0: sqrt2 (-1)^m Im Y_l^|m|."""
    sp = pytest.importorskip("scipy.special")
    r = np.random.default_rng(16)
    for _ in range(20):
        d = r.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = orc.sh_basis(d)
        for l in range(1, 4):
            for m in range(-l, l + 1):
                c = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                want = c.real if m == 0 else math.sqrt(2) * (-1) ** m * (c.real if m > 0 else c.imag)
                assert Y[l * l + l + m - 1] == pytest.approx(want, abs=1e-12)


# ---------------------------------------------------------------------------------------------
# backward against central finite differences of the oracle's own forward
# ---------------------------------------------------------------------------------------------
def _fd_scene(seed, n, mode, sh_deg):
    r = np.random.default_rng(seed)
    g = dict(mean4=np.c_[r.uniform(-0.35, 0.35, (n, 2)), r.uniform(2.5, 3.5, n), r.uniform(0.3, 0.7, n)],
             logscale4=np.c_[r.normal(-1.9, 0.25, (n, 3)), r.normal(-1.0, 0.3, n)],
             ql=r.normal(size=(n, 4)), qr=r.normal(size=(n, 4)), opacity=r.normal(-0.5, 0.5, n),
             rgb=r.uniform(0.2, 0.8, (n, 3)), sh=r.normal(0, 0.1, (n, (sh_deg + 1) ** 2 - 1, 3)),
             sh_deg=sh_deg, mode=mode)
    # one Gaussian past the field-of-view clamp, wide enough for its tail to reach the image
    g["mean4"][0, :3] = [2.6, 0.1, 3.0]
    g["logscale4"][0, :3] = [-0.6, -0.7, -0.5]
    return g


def _loss(orc, g, cam, w, S):
    img, T, nc, _ = orc.render(orc.project(g, cam, settings=S), cam, settings=S)
    return float(np.sum(w * img)), nc


@pytest.mark.parametrize("mode,cutoffs", [(0, False), (0, True), (1, False), (2, False)])
def test_backward_matches_central_differences(orc, mode, cutoffs):
    sh_deg = 3 if mode == 0 else 1
    g = _fd_scene(20 + mode, 16, mode, sh_deg)
    cam = synth.camera(32, 32, time=0.5)
    if cutoffs:
        S = orc.settings_array()
    else:
        S = orc.settings_array(alpha_min=0.0, T_min=0.0, q_max=1e30, ot_min=0.0)
    w = np.random.default_rng(7).normal(size=(32 * 32, 3))
    _, grads = orc.render_bwd(g, cam, w, settings=S)
    h = 1e-6
    checked = considered = 0
    for key in ("mean4", "logscale4", "ql", "qr", "opacity", "rgb", "sh"):
        arr = g[key]
        for idx in np.ndindex(arr.shape):
            if key == "logscale4" and mode != 0 and idx[-1] in (1, 2):
                continue
            considered += 1
            old = arr[idx]
            arr[idx] = old + h
            lp, ncp = _loss(orc, g, cam, w, S)
            arr[idx] = old - h
            lm, ncm = _loss(orc, g, cam, w, S)
            arr[idx] = old
            if cutoffs and not np.array_equal(ncp, ncm):
                continue  # a threshold decision flipped inside the stencil
            fd = (lp - lm) / (2 * h)
            an = grads[key][idx]
            assert abs(an - fd) <= 2e-6 * max(1.0, abs(fd)), (key, idx, an, fd)
            checked += 1
    assert considered > 400 and checked >= 0.8 * considered
    # the clamped-FOV Gaussian must have contributed
    assert np.abs(grads["mean4"][0]).sum() > 0


# ---------------------------------------------------------------------------------------------
# SCH appearance variant (Sec. 3.1)
# ---------------------------------------------------------------------------------------------
def test_sch_reduces_to_sh_and_matches_closed_forms(orc):
    C = orc.P
    g = _fd_scene(31, 12, 0, 1)
    cam = synth.camera(32, 32, time=0.3)
    base = orc.project(g, cam)
    # one temporal term, or all-zero coefficients: exactly the SH colour
    g1 = dict(g, sch_terms=1)
    assert np.array_equal(orc.project(g1, cam), base)
    g3 = dict(g, sch_terms=3, sch=np.zeros((12, 2, 4, 3)))
    assert np.array_equal(orc.project(g3, cam), base)
    # the constant harmonic of term m = 2: colour + cos(4 pi t) c
    g3["sch"][:, 1, 0, :] = 0.05
    P3 = orc.project(g3, cam)
    want = base[:, [C["r"], C["g"], C["b"]]] + np.cos(4 * np.pi * np.float32(0.3)) * 0.05
    np.testing.assert_allclose(P3[:, [C["r"], C["g"], C["b"]]], np.maximum(want, 0), atol=1e-12)
    # harmonic k = 1 (Y = c1 y with c1 = sqrt(3 / (4 pi))) of term m = 1: + cos(2 pi t) c1 dhat_y c
    g4 = dict(g, sch_terms=2, sch=np.zeros((12, 1, 4, 3)))
    g4["sch"][:, 0, 1, 1] = 0.2
    P4 = orc.project(g4, cam)
    eye = -np.asarray(cam["R"], np.float64).T @ np.asarray(cam["t"], np.float64)
    d = P4[:, [C["m3x"], C["m3y"], C["m3z"]]] - eye
    dy = d[:, 1] / np.linalg.norm(d, axis=1)
    want_g = base[:, C["g"]] + np.cos(2 * np.pi * np.float32(0.3)) * np.sqrt(3 / (4 * np.pi)) * dy * 0.2
    np.testing.assert_allclose(P4[:, C["g"]], np.maximum(want_g, 0), atol=1e-12)


def test_sch_backward_matches_central_differences(orc):
    g = _fd_scene(32, 10, 0, 2)
    g["sch_terms"] = 3
    g["sch"] = np.random.default_rng(5).normal(0, 0.05, (10, 2, 9, 3))
    cam = synth.camera(32, 32, time=0.37)
    S = orc.settings_array(alpha_min=0.0, T_min=0.0, q_max=1e30, ot_min=0.0)
    w = np.random.default_rng(8).normal(size=(32 * 32, 3))
    _, grads = orc.render_bwd(g, cam, w, settings=S)
    h = 1e-6
    for key, arr in (("sch", g["sch"]), ("mean4", g["mean4"])):
        for idx in list(np.ndindex(arr.shape))[:: 7 if key == "sch" else 1]:
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = _loss(orc, g, cam, w, S)
            arr[idx] = old - h
            lm, _ = _loss(orc, g, cam, w, S)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(grads[key][idx] - fd) <= 2e-6 * max(1.0, abs(fd)), (key, idx, grads[key][idx], fd)


# ---------------------------------------------------------------------------------------------
# tile pairs
# ---------------------------------------------------------------------------------------------
def _blendable_tiles(P, i, C, W, H, tile=16):
    """Brute force: the tiles holding a pixel where Gaussian i can be blended (q <= 9 and
    o_t exp(-q/2) >= 1/255), and the tiles holding a pixel with q <= 9 (the 3-sigma ellipse)."""
    ys, xs = np.divmod(np.arange(W * H), W)
    dx, dy = xs + 0.5 - P[i, C["u"]], ys + 0.5 - P[i, C["v"]]
    q = P[i, C["ca"]] * dx * dx + 2 * P[i, C["cb"]] * dx * dy + P[i, C["cc"]] * dy * dy
    tx = (W + tile - 1) // tile
    t_of = (ys // tile) * tx + xs // tile
    blend = (q <= 9) & (P[i, C["ot"]] * np.exp(-0.5 * q) >= 1 / 255)
    return set(t_of[blend].tolist()), set(t_of[q <= 9].tolist())


def test_tile_lists_are_the_tiles_of_blendable_pixels_in_order(orc):
    """Brute force over every pixel of the view: a Gaussian's tiles are exactly those holding a
    pixel centre with q <= 9 and o_t exp(-q/2) >= 1/255 (up to the pairs the oracle marks as within
    1e-4 of a threshold), listed by (tile, depth, id); fewer than the 3-sigma ellipse's tiles."""
    g = synth.gaussians_uniform(0)
    for cam, tile in ((synth.camera(128, 96, time=0.5), 16), (synth.camera(75, 41, 55.0, time=0.3), 8)):
        W, H = cam["W"], cam["H"]
        P = orc.project(g, cam)
        tiles, ids, st = orc.tile_lists(P, cam, tile=(tile, tile), tile_offset=7)
        C = orc.P
        key = list(zip(tiles, P[ids, C["depth"]], ids))
        assert key == sorted(key)
        assert len(set(zip(tiles.tolist(), ids.tolist()))) == len(tiles)
        have, maybe = {}, {}
        for t, i, s_ in zip(tiles.tolist(), ids.tolist(), st.tolist()):
            (have if s_ == 1 else maybe).setdefault(i, set()).add(t - 7)
        need_total = sigma3_total = 0
        for i in range(P.shape[0]):
            need, sigma3 = _blendable_tiles(P, i, C, W, H, tile)
            if P[i, C["visible"]] == 0:
                need = set()
            assert have.get(i, set()) <= need <= have.get(i, set()) | maybe.get(i, set()), i
            need_total += len(need)
            sigma3_total += len(sigma3) if need else 0
        assert (st == 1).sum() <= need_total <= len(tiles) and (st == 2).sum() < 0.01 * len(tiles)
        assert need_total < sigma3_total


def test_tile_lists_shrink_with_temporal_opacity_in_closed_form(orc):
    """One isotropic Gaussian facing the camera (pixel-space standard deviation s_px), 4x4 tiles:
    it can be blended out to radius s_px sqrt(min(9, 2 ln(255 o_t))), so its tiles span the tiles of
    the pixel centres inside that disc: at o_t = 0.2 less than the 3-sigma disc, just above the
    cull (o_t = 1.02/255) 0.2 sigma, at o_t = 0.99 the 3-sigma disc."""
    W = 1024
    cam = synth.camera(W, W, 60.0, time=0.5)
    C = orc.P
    ys, xs = np.divmod(np.arange(W * W), W)
    spans = {}
    for ot in (0.2, 1.02 / 255, 0.99):
        logit = math.log(ot / (1 - ot))
        g = dict(mean4=np.array([[0.0, 0.0, 3.0, 0.5]]), logscale4=np.log([[0.3, 0.3, 0.3, 1e3]]),
                 ql=np.array([[1.0, 0, 0, 0]]), qr=np.array([[1.0, 0, 0, 0]]), opacity=np.array([logit]),
                 rgb=np.ones((1, 3)), sh=np.zeros((1, 0, 3)), sh_deg=0, mode=0)
        P = orc.project(g, cam)
        assert P[0, C["ot"]] == pytest.approx(ot, rel=1e-6)
        s_px = cam["fx"] * 0.3 / 3.0                       # focal length x scale / depth
        s_px = math.sqrt(s_px * s_px + 0.3)                # plus the 0.3 px^2 dilation
        rho = s_px * math.sqrt(min(9.0, 2 * math.log(255 * ot)))
        inside = (xs + 0.5 - P[0, C["u"]]) ** 2 + (ys + 0.5 - P[0, C["v"]]) ** 2 <= rho * rho * (1 - 1e-9)
        want = set(((ys[inside] // 4) * (W // 4) + xs[inside] // 4).tolist())
        tiles, ids, st = orc.tile_lists(P, cam, tile=(4, 4))
        assert set(tiles[st == 1].tolist()) <= want <= set(tiles.tolist())
        tx = np.unique(np.asarray(sorted(want)) % (W // 4))
        spans[ot] = (len(tx), rho)
    assert spans[0.2][0] < 2 * 3 * s_px / 4 - 2            # narrower than the 3-sigma disc
    assert spans[1.02 / 255][0] < spans[0.2][0] / 5        # 0.2 sigma
    assert abs(spans[0.99][0] - 2 * 3 * s_px / 4) <= 2     # the 3-sigma disc binds


# ---------------------------------------------------------------------------------------------
# back-projection and grid pruning
# ---------------------------------------------------------------------------------------------
def test_backprojection_round_trip(orc):
    vid = synth.depth_video(2, n_frames=200, W=64, H=36, frames=[0, 117])
    for f in range(2):
        cam = vid["cams"][f]
        X = orc.backproject(cam, vid["depth"][f])
        xc = X @ np.asarray(cam["R"], np.float64).T + np.asarray(cam["t"], np.float64)
        u = float(cam["fx"]) * xc[:, 0] / xc[:, 2] + float(cam["cx"])
        v = float(cam["fy"]) * xc[:, 1] / xc[:, 2] + float(cam["cy"])
        ys, xs = np.divmod(np.arange(64 * 36), 64)
        # the float32 rotation is orthonormal only to ~1e-7, which bounds the round trip
        assert np.allclose(u, xs + 0.5, atol=1e-4) and np.allclose(v, ys + 0.5, atol=1e-4)
        assert np.allclose(xc[:, 2], vid["depth"][f].reshape(-1), rtol=1e-6)


def _cam_f32(cam):
    """The camera as the float32 values a device-side camera struct holds (kept as float64)."""
    out = dict(cam)
    out["R"] = np.asarray(cam["R"], np.float32).astype(np.float64)
    out["t"] = np.asarray(cam["t"], np.float32).astype(np.float64)
    for k in ("fx", "fy", "cx", "cy"):
        out[k] = float(np.float32(cam[k]))
    return out


def test_backprojection_f32_within_rounding_bound_of_f64(orc):
    """The float32 reading of Eq. 5 (a fixed sequence of correctly rounded float32 operations) lies
    within the forward-error bound of that sequence from the float64 back-projection of the same
    (float32-rounded) camera and depth: with u = 2^-24, X_c,x carries at most 3 roundings
    (subtract, divide, multiply), d_j = X_c,j - tau_j one more, and each output two products' and
    two sums' worth, so |X32_a - X64_a| <= 8 u sum_j |W_ja| (|X_c,j| + |tau_j|).  A dropped term, a
    wrong sign or a transposed rotation moves a point by ~|W_ja d_j|, orders of magnitude more."""
    vid = synth.depth_video(2, n_frames=200, W=96, H=54, frames=[0, 77, 199])
    u = 2.0 ** -24
    ys, xs = np.divmod(np.arange(96 * 54), 96)
    for f in range(3):
        cam = _cam_f32(vid["cams"][f])
        X64 = orc.backproject(cam, vid["depth"][f])
        X32 = orc.backproject_f32(cam, vid["depth"][f])
        assert X32.dtype == np.float32
        D = vid["depth"][f].reshape(-1).astype(np.float64)
        Xc = np.c_[D * (xs + 0.5 - cam["cx"]) / cam["fx"], D * (ys + 0.5 - cam["cy"]) / cam["fy"], D]
        R = np.asarray(cam["R"], np.float64)
        mag = (np.abs(Xc) + np.abs(cam["t"])[None, :]) @ np.abs(R)   # sum_j |W_ja| (|X_c,j| + |tau_j|)
        err = np.abs(X32.astype(np.float64) - X64)
        assert np.all(err <= 8 * u * mag), float((err / (u * mag)).max())
        # the bound is not vacuous: the float32 result is not the float64 one rounded at the end
        assert (X32.astype(np.float64) != X64.astype(np.float32).astype(np.float64)).any()
    # the video helper concatenates frames in point order f*H*W + py*W + px
    cat = orc.backproject_video_f32(vid)
    assert np.array_equal(cat[96 * 54:2 * 96 * 54], orc.backproject_f32(vid["cams"][1], vid["depth"][1]))


def test_backprojection_f32_single_pixel_by_hand(orc):
    """One pixel of the float32 sequence worked through with numpy float32 scalars in the stated
    order (every operation rounds to float32, none fused)."""
    R = np.array([[0.8, -0.6, 0.0], [0.36, 0.48, -0.8], [0.48, 0.64, 0.6]])
    cam = dict(R=R, t=np.array([0.1, -0.2, 0.3]), fx=500.0, fy=510.0, cx=320.0, cy=180.0, W=4, H=3, time=0.0)
    depth = np.full((3, 4), 2.5, np.float32)
    depth[2, 3] = np.float32(3.1)
    out = orc.backproject_f32(cam, depth)[2 * 4 + 3]
    f = np.float32
    D = f(3.1)
    xc = D * ((f(3) + f(0.5) - f(320.0)) / f(500.0))
    yc = D * ((f(2) + f(0.5) - f(180.0)) / f(510.0))
    d = [xc - f(0.1), yc - f(-0.2), D - f(0.3)]
    Rf = R.astype(np.float32)
    want = [(Rf[0, a] * d[0] + Rf[1, a] * d[1]) + Rf[2, a] * d[2] for a in range(3)]
    assert np.array_equal(out, np.array(want, np.float32))


@pytest.mark.parametrize("min_support", [1, 2, 5])
def test_prune_matches_numpy_groupby(orc, min_support):
    r = np.random.default_rng(30 + min_support)
    n = 20000
    xyz = (r.normal(size=(n, 3)) * 0.3).astype(np.float32)
    rgb = r.uniform(0, 1, (n, 3)).astype(np.float32)
    t = r.uniform(0, 1, n).astype(np.float32)
    dyn = (r.uniform(size=n) < 0.3).astype(np.uint8)
    vs, vd = 0.05, 0.08
    out = orc.prune(xyz, vs, vd, min_support, rgb=rgb, t=t, dyn=dyn)
    inv = np.where(dyn[:, None] == 1, np.float32(1) / np.float32(vd), np.float32(1) / np.float32(vs)).astype(np.float32)
    cell = np.floor(xyz * inv).astype(np.int64)       # float32 product, then floor
    key = np.c_[dyn.astype(np.int64), cell]
    uk, inverse, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inverse = inverse.reshape(-1)
    rep = np.full(len(uk), n, np.int64)
    np.minimum.at(rep, inverse, np.arange(n))
    keep = counts >= min_support
    order = np.argsort(rep[keep])
    assert np.array_equal(out["rep"], rep[keep][order])
    assert np.array_equal(out["count"], counts[keep][order])
    sums = np.stack([np.bincount(inverse, weights=xyz[:, k].astype(np.float64)) for k in range(3)], -1)
    assert np.allclose(out["centroid"], (sums / counts[:, None])[keep][order], rtol=0, atol=1e-12)
    tsum = np.bincount(inverse, weights=t.astype(np.float64))
    assert np.allclose(out["t"], (tsum / counts)[keep][order], atol=1e-12)
    assert np.array_equal(out["flag"], uk[keep][order][:, 0])
    # invariants: dropped points + kept counts = n; centroid lies in its voxel (convexity)
    assert out["count"].sum() == n - counts[~keep].sum()
    vsz = np.where(out["flag"] == 1, vd, vs)[:, None]
    cells = uk[keep][order][:, 1:]
    assert np.all(out["centroid"] >= cells * vsz - 1e-6) and np.all(out["centroid"] <= (cells + 1) * vsz + 1e-6)


def test_prune_full_variant_keeps_every_dynamic_point(orc):
    """voxel_dynamic = 0 (the Full model): static points are pruned as usual, and every dynamic point
    is kept as its own voxel, whatever the minimum support."""
    r = np.random.default_rng(40)
    n = 8000
    xyz = (r.normal(size=(n, 3)) * 0.2).astype(np.float32)
    t = r.uniform(0, 1, n).astype(np.float32)
    dyn = (r.uniform(size=n) < 0.25).astype(np.uint8)
    vs, ms = 0.05, 3
    out = orc.prune(xyz, vs, 0.0, ms, t=t, dyn=dyn)
    # static part: numpy group-by with the minimum support
    st = np.nonzero(dyn == 0)[0]
    cell = np.floor(xyz[st] * (np.float32(1) / np.float32(vs))).astype(np.int64)
    uk, inverse, counts = np.unique(cell, axis=0, return_inverse=True, return_counts=True)
    rep = np.full(len(uk), n, np.int64)
    np.minimum.at(rep, inverse.reshape(-1), st)
    want_rep = np.sort(np.concatenate([rep[counts >= ms], np.nonzero(dyn)[0]]))
    assert np.array_equal(out["rep"], want_rep)
    d = dyn[out["rep"]] == 1
    assert np.array_equal(out["flag"], dyn[out["rep"]])
    assert np.all(out["count"][d] == 1)
    assert np.array_equal(out["centroid"][d], xyz[out["rep"][d]].astype(np.float64))
    assert np.array_equal(out["t"][d], t[out["rep"][d]].astype(np.float64))


# ---------------------------------------------------------------------------------------------
# Adam
# ---------------------------------------------------------------------------------------------
def test_adam_matches_torch(orc):
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(40)
    p0 = r.normal(size=100)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-15)
    mine = (p0.copy(), np.zeros(100), np.zeros(100))
    for step in range(1, 6):
        gr = r.normal(size=100)
        p.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
        mine = orc.adam_step(mine[0], gr, mine[1], mine[2], 3e-3, step)
    st = opt.state[p]
    assert np.allclose(mine[0], p.detach().numpy(), rtol=0, atol=1e-13)
    assert np.allclose(mine[1], st["exp_avg"].numpy(), atol=1e-15)
    assert np.allclose(mine[2], st["exp_avg_sq"].numpy(), atol=1e-15)
