"""Learned initialisation: data from plain fits, MLP training with the library's kernels, and the
comparison with the plain heuristic initialisation (seconds and iterations to a held-out PSNR).

A scene is a seeded room video of the synthetic generator at reduced size (so that 64 scenes can be
fitted in minutes): its depth maps are pruned on the GPU (Sec. 3.2), the kept points get
neighbourhood features, and targets are rendered from the matching hidden 4D Gaussian scene.  The
plain method initialises the temporal scale and rotation by the heuristic of Sec. 4.1 / Sec. 3.3;
the learned one asks the MLP.  Both use the same spatial scale (mean distance to the 3 nearest
pruned points) and the same training step (slice/project, bin, render, L1 + D-SSIM loss, backward, Adam).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

import synth

from . import _lib as L
from . import rasterizer as R
from . import train as T
from .prune import Pruner

N_OUT = 12


@dataclass
class SceneConfig:
    n_frames: int = 200          # length of the video (time axis), frames sampled every `stride`
    stride: int = 4
    W: int = 320                 # depth-map resolution
    H: int = 180
    voxel: float = 0.02
    min_support: int = 2
    view: tuple = (480, 270)     # training / evaluation resolution
    batch: int = 4               # views per step
    heldout: int = 8             # held-out views at half-frame offsets
    hidden_n: int = 60000        # Gaussians of the hidden scene
    iters: int = 2000
    eval_every: int = 50


@dataclass
class Scene:
    seed: int
    cfg: SceneConfig
    n: int = 0
    pts: dict = field(default_factory=dict)
    feats: torch.Tensor = None
    knn3: torch.Tensor = None
    bank: torch.Tensor = None
    cam_bank: torch.Tensor = None
    held_img: torch.Tensor = None
    held_cams: torch.Tensor = None


def _camera_centre(cam) -> np.ndarray:
    return -np.asarray(cam["R"], np.float64).T @ np.asarray(cam["t"], np.float64)


def build_scene(seed: int, cfg: SceneConfig, dev) -> Scene:
    frames = list(range(0, cfg.n_frames, cfg.stride))
    vid = synth.depth_video(seed, n_frames=cfg.n_frames, W=cfg.W, H=cfg.H, frames=frames)
    F = len(frames)
    pr = Pruner(F * cfg.W * cfg.H, 1 << 22 if F * cfg.W * cfg.H > (1 << 24) else 1 << 20, device=dev)
    out = pr.prune_depth(torch.from_numpy(vid["depth"]).to(dev), torch.from_numpy(vid["rgb"]).to(dev),
                         torch.from_numpy(vid["dyn"]).to(dev), R.cameras_tensor(vid["cams"], dev), cfg.voxel,
                         cfg.voxel, cfg.min_support)
    if int(out["status"].item()) != 0:
        raise L.I4DError("pruning table overflow")
    n = int(out["n_kept"].item())
    sc = Scene(seed, cfg, n)
    sc.pts = {k: out[k][:n].clone() for k in ("xyz", "rgb", "t", "flag")}
    ref = np.mean([_camera_centre(c) for c in vid["cams"]], axis=0)
    slots = 1
    while slots < 2 * n:
        slots <<= 1
    sc.feats = torch.zeros(n, 64, device=dev)
    sc.knn3 = torch.zeros(n, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(L.i4d_knn_workspace_size(n, slots), dtype=torch.uint8, device=dev)
    L.i4d_knn_features(sc.pts["xyz"], sc.pts["rgb"], sc.pts["t"], sc.pts["flag"], cfg.voxel, 2, ref, sc.feats,
                       sc.knn3, slots, status, ws)
    if int(status.item()) != 0:
        raise L.I4DError("kNN table overflow")
    # targets: the hidden scene of the same room seen from the arc, at the video frames and at
    # held-out half-frame offsets
    hidden = synth.room_gaussians(1000 + seed, cfg.hidden_n, video_seed=seed, n_frames=cfg.n_frames)
    hp = R.pack_params(hidden, dev)
    W, H = cfg.view
    cams = [synth.arc_camera(k, cfg.n_frames, W, H) for k in frames]
    held = [synth.arc_camera(k, cfg.n_frames, W, H, time=(k + 0.5) / (cfg.n_frames - 1))
            for k in np.linspace(cfg.stride, cfg.n_frames - 2 * cfg.stride, cfg.heldout).astype(int)]
    sc.bank = torch.empty(len(cams), 3 * W * H, device=dev)
    hr = R.Rasterizer(hidden["mean4"].shape[0], 0, 0, [(W, H)] * 8, device=dev)
    allc = cams + held
    imgs = []
    for k0 in range(0, len(allc), 8):
        chunk = allc[k0:k0 + 8]
        chunk = chunk + [chunk[-1]] * (8 - len(chunk))
        img = hr.forward(hp, R.cameras_tensor(chunk, dev)).view(8, 3 * W * H)
        imgs.append(img[: min(8, len(allc) - k0)].clone())
    allimg = torch.cat(imgs)
    sc.bank = allimg[: len(cams)].contiguous()
    sc.held_img = allimg[len(cams):].contiguous().view(-1)
    sc.cam_bank = R.cameras_tensor(cams, dev)
    sc.held_cams = R.cameras_tensor(held, dev)
    return sc


def init_params(sc: Scene, weights: torch.Tensor = None, opacity: float = 0.1, gate: str = "all"):
    """Heuristic (weights None) or learned initialisation of the scene's Gaussians.  gate "dynamic":
    the network's proposals replace the heuristic only on the points of the dynamic mask; static
    points keep the heuristic of Sec. 4.1 (temporal scale of the whole video, R = I), which is what a
    static point's fit keeps."""
    n, dev = sc.n, sc.feats.device
    params = torch.empty(5 * n * 4, device=dev)
    st_dyn, st_static = T.temporal_scales(sc.cfg.n_frames)
    y = None
    if weights is not None:
        y = torch.empty(n, N_OUT, device=dev)
        L.i4d_mlp_forward(sc.feats, weights, y)
        heur = torch.zeros_like(y)
        heur[:, 0] = torch.where(sc.pts["flag"] != 0, math.log(st_dyn), math.log(st_static))
        heur[:, 4] = heur[:, 8] = 1.0
        if gate == "dynamic":
            static = sc.pts["flag"] == 0
            y[static] = heur[static]
        elif gate == "st":          # the temporal scale from the network, the rotation of the heuristic
            y[:, 4:] = heur[:, 4:]
        elif gate == "half":        # halfway between the heuristic and the proposal (normalised quaternions)
            ql = y[:, 4:8] / y[:, 4:8].norm(dim=1, keepdim=True).clamp_min(1e-12)
            qr = y[:, 8:12] / y[:, 8:12].norm(dim=1, keepdim=True).clamp_min(1e-12)
            ql = ql * torch.where(ql[:, :1] < 0, -1.0, 1.0)
            qr = qr * torch.where(qr[:, :1] < 0, -1.0, 1.0)
            y = 0.5 * (y + heur)
            y[:, 4:8] = 0.5 * (ql + heur[:, 4:8])
            y[:, 8:12] = 0.5 * (qr + heur[:, 8:12])
        elif gate != "all":
            raise ValueError(gate)
    fb = torch.zeros(1, dtype=torch.int32, device=dev)
    L.i4d_init_learned(sc.pts["xyz"], sc.pts["rgb"], sc.pts["t"], sc.pts["flag"], sc.knn3, y, n, 0, st_dyn, st_static,
                       opacity, params, fb)
    return params, int(fb.item())


class Evaluator:
    """Held-out PSNR of the current parameters (forward only)."""

    def __init__(self, sc: Scene):
        self.sc = sc
        self.rast = R.Rasterizer(sc.n, 0, 0, [sc.cfg.view] * sc.cfg.heldout, device=sc.feats.device)
        self.out = torch.zeros(1, device=sc.feats.device)

    def psnr(self, params) -> float:
        img = self.rast.forward(params, self.sc.held_cams)
        L.i4d_psnr(img, self.sc.held_img, self.out)
        return float(self.out.item())


def fit(sc: Scene, params: torch.Tensor, iters: int = None, eval_every: int = None, seed: int = 0,
        snapshot_at: int = None):
    """Train with the plain step; returns (history [(iteration, train seconds, held-out PSNR)], params),
    and with snapshot_at also the motion values (motion_targets) at that iteration."""
    cfg = sc.cfg
    iters = cfg.iters if iters is None else iters
    eval_every = cfg.eval_every if eval_every is None else eval_every
    step = T.TrainStep(params, sc.n, 0, 0, [cfg.view] * cfg.batch, steps=iters, loss_kind=L.LOSS_L1,
                       dssim=T.DSSIM_LAMBDA)
    ev = Evaluator(sc)
    rng = np.random.default_rng(seed)
    nf = sc.bank.shape[0]
    picks = torch.from_numpy(np.stack([rng.choice(nf, cfg.batch, replace=False) for _ in range(iters + 2)])
                             ).to(sc.feats.device)

    def load(k):
        torch.index_select(sc.bank, 0, picks[k], out=step.target.view(cfg.batch, -1))
        torch.index_select(sc.cam_bank, 0, picks[k], out=step.cams)

    # size the bins on the first batch with room for the Gaussians to grow, then capture
    load(0)
    step.rast.forward(params, step.cams, check_capacity=True)
    step.rast._alloc_bins(int(3.0 * int(step.rast.n_inst.item())) + 65536)
    step.capture(warmup=0)
    hist = [(0, 0.0, ev.psnr(params))]
    overflows = 0
    train_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = 0
    while k < iters:
        todo = min(eval_every, iters - k)
        e0.record()
        for j in range(todo):
            load(k + j + 1)
            step.replay()
        e1.record()
        torch.cuda.synchronize()
        train_ms += e0.elapsed_time(e1)
        k += todo
        if step.overflowed():  # a step of this chunk lost tile pairs: grow the bins, recapture, report
            overflows += 1
            step.rast._alloc_bins(int(1.5 * int(step.rast.n_inst.item())) + 65536)
            step.capture(warmup=0)
        hist.append((k, train_ms / 1e3, ev.psnr(params)))
        if snapshot_at is not None and k == snapshot_at:
            snap = motion_targets(params, sc.n)
    if overflows:
        hist.append(("overflow_chunks", overflows, None))
    if snapshot_at is not None:
        return hist, params, snap
    return hist, params


def _initial_weights(seed: int) -> np.ndarray:
    """He-style random weights with the quaternion heads starting at the identity rotation."""
    r = np.random.default_rng(seed)
    parts = []
    for o, i in ((64, 64), (64, 64), (12, 64)):
        parts.append(r.normal(0.0, 1.0 / math.sqrt(i), size=o * i))
        parts.append(np.zeros(o))
    w = np.concatenate(parts).astype(np.float32)
    off = 64 * 64 + 64 + 64 * 64 + 64 + 12 * 64
    w[off + 4] = 1.0
    w[off + 8] = 1.0
    return w


def train_mlp(feats: torch.Tensor, targets: torch.Tensor, steps: int = 1500, lr: float = 2e-3, seed: int = 0,
              w_st: float = 1.0, w_v: float = 1.0, w_R: float = 1.0, log=None):
    """Full-batch Adam on the MLP weights with the library's gradient kernel."""
    dev = feats.device
    nw = L.i4d_mlp_weight_count()
    w = torch.from_numpy(_initial_weights(seed)).to(dev)
    g = torch.zeros(nw, device=dev)
    m = torch.zeros(nw, device=dev)
    v = torch.zeros(nw, device=dev)
    stepc = torch.zeros(1, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, device=dev)
    ws = torch.empty(L.i4d_mlp_grad_workspace_size(feats.shape[0]), dtype=torch.uint8, device=dev)
    grp = L.AdamGroup()
    grp.begin, grp.end = 0, nw
    for k in range(4):
        grp.lr_init[k], grp.lr_final[k] = lr, lr * 0.05
    grp.decay_steps = steps
    curve = []
    for s in range(steps):
        L.i4d_mlp_grad(feats, targets, w, w_st, w_v, w_R, g, loss, ws)
        L.i4d_adam_step(w, g, m, v, [grp], stepc, 0.9, 0.999, 1e-8)
        if s % 100 == 0 or s == steps - 1:
            curve.append((s, float(loss.item())))
            if log:
                log(f"mlp step {s} loss {curve[-1][1]:.5f}")
    return w, curve


def motion_targets(params: torch.Tensor, n: int) -> torch.Tensor:
    g = L.Gaussians()
    g.params, g.n, g.sh_deg, g.mode = params.data_ptr(), n, 0, 0
    out = torch.empty(n, 20, device=params.device)
    L.i4d_motion_targets(g, out)
    return out


def heuristic_targets(sc: Scene) -> torch.Tensor:
    """The heuristic initialisation's own motion values, to judge the MLP's error against."""
    p, _ = init_params(sc, None)
    return motion_targets(p, sc.n)


def target_loss(pred: torch.Tensor, tgt: torch.Tensor, w_st=1.0, w_v=1.0, w_R=1.0) -> float:
    """Mean target loss of a set of motion values (n x 20 form) against fitted targets."""
    e0 = pred[:, 0] - tgt[:, 0]
    ev = pred[:, 1:4] - tgt[:, 1:4]
    eR = pred[:, 4:] - tgt[:, 4:]
    return float((w_st * e0 ** 2 + w_v * (ev ** 2).sum(1) + w_R * (eR ** 2).sum(1)).mean().item())


def reach(hist, target_psnr, tol=0.1):
    """First (iteration, seconds) at which the held-out PSNR is within tol dB of target_psnr."""
    for it, sec, p in hist:
        if p is not None and p >= target_psnr - tol:
            return it, sec
    return None, None


def final(hist):
    return [h for h in hist if h[2] is not None][-1]


def experiment(train_seeds, test_seeds, cfg: SceneConfig = None, mlp_steps: int = 1500, log=print, dev=None,
               gates=("all",), mid_iter: int = None):
    """Train the MLP on plain fits of the training scenes; on each test scene compare seconds and
    iterations to the plain method's final held-out PSNR (within 0.1 dB), for each proposal gate
    ("all": every point takes the network's proposal; "dynamic": only the dynamic points; "st": the
    temporal scale only; "half": halfway between heuristic and proposal).  With mid_iter, a second
    network is trained on the plain fits' motion values at that iteration and tested with gate all
    (tag "learned_mid")."""
    cfg = cfg or SceneConfig()
    dev = dev or torch.device("cuda")
    feats, tgts, tgts_mid = [], [], []
    t0 = time.time()
    for s in train_seeds:
        sc = build_scene(s, cfg, dev)
        params, _ = init_params(sc, None)
        if mid_iter is not None:
            hist, params, snap = fit(sc, params, seed=s, snapshot_at=mid_iter)
            tgts_mid.append(snap)
        else:
            hist, params = fit(sc, params, seed=s)
        feats.append(sc.feats)
        tgts.append(motion_targets(params, sc.n))
        log(f"train scene {s}: n={sc.n} plain PSNR {final(hist)[2]:.2f} dB ({time.time() - t0:.0f} s)")
        del sc
    F = torch.cat(feats)
    w, curve = train_mlp(F, torch.cat(tgts), steps=mlp_steps, log=log)
    nets = [(gate, w, "learned" if gate == "all" else f"learned_{gate}") for gate in gates]
    if mid_iter is not None:
        w_mid, _ = train_mlp(F, torch.cat(tgts_mid), steps=mlp_steps, log=log)
        nets.append(("all", w_mid, "learned_mid"))
    del F
    rows = []
    for s in test_seeds:
        sc = build_scene(s, cfg, dev)
        p_plain, _ = init_params(sc, None)
        h_plain, p_plain = fit(sc, p_plain, seed=s)
        fitted = motion_targets(p_plain, sc.n)
        target = final(h_plain)[2]
        it_p, sec_p = reach(h_plain, target)
        row = dict(seed=s, n=sc.n, n_dynamic=int(sc.pts["flag"].sum().item()), plain_psnr_final=target,
                   plain_iters=it_p, plain_seconds=sec_p, plain_seconds_final=final(h_plain)[1],
                   init_psnr_plain=h_plain[0][2], target_loss_heuristic=target_loss(heuristic_targets(sc), fitted),
                   plain_curve=[(h[0], h[2]) for h in h_plain if h[2] is not None])
        for gate, wt, tag in nets:
            p_learn, fallbacks = init_params(sc, wt, gate=gate)
            err_learned = target_loss(motion_targets(p_learn, sc.n), fitted)
            h_learn, _ = fit(sc, p_learn, seed=s)
            it_l, sec_l = reach(h_learn, target)
            row.update({f"{tag}_psnr_final": final(h_learn)[2], f"{tag}_iters": it_l, f"{tag}_seconds": sec_l,
                        f"{tag}_seconds_final": final(h_learn)[1], f"init_psnr_{tag}": h_learn[0][2],
                        f"target_loss_{tag}": err_learned, f"fallbacks_{tag}": fallbacks,
                        f"{tag}_curve": [(h[0], h[2]) for h in h_learn if h[2] is not None]})
        rows.append(row)
        log(f"test scene {s}: " + ", ".join(f"{k}={v:.3f}" if isinstance(v, float) else f"{k}={v}"
                                            for k, v in rows[-1].items() if not k.endswith("curve")))
        del sc
    return rows, curve, [tag for _, _, tag in nets]


# the full-size scenes: the benched room video (200 frames of 640x360 depth, voxel 0.01, support 3,
# ~1.13 M Gaussians) fitted from 960x540 views against a 200k-Gaussian hidden scene
FULL_SIZE = dict(stride=1, W=640, H=360, voxel=0.01, min_support=3, view=(960, 540), batch=4, hidden_n=200000)


def summarize(rows, tags):
    """Means over the test scenes where each run reached the plain fit's final PSNR."""
    out = {}
    for tag in tags:
        ok = [r for r in rows if r[f"{tag}_seconds"] is not None and r["plain_seconds"] is not None]
        out[tag] = dict(reached=len(ok), of=len(rows),
                        mean_plain_iters=float(np.mean([r["plain_iters"] for r in ok])) if ok else None,
                        mean_iters=float(np.mean([r[f"{tag}_iters"] for r in ok])) if ok else None,
                        mean_plain_seconds=float(np.mean([r["plain_seconds"] for r in ok])) if ok else None,
                        mean_seconds=float(np.mean([r[f"{tag}_seconds"] for r in ok])) if ok else None,
                        faster_in=int(sum(r[f"{tag}_seconds"] < r["plain_seconds"] for r in ok)),
                        mean_plain_psnr_final=float(np.mean([r["plain_psnr_final"] for r in rows])),
                        mean_psnr_final=float(np.mean([r[f"{tag}_psnr_final"] for r in rows])))
    return out


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned vs heuristic initialisation on seeded room scenes")
    ap.add_argument("--train", type=int, default=64, help="training scenes (seeds 100, 101, ...)")
    ap.add_argument("--test", type=int, default=8, help="test scenes (seeds 200, 201, ...)")
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--mlp-steps", type=int, default=1500)
    ap.add_argument("--size", choices=["reduced", "full"], default="reduced")
    ap.add_argument("--gates", default="all,half", help="proposal gates to test (all, dynamic, st, half)")
    ap.add_argument("--mid-iter", type=int, default=None,
                    help="also train on the plain fits' motion values at this iteration")
    ap.add_argument("--out", default=None, help="write the JSON summary here")
    a = ap.parse_args(argv)
    from . import build as B
    B.build()
    cfg = SceneConfig(iters=a.iters, **(FULL_SIZE if a.size == "full" else {}))
    gates = tuple(a.gates.split(","))
    rows, curve, tags = experiment(list(range(100, 100 + a.train)), list(range(200, 200 + a.test)), cfg,
                                   a.mlp_steps, gates=gates, mid_iter=a.mid_iter)
    import sys
    args = list(argv) if argv is not None else sys.argv[1:]
    summary = dict(command="python -m paper_2510_01119_gb300.learned_init " + " ".join(args), config=cfg.__dict__,
                   size=a.size, train_scenes=a.train, test_scenes=a.test, mlp_loss_curve=curve, rows=rows,
                   summary=summarize(rows, tags))
    text = json.dumps(summary, default=float)
    if a.out:
        open(a.out, "w").write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
