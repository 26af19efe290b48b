"""One optimisation step of the method (Sec. 3.3 / Sec. 4.1) as a fixed sequence of libi4d calls:
slice_project -> bin_tiles -> render_fwd -> loss -> render_bwd -> adam_step, on pointer-stable
device buffers so that the step can be captured once as a CUDA graph and replayed.
"""
from __future__ import annotations

import math

import torch

from . import _lib as L
from .rasterizer import PLANE_MEAN, PLANE_ORGB, PLANE_QL, PLANE_QR, PLANE_SCALE, PLANE_SH, Rasterizer, n_planes

# Learning rates of the standard 3D splatting optimiser with the paper's position rate
# (Sec. 4.1: position learning rate 1e-5, decayed over the scheduler's length).
DEFAULT_LR = dict(position=1e-5, position_final=1e-7, time=1e-5, scale=5e-3, rotation=1e-3, opacity=5e-2,
                  rgb=2.5e-3, sh=2.5e-3 / 20.0)


def adam_groups(n: int, sh_deg: int, steps: int, lr: dict = None, sch_terms: int = 0):
    lr = dict(DEFAULT_LR, **(lr or {}))
    groups = []

    def grp(plane_lo, plane_hi, lanes0, lanes1=None, decay=0):
        g = L.AdamGroup()
        g.begin, g.end = plane_lo * 4 * n, plane_hi * 4 * n
        lanes1 = lanes0 if lanes1 is None else lanes1
        for k in range(4):
            g.lr_init[k], g.lr_final[k] = lanes0[k], lanes1[k]
        g.decay_steps = decay
        groups.append(g)

    p, pf, t = lr["position"], lr["position_final"], lr["time"]
    grp(PLANE_MEAN, PLANE_MEAN + 1, [p, p, p, t], [pf, pf, pf, t * pf / p], decay=steps)
    grp(PLANE_SCALE, PLANE_SCALE + 1, [lr["scale"]] * 4)
    grp(PLANE_QL, PLANE_QR + 1, [lr["rotation"]] * 4)
    grp(PLANE_ORGB, PLANE_ORGB + 1, [lr["opacity"], lr["rgb"], lr["rgb"], lr["rgb"]])
    if sh_deg > 0:
        grp(PLANE_SH, n_planes(sh_deg), [lr["sh"]] * 4)
    if sch_terms > 1:  # the SCH variant's coefficients learn at the SH rate
        grp(n_planes(sh_deg), n_planes(sh_deg, sch_terms), [lr["sh"]] * 4)
    return groups


# the D-SSIM weight of the standard 3D Gaussian splatting loss (Sec. 4.1 adopts its loss weights)
DSSIM_LAMBDA = 0.2


class TrainStep:
    """Device-resident training step for a fixed batch layout (view sizes) of n Gaussians.  The loss is
    (1 - dssim) L1 + dssim (1 - SSIM) when dssim > 0, else i4d_loss of loss_kind (L1 or MSE)."""

    def __init__(self, params: torch.Tensor, n: int, sh_deg: int, mode: int, sizes, steps: int,
                 loss_kind: int = L.LOSS_L1, capacity: int = None, tile=(16, 16), lr: dict = None,
                 dssim: float = 0.0, sch_terms: int = 0, batch: int = 0):
        self.params = params
        self.n, self.sh_deg, self.mode = n, sh_deg, mode
        # the step needs no per-pixel fragment counts (Rasterizer.count can be switched on to read them)
        self.rast = Rasterizer(n, sh_deg, mode, sizes, tile=tile, capacity=capacity, sch_terms=sch_terms,
                               batch=batch, count=False)
        dev = params.device
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.cams = torch.zeros(len(sizes), 20, dtype=torch.float32, device=dev)
        self.target = torch.zeros(3 * self.rast.total_pixels, dtype=torch.float32, device=dev)
        self.dL = torch.empty_like(self.target)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.loss_kind = loss_kind
        self.dssim = float(dssim)
        self.ssim = torch.zeros(1, dtype=torch.float32, device=dev)
        self.loss_ws = (torch.empty(L.i4d_photometric_loss_workspace_size(self.rast.views), dtype=torch.uint8,
                                    device=dev) if self.dssim > 0 else None)
        self.groups = adam_groups(n, sh_deg, steps, lr, sch_terms)
        self.graph = None

    def run(self):
        """Enqueue one step on the current stream (no host synchronisation)."""
        r = self.rast
        r.project(self.params, self.cams)
        r.bin()
        r.composite()
        if self.dssim > 0:
            L.i4d_photometric_loss(r.views, r.img, self.target, self.dssim, self.dL, self.loss, self.ssim,
                                   self.loss_ws)
        else:
            L.i4d_loss(r.img, self.target, self.loss_kind, self.dL, self.loss)
        r.backward(self.params, self.cams, self.dL)
        L.i4d_adam_step(self.params, r.grads, self.m, self.v, self.groups, self.step_count)

    def capture(self, warmup: int = 1):
        """Capture run() into a CUDA graph (after eager warm-up steps on a side stream)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

    def overflowed(self) -> bool:
        """True if the last bin step exceeded the instance capacity (host sync)."""
        return int(self.rast.status.item()) != 0 or int(self.rast.n_inst.item()) > self.rast.capacity


def sizes_for_batch(full=(960, 540), half=(480, 270), n_full=4, n_half=4):
    return [full] * n_full + [half] * n_half


def scale_for_voxel(voxel: float) -> float:
    """Isotropic spatial scale of a freshly initialised Gaussian: half the voxel edge (the
    distance between neighbouring pruned centroids is about one voxel)."""
    return 0.5 * voxel


def temporal_scales(n_frames: int):
    """(s_t dynamic, s_t static) in the normalised time axis: two frames, and the video length."""
    return 2.0 / max(n_frames - 1, 1), 1.0


def log_lr(lr0, lr1, frac):
    return math.exp((1 - frac) * math.log(lr0) + frac * math.log(lr1))
