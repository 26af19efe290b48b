"""Device buffers and autograd glue around libi4d (PyTorch supplies memory, streams, autograd).

The flat parameter layout (see include/i4d.h): planes of N float4 -- mean4, logscale4, q_l, q_r,
(opacity logit, r, g, b), then the SH planes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

PLANE_MEAN, PLANE_SCALE, PLANE_QL, PLANE_QR, PLANE_ORGB, PLANE_SH = 0, 1, 2, 3, 4, 5


def sh_planes(deg: int) -> int:
    return {0: 0, 1: 3, 2: 6, 3: 12}[deg]


def sch_planes(deg: int, nt: int) -> int:
    """Planes of the SCH variant's (nt - 1) x (deg + 1)^2 x 3 coefficients (0 for nt <= 1)."""
    return ((nt - 1) * (deg + 1) ** 2 * 3 + 3) // 4 if nt > 1 else 0


def n_planes(deg: int, nt: int = 0) -> int:
    return 5 + sh_planes(deg) + sch_planes(deg, nt)


def pack_params(g: dict, device="cuda") -> torch.Tensor:
    """Gaussian dict (mean4 (n,4), logscale4, ql, qr, opacity (n,), rgb (n,3), sh (n,K,3), sh_deg; for the
    SCH variant also sch_terms N_t and sch (n, N_t - 1, (deg + 1)^2, 3)) -> flat float32 tensor."""
    n = int(np.asarray(g["mean4"]).shape[0])
    deg = int(g.get("sh_deg", 0))
    nt = int(g.get("sch_terms", 0))
    planes = np.zeros((n_planes(deg, nt), n, 4), np.float32)
    planes[PLANE_MEAN] = g["mean4"]
    planes[PLANE_SCALE] = g["logscale4"]
    planes[PLANE_QL] = g["ql"]
    planes[PLANE_QR] = g["qr"]
    planes[PLANE_ORGB, :, 0] = g["opacity"]
    planes[PLANE_ORGB, :, 1:] = g["rgb"]
    if deg > 0:
        K = (deg + 1) ** 2 - 1
        flat = np.zeros((n, sh_planes(deg) * 4), np.float32)
        flat[:, :3 * K] = np.asarray(g["sh"], np.float32).reshape(n, 3 * K)
        planes[PLANE_SH:PLANE_SH + sh_planes(deg)] = flat.reshape(n, sh_planes(deg), 4).transpose(1, 0, 2)
    if nt > 1:
        m = (nt - 1) * (deg + 1) ** 2 * 3
        flat = np.zeros((n, sch_planes(deg, nt) * 4), np.float32)
        flat[:, :m] = np.asarray(g["sch"], np.float32).reshape(n, m)
        planes[PLANE_SH + sh_planes(deg):] = flat.reshape(n, sch_planes(deg, nt), 4).transpose(1, 0, 2)
    return torch.from_numpy(planes.reshape(-1)).to(device)


def unpack_params(flat: torch.Tensor, n: int, deg: int, nt: int = 0) -> dict:
    """Inverse of pack_params (numpy float32 dict, same keys)."""
    a = flat.detach().cpu().numpy().reshape(n_planes(deg, nt), n, 4)
    out = dict(mean4=a[PLANE_MEAN].copy(), logscale4=a[PLANE_SCALE].copy(), ql=a[PLANE_QL].copy(),
               qr=a[PLANE_QR].copy(), opacity=a[PLANE_ORGB, :, 0].copy(), rgb=a[PLANE_ORGB, :, 1:].copy(),
               sh_deg=deg)
    K = (deg + 1) ** 2 - 1
    if deg > 0:
        out["sh"] = a[PLANE_SH:PLANE_SH + sh_planes(deg)].transpose(1, 0, 2).reshape(n, -1)[:, :3 * K].reshape(
            n, K, 3).copy()
    else:
        out["sh"] = np.zeros((n, 0, 3), np.float32)
    if nt > 1:
        m = (nt - 1) * (deg + 1) ** 2 * 3
        out["sch_terms"] = nt
        out["sch"] = a[PLANE_SH + sh_planes(deg):].transpose(1, 0, 2).reshape(n, -1)[:, :m].reshape(
            n, nt - 1, (deg + 1) ** 2, 3).copy()
    return out


def camera_array(cams) -> np.ndarray:
    """List of camera dicts (R, t, fx, fy, cx, cy, time) -> (V, 20) float32 in the i4d_camera layout."""
    out = np.zeros((len(cams), 20), np.float32)
    for k, c in enumerate(cams):
        out[k, 0:9] = np.asarray(c["R"], np.float32).reshape(9)
        out[k, 9:12] = np.asarray(c["t"], np.float32).reshape(3)
        out[k, 12:17] = [c["fx"], c["fy"], c["cx"], c["cy"], c["time"]]
    return out


def cameras_tensor(cams, device="cuda") -> torch.Tensor:
    return torch.from_numpy(camera_array(cams)).to(device)


class Rasterizer:
    """Owns every device buffer of the forward/backward of one batch of views."""

    def __init__(self, n: int, sh_deg: int, mode: int, sizes, tile=(16, 16), capacity: int = None,
                 settings: dict = None, device="cuda", sch_terms: int = 0, batch: int = 0, count: bool = True):
        """batch: list entries the forward stages per warp and round (16, 32, 64; 0 = 32); count:
        write n_contrib (fragments blended per pixel) in the forward."""
        L.load()
        self.n, self.sh_deg, self.mode = int(n), int(sh_deg), int(mode)
        self.sch_terms = int(sch_terms)
        self.sizes = [(int(w), int(h)) for (w, h) in sizes]
        self.tile = tuple(tile)
        self.device = torch.device(device)
        self.views = L.make_views(self.sizes, self.tile)
        self.settings = L.default_settings(**(settings or {}))
        self.tune = L.Tune()
        self.tune.batch = int(batch)
        self.count = bool(count)
        self.V = len(self.sizes)
        self.total_tiles = int(L.load().i4d_total_tiles(ctypes.byref(self.views)))
        self.total_pixels = int(L.load().i4d_total_pixels(ctypes.byref(self.views)))
        VN = self.V * self.n
        dev = self.device
        self.proj = torch.empty(4 * VN * 4, dtype=torch.float32, device=dev)
        self.touched = torch.empty(max(VN, 1), dtype=torch.int32, device=dev)
        self.ranges = torch.empty(3 * max(self.total_tiles, 1), dtype=torch.int32, device=dev)
        self.n_inst = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.img = torch.empty(3 * self.total_pixels, dtype=torch.float32, device=dev)
        self.T_final = torch.empty(self.total_pixels, dtype=torch.float32, device=dev)
        self.last = torch.empty(self.total_pixels, dtype=torch.int32, device=dev)
        self.n_contrib = torch.empty(self.total_pixels, dtype=torch.int32, device=dev)
        self.grad2d = torch.empty(L.GRAD2D_FLOATS * max(VN, 1), dtype=torch.float32, device=dev)
        self.grads = torch.empty(n_planes(self.sh_deg, self.sch_terms) * self.n * 4, dtype=torch.float32,
                                 device=dev)
        self._alloc_bins(capacity if capacity else max(1 << 16, 8 * VN))

    def _alloc_bins(self, capacity: int):
        self.capacity = int(capacity)
        self.ids = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
        ws = L.i4d_bin_tiles_workspace_size(self.views, self.n, self.capacity)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def gaussians(self, params: torch.Tensor) -> L.Gaussians:
        g = L.Gaussians()
        g.params = params.data_ptr()
        g.n, g.sh_deg, g.mode, g.sch_terms = self.n, self.sh_deg, self.mode, self.sch_terms
        return g

    # ---- the three forward calls ----------------------------------------------------------------------
    def project(self, params, cams):
        L.i4d_slice_project(self.gaussians(params), self.views, cams, self.settings, self.proj, self.touched)

    def bin(self):
        L.i4d_bin_tiles(self.views, self.n, self.proj, self.touched, self.capacity, self.ids, self.ranges,
                        self.n_inst, self.status, self.ws)

    def composite(self):
        L.i4d_render_fwd(self.views, self.n, self.proj, self.ids, self.ranges, self.settings, self.tune, self.img,
                         self.T_final, self.last, self.n_contrib if self.count else None)

    def forward(self, params: torch.Tensor, cams: torch.Tensor, check_capacity: bool = True) -> torch.Tensor:
        """slice_project -> bin_tiles -> render_fwd.  With check_capacity the instance count is read
        back (one host sync) and the bins are regrown and redone on overflow."""
        self.project(params, cams)
        self.bin()
        if check_capacity:
            n_inst = int(self.n_inst.item())
            if n_inst > self.capacity:
                self._alloc_bins(int(n_inst * 1.25) + 1024)
                self.bin()
        self.composite()
        return self.img

    def backward(self, params: torch.Tensor, cams: torch.Tensor, dL_dimg: torch.Tensor) -> torch.Tensor:
        L.i4d_render_bwd(self.gaussians(params), self.views, cams, self.settings, self.proj, self.touched, self.ids,
                         self.ranges, self.T_final, self.last, dL_dimg.contiguous(), self.grad2d, self.grads)
        return self.grads

    # ---- helpers -------------------------------------------------------------------------------------------
    def split_images(self, img: torch.Tensor = None):
        """Flat image buffer -> list of (3, H, W) views."""
        img = self.img if img is None else img
        out, off = [], 0
        for (W, H) in self.sizes:
            out.append(img[off:off + 3 * W * H].view(3, H, W))
            off += 3 * W * H
        return out

    def split_pixels(self, buf: torch.Tensor):
        out, off = [], 0
        for (W, H) in self.sizes:
            out.append(buf[off:off + W * H].view(H, W))
            off += W * H
        return out

    def tile_lists(self):
        """Host copy of the sorted (tile, id) pairs: (tiles int64, ids int64)."""
        n = min(int(self.n_inst.item()), self.capacity)
        ids = self.ids[:n].cpu().numpy().astype(np.int64)
        rg = self.ranges[:2 * self.total_tiles].view(-1, 2).cpu().numpy().astype(np.int64)
        tiles = np.zeros(n, np.int64)
        for t in np.nonzero(rg[:, 1] > rg[:, 0])[0]:
            tiles[rg[t, 0]:rg[t, 1]] = t
        return tiles, ids


class Render4D(torch.autograd.Function):
    """img = render(params, cams); backward through i4d_render_bwd (transmittance recomputed)."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, cams: torch.Tensor, rast: Rasterizer):
        img = rast.forward(params.detach(), cams)
        ctx.rast = rast
        ctx.save_for_backward(params, cams)
        return img.clone()

    @staticmethod
    def backward(ctx, grad_img):
        params, cams = ctx.saved_tensors
        g = ctx.rast.backward(params.detach(), cams, grad_img.contiguous())
        return g.clone(), None, None


def render(params: torch.Tensor, cams: torch.Tensor, rast: Rasterizer) -> torch.Tensor:
    return Render4D.apply(params, cams, rast)
