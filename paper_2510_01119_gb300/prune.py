"""Voxel-grid pruning through libi4d (Eq. 5 back-projection + Sec. 3.2 grid pruning)."""
from __future__ import annotations

import torch

from . import _lib as L


def _outputs(capacity: int, device):
    return dict(rep=torch.empty(capacity, dtype=torch.int32, device=device),
                count=torch.empty(capacity, dtype=torch.int32, device=device),
                xyz=torch.empty(capacity, 3, dtype=torch.float32, device=device),
                rgb=torch.empty(capacity, 3, dtype=torch.float32, device=device),
                t=torch.empty(capacity, dtype=torch.float32, device=device),
                flag=torch.empty(capacity, dtype=torch.uint8, device=device),
                n_kept=torch.zeros(1, dtype=torch.int64, device=device),
                status=torch.zeros(1, dtype=torch.int32, device=device))


def table_slots_for(n_points: int, expected_voxels: int = None) -> int:
    target = 2 * (expected_voxels if expected_voxels else max(n_points // 8, 1024))
    s = 1024
    while s < target:
        s <<= 1
    return s


class Pruner:
    """Owns the hash-table workspace; call prune_depth / prune_xyz (results stay on the device)."""

    def __init__(self, n_points: int, table_slots: int, capacity: int = None, device="cuda"):
        L.load()
        self.table_slots = int(table_slots)
        self.capacity = int(capacity or table_slots)
        self.device = torch.device(device)
        self.ws = torch.empty(L.i4d_prune_workspace_size(n_points, self.table_slots), dtype=torch.uint8,
                              device=self.device)
        self.out = _outputs(self.capacity, self.device)

    def prune_depth(self, depth, rgb, dyn, cams, voxel_static, voxel_dynamic=None, min_support=1):
        F, H, W = depth.shape
        o = self.out
        L.i4d_prune_points(depth, rgb, dyn, cams, F, W, H, voxel_static,
                           voxel_dynamic if voxel_dynamic is not None else voxel_static, min_support,
                           self.table_slots, self.capacity, o["rep"], o["count"], o["xyz"], o["rgb"], o["t"],
                           o["flag"], o["n_kept"], o["status"], self.ws)
        return o

    def prune_xyz(self, xyz, rgb=None, t=None, dyn=None, voxel_static=0.01, voxel_dynamic=None, min_support=1):
        o = self.out
        L.i4d_prune_points_xyz(xyz, rgb, t, dyn, voxel_static,
                               voxel_dynamic if voxel_dynamic is not None else voxel_static, min_support,
                               self.table_slots, self.capacity, o["rep"], o["count"], o["xyz"], o["rgb"], o["t"],
                               o["flag"], o["n_kept"], o["status"], self.ws)
        return o

    def result(self):
        """Host copy of the kept voxels (syncs); raises on device-reported overflow."""
        o = self.out
        st = int(o["status"].item())
        if st != 0:
            raise L.I4DError(f"prune: {L.STATUS.get(st, st)} (kept {int(o['n_kept'].item())})")
        k = int(o["n_kept"].item())
        return {key: (v[:k].cpu().numpy() if key not in ("n_kept", "status") else v.cpu().numpy())
                for key, v in o.items()}


def adaptive_voxel(depth: torch.Tensor, cams: torch.Tensor, lambda_s: float = 1.0) -> torch.Tensor:
    """Eq. 6 on the GPU: lambda_s times the mean over frames of mean depth / focal length (1 float)."""
    out = torch.zeros(1, dtype=torch.float32, device=depth.device)
    ws = torch.empty(L.i4d_adaptive_voxel_workspace_size(depth.shape[0]), dtype=torch.uint8, device=depth.device)
    L.i4d_adaptive_voxel(depth, cams, lambda_s, out, ws)
    return out


def motion_masks(prob: torch.Tensor, W: int, H: int):
    """Otsu masks of the low-resolution motion-probability maps (F, h, w) at W x H: (masks, thresholds)."""
    F = prob.shape[0]
    mask = torch.empty(F, H, W, dtype=torch.uint8, device=prob.device)
    th = torch.empty(F, dtype=torch.int32, device=prob.device)
    ws = torch.empty(L.i4d_motion_masks_workspace_size(F), dtype=torch.uint8, device=prob.device)
    L.i4d_motion_masks(prob, W, H, mask, th, ws)
    return mask, th


def model_voxels(model: str, unit: float):
    """(voxel_static, voxel_dynamic) of the paper's two models (Sec. 4.1) for the Eq. 6 unit
    (lambda_s = 1): Lite prunes both regions at 4 units; Full prunes static regions at 1 unit and
    keeps every dynamic point (voxel_dynamic = 0)."""
    if model == "lite":
        return 4.0 * unit, 4.0 * unit
    if model == "full":
        return 1.0 * unit, 0.0
    raise ValueError(model)
