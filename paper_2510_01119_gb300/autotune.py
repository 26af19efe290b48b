"""Launch autotuner: picks the screen-tile shape and the forward's staging batch (list entries each
warp tests and stages in shared memory per round) of a training step by timing it.

The rendered image depends on neither (a Gaussian covers a pixel exactly when its q <= q_max test
passes, whatever the binning, and every staged entry is visited in list order whatever the batch),
so both are pure performance choices: small tiles shorten each tile's list but multiply the tile
pairs to sort, large tiles do the opposite; a larger batch takes fewer staging rounds but stops
later once a warp's pixels are saturated.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import train as T

TILES = [(16, 16), (16, 8), (32, 16), (32, 8), (8, 8)]
BATCHES = [32, 16, 64]


def tune(params: torch.Tensor, n: int, sizes, cams: torch.Tensor, target: torch.Tensor, steps: int = 3,
         tiles=TILES, batches=BATCHES, log=None, dssim: float = 0.0):
    """Time `steps` eager training steps per (tile shape, batch) on copies of the parameters;
    returns (best (tile, batch), {(tile, batch): ms per step})."""
    res = {}
    for tile in tiles:
        for batch in batches:
            p = params.clone()
            st = T.TrainStep(p, n, 0, 0, sizes, steps=1000, loss_kind=L.LOSS_L1, tile=tile, dssim=dssim,
                             batch=batch)
            st.cams.copy_(cams)
            st.target.copy_(target)
            st.rast.forward(p, st.cams, check_capacity=True)
            st.rast._alloc_bins(int(1.5 * int(st.rast.n_inst.item())) + 65536)
            st.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                st.run()
            e1.record()
            torch.cuda.synchronize()
            res[(tile, batch)] = e0.elapsed_time(e1) / steps
            if log:
                log(f"tile {tile} batch {batch}: {res[(tile, batch)]:.3f} ms/step")
            del st, p
            torch.cuda.empty_cache()
    best = min(res, key=res.get)
    return best, res
