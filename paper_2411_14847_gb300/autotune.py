"""Autotuner for the compositing launch shape: tile side x Gaussians staged per batch.

Times a few graph-replayed shift-stage iterations for each candidate (tile, batch) pair on
the caller's workload and returns the fastest. Results are identical across candidates by
construction (the per-pixel sequence of blended Gaussians does not depend on the tiling),
so the choice only affects speed.
"""
from __future__ import annotations

import torch

from . import dass as D
from .timestep import ShiftStage

CANDIDATES = [(t, b) for t in (8, 16, 32) for b in (32, 64, 128, 256)]


def autotune(g, cams, targets, dyn_idx, offsets, candidates=CANDIDATES, iters=4, lambda_dssim=0.2):
    table = {}
    for tile, batch in candidates:
        st = ShiftStage(g, cams, targets, dyn_idx, offsets.clone(), tile=tile, batch=batch,
                        lambda_dssim=lambda_dssim, stats=True)
        st.run(1)                      # warm-up (graph instantiation, caches)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st.stream)
        st.run(iters)
        e1.record(st.stream)
        torch.cuda.synchronize()
        table[f"{tile}x{batch}"] = e0.elapsed_time(e1) / iters
        del st
    best = min(table, key=table.get)
    tile, batch = (int(x) for x in best.split("x"))
    return (tile, batch), table
