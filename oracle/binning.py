"""Brute-force tile binning and (tile, depth, index) ordering, in FP32 (NumPy).

Test infrastructure (see oracle/__init__.py).

The paper names tile-based rasterisation (Sec. 1, Sec. 4.2) without describing it; the
ordering it must produce is fixed by the compositing definition: within each tile,
Gaussians in ascending depth, ties by index. The tile rectangle of a projected Gaussian
with centre (u, v) and pixel radius r on a B x B tiling is
  x in [max(0, floor((u - r)/B)), min(tiles_x - 1, floor((u + r)/B))]   (same for y),
evaluated in float32 because it decides integers that the CUDA path decides in float32.
This is the one place where the oracle works in the kernel's precision.
"""
from __future__ import annotations

import numpy as np


def tile_layout(cams, tile):
    """Per camera (tiles_x, tiles_y, first global tile id); tiles of camera c follow camera c-1."""
    out = []
    base = 0
    for cam in cams:
        tx = (cam.width + tile - 1) // tile
        ty = (cam.height + tile - 1) // tile
        out.append((tx, ty, base))
        base += tx * ty
    return out, base


def tile_rect(u, v, r, tiles_x, tiles_y, tile):
    f = np.float32
    u, v, rr = f(u), f(v), f(r)
    B = f(tile)
    x0 = max(0, int(np.floor((u - rr) / B)))
    x1 = min(tiles_x - 1, int(np.floor((u + rr) / B)))
    y0 = max(0, int(np.floor((v - rr) / B)))
    y1 = min(tiles_y - 1, int(np.floor((v + rr) / B)))
    return x0, x1, y0, y1


def bin_and_sort(u, v, radius, depth, rec_cam, cams, tile):
    """All (global tile, depth bits, record) triples, sorted lexicographically.

    u, v, depth: float32 [R]; radius: int [R] (0 = not visible); rec_cam: camera of each
    record. Returns (sorted record ids [M], sorted tile ids [M], ranges [T_total, 2]).
    """
    layout, total = tile_layout(cams, tile)
    triples = []
    depth_bits = np.asarray(depth, dtype=np.float32).view(np.uint32)
    for rec in range(len(u)):
        if radius[rec] <= 0:
            continue
        tx, ty, base = layout[int(rec_cam[rec])]
        x0, x1, y0, y1 = tile_rect(u[rec], v[rec], radius[rec], tx, ty, tile)
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                triples.append((base + y * tx + x, int(depth_bits[rec]), rec))
    triples.sort()
    recs = np.array([t[2] for t in triples], dtype=np.int64)
    tiles = np.array([t[0] for t in triples], dtype=np.int64)
    ranges = np.zeros((total, 2), dtype=np.int64)
    for i, t in enumerate(tiles.tolist()):
        if i == 0 or tiles[i - 1] != t:
            ranges[t, 0] = i
        if i == len(tiles) - 1 or tiles[i + 1] != t:
            ranges[t, 1] = i + 1
    return recs, tiles, ranges
