"""Brute-force tile binning and (tile, depth, index) ordering (NumPy, FP64).

Test infrastructure (see oracle/__init__.py).

The paper names tile-based rasterisation (Sec. 1, Sec. 4.2) without describing it; the
ordering it must produce is fixed by the compositing definition (App. A.1): within each tile,
Gaussians in ascending depth, ties by index. Reading of the binning rule: a visible record
(radius > 0) with centre (u, v), conic (a, b, c) and opacity o is listed in a B x B tile iff its
footprint ellipse {d : a dx^2 + 2 b dx dy + c dy^2 <= k2}, k2 = 2 ln(255 o) + 0.01, reaches a
pixel centre of the tile (pixel centres of tile (tx, ty) span [tx B, tx B + B - 1] x
[ty B, ty B + B - 1]). Every pixel whose alpha = o exp(-q/2) is >= 1/255 has q <= 2 ln(255 o)
and lies inside the ellipse, so listing exactly these tiles loses nothing.

The decision compares floating-point values with a threshold; the kernel decides in float32,
this brute force in float64. Decisions whose minimum of q over the tile lies within a relative
1e-4 of k2 are reported as ambiguous: both outcomes are correct there.
"""
from __future__ import annotations

import math

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


def rect_min_quadratic(a, b, c, x0, x1, y0, y1):
    """min over [x0,x1] x [y0,y1] of a x^2 + 2 b x y + c y^2 (positive definite), by brute
    geometry: 0 if the origin is inside, else the smallest of the 1-D minima on the four edges."""
    if x0 <= 0 <= x1 and y0 <= 0 <= y1:
        return 0.0
    best = math.inf
    for X in (x0, x1):
        y = min(max(-b * X / c, y0), y1)
        best = min(best, a * X * X + 2 * b * X * y + c * y * y)
    for Y in (y0, y1):
        x = min(max(-b * Y / a, x0), x1)
        best = min(best, a * x * x + 2 * b * x * Y + c * Y * Y)
    return best


def footprint_tiles(u, v, conic, opacity, tiles_x, tiles_y, tile, amb_rel=1e-4):
    """(sure, ambiguous) lists of (tx, ty) tiles reached by the footprint ellipse."""
    a, b, c = (float(x) for x in conic)
    o = float(opacity)
    det = a * c - b * b
    if not (255.0 * o > 1.0) or det <= 0:
        return [], []
    k2 = 2.0 * math.log(255.0 * o) + 0.01
    ex = math.sqrt(k2 * c / det) * (1 + 1e-5) + 1e-3
    ey = math.sqrt(k2 * a / det) * (1 + 1e-5) + 1e-3
    sure, amb = [], []
    for ty in range(max(0, math.floor((v - ey) / tile)), min(tiles_y - 1, math.floor((v + ey) / tile)) + 1):
        for tx in range(max(0, math.floor((u - ex) / tile)), min(tiles_x - 1, math.floor((u + ex) / tile)) + 1):
            q = rect_min_quadratic(a, b, c, tx * tile - u, tx * tile + tile - 1 - u,
                                   ty * tile - v, ty * tile + tile - 1 - v)
            if abs(q - k2) <= amb_rel * k2:
                amb.append((tx, ty))
            elif q < k2:
                sure.append((tx, ty))
    return sure, amb


def bin_records(u, v, conic, opacity, radius, rec_cam, cams, tile):
    """Per global tile: the records surely listed and the records that may be listed.

    Returns (sure: dict tile -> set(rec), maybe: dict tile -> set(rec), total_tiles)."""
    layout, total = tile_layout(cams, tile)
    sure, maybe = {}, {}
    for rec in range(len(u)):
        if radius[rec] <= 0:
            continue
        tx_n, ty_n, base = layout[int(rec_cam[rec])]
        s, a = footprint_tiles(float(u[rec]), float(v[rec]), conic[rec], opacity[rec], tx_n, ty_n, tile)
        for tx, ty in s:
            sure.setdefault(base + ty * tx_n + tx, set()).add(rec)
        for tx, ty in a:
            maybe.setdefault(base + ty * tx_n + tx, set()).add(rec)
    return sure, maybe, total


def order_key(depth, rec):
    """Sort key within a tile: (depth as float32 bit pattern, record index)."""
    return (int(np.asarray(depth, dtype=np.float32).view(np.uint32)), int(rec))
