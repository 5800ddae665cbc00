"""Identity-feature rendering and the per-Gaussian dynamics query of the shift stage (Sec. 3.3).

Test infrastructure (see oracle/__init__.py). References are to arXiv 2411.14847.

Every Gaussian carries an object-identity feature (Gaussian Grouping); features are rendered
exactly like colours; a linear classifier gives per-pixel object IDs; the IDs found inside the
dynamic image areas (optical flow above a threshold -- an input here) select the dynamic Gaussians:
those whose own feature classifies into one of them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import composite as comp
from .gaussians import t64


def render_features(proj, features, width, height):
    """Per-pixel composited features [H, W, F] (black background): the colour compositing of
    App. A.1 with each Gaussian's colour replaced by its feature vector."""
    f = t64(features)
    F = f.shape[1]
    if proj["mean2d"].shape[0] == 0:
        return torch.zeros((height, width, F), dtype=torch.float64)
    px, py = comp.pixel_grid(width, height)
    r = comp.composite_pixels(dict(proj, rgb=f), px, py, bg=np.zeros(F))
    return r["color"].reshape(height, width, F)


def object_ids(x, W, b):
    """argmax_k (W x + b)_k per row, ties to the lower k."""
    logits = np.asarray(x, dtype=np.float64) @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
    return np.argmax(logits, axis=1)


def dynamic_objects(ids, dyn_area, n_classes, min_pixels):
    """obj_mask[k] = at least min_pixels dynamic-area pixels carry ID k."""
    ids = np.asarray(ids).reshape(-1)
    area = np.asarray(dyn_area).reshape(-1) != 0
    counts = np.bincount(ids[area], minlength=n_classes)
    return counts >= min_pixels


def dynamic_gaussians(features, W, b, obj_mask):
    """Dynamics mask of the Gaussians: their own feature's object ID is a dynamic object."""
    return np.asarray(obj_mask)[object_ids(features, W, b)]
