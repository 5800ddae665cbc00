"""Fidelity loss (1 - lambda) L1 + lambda D-SSIM (Eq. 2 without the mask term, Eq. 3), FP64.

Test infrastructure (see oracle/__init__.py).

Readings: SSIM uses an 11x11 Gaussian window with sigma = 1.5 normalised to sum 1,
zero padding, C1 = 0.01^2, C2 = 0.03^2 (the standard SSIM constants for [0,1] images);
D-SSIM = 1 - SSIM; both L1 and SSIM are means over pixels and channels of one camera and
the camera losses are averaged. lambda = 0.2 for the batched workloads.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

from .gaussians import DT

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
WINDOW = 11
SIGMA = 1.5


def gaussian_window(size=WINDOW, sigma=SIGMA):
    """Separable 1-D Gaussian taps g (sum 1); the 2-D window is outer(g, g)."""
    x = torch.arange(size, dtype=DT) - (size - 1) / 2.0
    g = torch.exp(-(x * x) / (2.0 * sigma * sigma))
    return g / g.sum()


def _filter(img):
    """Zero-padded 'same' correlation of each channel of img [3,H,W] with the 11x11 window."""
    g = gaussian_window()
    w2 = torch.outer(g, g)[None, None].expand(img.shape[0], 1, WINDOW, WINDOW)
    return F.conv2d(img[None], w2, padding=WINDOW // 2, groups=img.shape[0])[0]


def window_moments(y):
    """The window statistics of one image that SSIM needs from it alone: (w * y, w * y^2)."""
    return _filter(y), _filter(y * y)


def ssim_map(x, y):
    """Per-pixel, per-channel SSIM of images x, y [3,H,W]."""
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    num = (2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)
    den = (mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2)
    return num / den


def ssim_direct(x, y):
    """SSIM map by direct double loops over the window (slow; pins `ssim_map` on tiny images)."""
    g = gaussian_window().tolist()
    C, H, W = x.shape
    h = WINDOW // 2
    out = torch.zeros_like(x)
    xs, ys = x.tolist(), y.tolist()
    for c in range(C):
        for i in range(H):
            for j in range(W):
                mx = my = xx = yy = xy = 0.0
                for a in range(-h, h + 1):
                    for b in range(-h, h + 1):
                        ii, jj = i + a, j + b
                        if 0 <= ii < H and 0 <= jj < W:
                            w = g[a + h] * g[b + h]
                            p, q = xs[c][ii][jj], ys[c][ii][jj]
                            mx += w * p
                            my += w * q
                            xx += w * p * p
                            yy += w * q * q
                            xy += w * p * q
                sx, sy, s = xx - mx * mx, yy - my * my, xy - mx * my
                out[c, i, j] = ((2 * mx * my + SSIM_C1) * (2 * s + SSIM_C2)) / (
                    (mx * mx + my * my + SSIM_C1) * (sx + sy + SSIM_C2))
    return out


def l1(x, y):
    return torch.mean(torch.abs(x - y))


def fidelity_loss(images, targets, lam):
    """L = mean_c[(1 - lam) L1_c + lam (1 - SSIM_c)] over cameras (Eq. 3)."""
    terms = []
    for x, y in zip(images, targets):
        t = (1.0 - lam) * l1(x, y)
        if lam != 0.0:
            t = t + lam * (1.0 - torch.mean(ssim_map(x, y)))
        terms.append(t)
    return torch.stack(terms).mean()


def loss_and_image_grad(images, targets, lam):
    """Loss value and dL/d(image) for each camera, by autograd of `fidelity_loss`."""
    xs = [torch.as_tensor(x, dtype=DT).detach().clone().requires_grad_(True) for x in images]
    ys = [torch.as_tensor(y, dtype=DT) for y in targets]
    loss = fidelity_loss(xs, ys, lam)
    loss.backward()
    return float(loss.detach()), [x.grad.detach() for x in xs]


def constant_shift_ssim(a, b):
    """Closed-form SSIM of two constant images a, b away from the borders: (2ab + C1)/(a^2 + b^2 + C1)."""
    return (2 * a * b + SSIM_C1) / (a * a + b * b + SSIM_C1)


__all__ = ["gaussian_window", "ssim_map", "ssim_direct", "l1", "fidelity_loss", "loss_and_image_grad",
           "constant_shift_ssim", "SSIM_C1", "SSIM_C2", "math"]
