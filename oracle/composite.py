"""Untiled per-pixel front-to-back alpha compositing (FP64).

Test infrastructure (see oracle/__init__.py).

Definition (App. A.1, the blending equation C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j)),
with the readings used throughout this project:
  * order: the i-th *nearest* Gaussian (ascending camera depth, ties by index) -- the
    appendix's "i-th greatest depth" is read as a slip, since front-to-back blending with
    a product of (1 - alpha_j) over the preceding terms needs the nearest first;
  * alpha_i(x) = min(0.99, o_i exp(-1/2 d^T conic_i d)), d = x - mean2D_i, pixel centres
    at integer coordinates;
  * a Gaussian with alpha_i < 1/255 is skipped;
  * before adding Gaussian i, if T (1 - alpha_i) < 1e-4 the pixel stops and i is not added;
  * C = sum of added c_i alpha_i T_i + T_final * bg.
No tiles, no sort keys, no early exit beyond the definition's own stop rule.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .gaussians import DT

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_STOP = 1e-4


def depth_order(proj):
    """Indices of valid Gaussians sorted by (depth ascending, index ascending)."""
    idx = torch.nonzero(proj["valid"], as_tuple=False).flatten()
    d = proj["depth"].detach()[idx]
    o = torch.sort(d, stable=True).indices
    return idx[o]


def _ordered(proj, order):
    return (proj["mean2d"][order], proj["conic"][order], proj["opacity"][order], proj["rgb"][order])


def alpha_matrix(mean2d, conic, opacity, px, py):
    """alpha[p, i] = min(0.99, o_i exp(-1/2 d^T conic_i d)) for pixel p = (px, py)."""
    dx = px[:, None] - mean2d[None, :, 0]
    dy = py[:, None] - mean2d[None, :, 1]
    power = -0.5 * (conic[None, :, 0] * dx * dx + conic[None, :, 2] * dy * dy) - conic[None, :, 1] * dx * dy
    return torch.clamp_max(opacity[None, :] * torch.exp(power), ALPHA_MAX)


def composite_pixels(proj, px, py, bg=None, order=None, chunk=None, want_flags=False,
                     eps_alpha=1e-3, eps_t=1e-3):
    """Composite the given pixels. px, py: float64 [P] pixel-centre coordinates.

    Returns dict(color [P,3], T_final [P], n_last [P] (Gaussian index of the last added
    Gaussian, -1 if none), n_contrib [P]) and, if want_flags, `flagged` [P] marking pixels
    where a skip or stop decision lies within a relative eps of its threshold (FP32 and FP64
    may legitimately take either branch there).
    """
    if order is None:
        order = depth_order(proj)
    mean2d, conic, opac, rgb = _ordered(proj, order)
    P = px.shape[0]
    n = order.shape[0]
    if chunk is None:
        chunk = max(1, min(P, (1 << 22) // max(1, n)))
    bgv = torch.zeros(3, dtype=DT) if bg is None else torch.as_tensor(bg, dtype=DT)
    colors, tfin, nlast, ncon, flags = [], [], [], [], []
    for s in range(0, P, chunk):
        cx = px[s:s + chunk]
        cy = py[s:s + chunk]
        if n == 0:
            m = cx.shape[0]
            colors.append(bgv.expand(m, 3).clone())
            tfin.append(torch.ones(m, dtype=DT))
            nlast.append(torch.full((m,), -1, dtype=torch.long))
            ncon.append(torch.zeros(m, dtype=torch.long))
            flags.append(torch.zeros(m, dtype=torch.bool))
            continue
        alpha = alpha_matrix(mean2d, conic, opac, cx, cy)
        with torch.no_grad():
            a = alpha.detach()
            keep = a >= ALPHA_MIN
            a_eff = torch.where(keep, a, torch.zeros_like(a))
            t_after = torch.cumprod(1.0 - a_eff, dim=1)
            stop = t_after < T_STOP            # monotone: the first True is the excluded Gaussian
            included = keep & ~stop
            if want_flags:
                t_before = torch.cat([torch.ones_like(t_after[:, :1]), t_after[:, :-1]], dim=1)
                first_stop = torch.where(stop.any(1), stop.float().argmax(1), torch.full((a.shape[0],), n))
                upto = torch.arange(n)[None, :] <= first_stop[:, None]
                near_a = (torch.abs(a * 255.0 - 1.0) < eps_alpha) & upto
                near_t = keep & upto & (torch.abs(t_before * (1.0 - a) * 1e4 - 1.0) < eps_t)
                flags.append((near_a | near_t).any(1))
        a_inc = torch.where(included, alpha, torch.zeros_like(alpha))
        one_minus = 1.0 - a_inc
        t_cum = torch.cumprod(one_minus, dim=1)
        t_before = torch.cat([torch.ones_like(t_cum[:, :1]), t_cum[:, :-1]], dim=1)
        w = a_inc * t_before
        t_final = t_cum[:, -1]
        col = w @ rgb + t_final[:, None] * bgv[None, :]
        colors.append(col)
        tfin.append(t_final)
        with torch.no_grad():
            cnt = included.sum(1)
            last_pos = torch.where(cnt > 0, n - 1 - torch.flip(included, [1]).float().argmax(1),
                                   torch.full_like(cnt, -1))
            nl = torch.where(last_pos >= 0, order[last_pos.clamp_min(0)], torch.full_like(cnt, -1))
        nlast.append(nl)
        ncon.append(cnt)
    out = dict(color=torch.cat(colors), T_final=torch.cat(tfin), n_last=torch.cat(nlast),
               n_contrib=torch.cat(ncon))
    if want_flags:
        out["flagged"] = torch.cat(flags)
    return out


def pixel_grid(width, height):
    ys, xs = torch.meshgrid(torch.arange(height, dtype=DT), torch.arange(width, dtype=DT), indexing="ij")
    return xs.reshape(-1), ys.reshape(-1)


def render_image(proj, width, height, bg=None, want_flags=False):
    """Full image [3,H,W] plus T_final/n_last [H,W] (and flags) for one camera."""
    px, py = pixel_grid(width, height)
    r = composite_pixels(proj, px, py, bg=bg, want_flags=want_flags)
    out = dict(image=r["color"].T.reshape(3, height, width), T_final=r["T_final"].reshape(height, width),
               n_last=r["n_last"].reshape(height, width), n_contrib=r["n_contrib"].reshape(height, width))
    if want_flags:
        out["flagged"] = r["flagged"].reshape(height, width)
    return out


def pixel_alternatives(proj, x, y, order=None, bg=None, eps_alpha=1e-3, eps_t=1e-3, max_events=3):
    """All colours the definition yields at pixel (x, y) when each decision that sits within
    a relative eps of its threshold (alpha vs 1/255, T(1-alpha) vs 1e-4) may go either way.

    Plain scalar loop (Python floats) over the depth-ordered Gaussians. Returns a list of
    (color tuple, T_final) pairs, or None when more than `max_events` near-threshold
    decisions occur on one path (the pixel is then excluded from comparison and counted).
    """
    if order is None:
        order = depth_order(proj)
    mean2d, conic, opac, rgb = (t.detach().numpy() for t in _ordered(proj, order))
    dx = x - mean2d[:, 0]
    dy = y - mean2d[:, 1]
    power = -0.5 * (conic[:, 0] * dx * dx + conic[:, 2] * dy * dy) - conic[:, 1] * dx * dy
    alpha = np.minimum(ALPHA_MAX, opac * np.exp(power))
    cand = np.nonzero(alpha >= ALPHA_MIN * (1.0 - 2 * eps_alpha))[0]
    bgv = (0.0, 0.0, 0.0) if bg is None else tuple(float(b) for b in bg)
    results = []

    def run(pos, T, col, events):
        while pos < len(cand):
            i = cand[pos]
            a = float(alpha[i])
            options = [a >= ALPHA_MIN]
            if abs(a * 255.0 - 1.0) < eps_alpha:
                options = [True, False]
            if len(options) == 2:
                if events >= max_events:
                    raise OverflowError
                for take in options:
                    if take:
                        _step_take(pos, i, a, T, col, events + 1)
                    else:
                        run(pos + 1, T, col, events + 1)
                return
            if not options[0]:
                pos += 1
                continue
            _step_take(pos, i, a, T, col, events)
            return
        results.append((tuple(col[c] + T * bgv[c] for c in range(3)), T))

    def _step_take(pos, i, a, T, col, events):
        test = T * (1.0 - a)
        stops = [test < T_STOP]
        if abs(test * 1e4 - 1.0) < eps_t:
            if events >= max_events:
                raise OverflowError
            stops = [True, False]
            events += 1
        for st in stops:
            if st:
                results.append((tuple(col[c] + T * bgv[c] for c in range(3)), T))
            else:
                ncol = [col[c] + float(rgb[i, c]) * a * T for c in range(3)]
                run(pos + 1, test, ncol, events)

    try:
        run(0, 1.0, [0.0, 0.0, 0.0], 0)
    except OverflowError:
        return None
    return results


def composite_reference_loop(proj, x, y, bg=None):
    """Straight scalar loop over *all* Gaussians in depth order at one pixel (no vectorisation).

    Used only to pin the vectorised `composite_pixels` on tiny scenes.
    """
    order = depth_order(proj)
    m = proj["mean2d"].detach().numpy()
    cn = proj["conic"].detach().numpy()
    op = proj["opacity"].detach().numpy()
    rgb = proj["rgb"].detach().numpy()
    T = 1.0
    col = [0.0, 0.0, 0.0]
    last = -1
    for i in order.tolist():
        dx = x - m[i, 0]
        dy = y - m[i, 1]
        pw = -0.5 * (cn[i, 0] * dx * dx + cn[i, 2] * dy * dy) - cn[i, 1] * dx * dy
        a = min(ALPHA_MAX, op[i] * math.exp(pw))
        if a < ALPHA_MIN:
            continue
        if T * (1.0 - a) < T_STOP:
            break
        for c in range(3):
            col[c] += rgb[i, c] * a * T
        T *= 1.0 - a
        last = i
    bgv = (0.0, 0.0, 0.0) if bg is None else bg
    return [col[c] + T * bgv[c] for c in range(3)], T, last
