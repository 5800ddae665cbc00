"""End-to-end forward and gradients of the per-timestep render loss (FP64, autograd).

Test infrastructure (see oracle/__init__.py).

Chain (App. A.1 + Sec. 3.2/3.3): parameters -> [selective-inheritance mask, Eq. 1] ->
[dynamics-aware shift of the dynamic rows, Sec. 3.3] -> activations -> EWA projection per
camera -> untiled per-pixel compositing -> images -> fidelity loss (Eq. 3).
Gradients are the exact derivatives of this definition by reverse-mode autodiff that
stores every alpha (no recomputation from T_final, unlike the CUDA backward).
"""
from __future__ import annotations

import numpy as np
import torch

from . import composite as comp
from .gaussians import DT, activate, footprint_radius, project, t64
from .loss import loss_and_image_grad
from .stages import shift

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _leaves(arrays, offsets):
    leaves = {k: t64(np.asarray(arrays[k], dtype=np.float64)).clone().requires_grad_(True) for k in PARAMS}
    off = None
    if offsets is not None:
        off = t64(np.asarray(offsets, dtype=np.float64)).clone().requires_grad_(True)
    return leaves, off


def _render_inputs(leaves, off, dyn_idx, keep):
    means, quats = leaves["means"], leaves["quats"]
    if off is not None:
        means, quats = shift(means, quats, dyn_idx, off)
    s, qn, o = activate(leaves["log_scales"], quats, leaves["opacity_logit"], keep=keep)
    return means, s, qn, o


def project_all(arrays, cams, sh_degree, dyn_idx=None, offsets=None, keep=None):
    """Projection dicts for every camera (no gradients)."""
    with torch.no_grad():
        leaves, off = _leaves(arrays, offsets)
        means, s, qn, o = _render_inputs(leaves, off, dyn_idx, keep)
        return [project(means, s, qn, o, leaves["sh"], sh_degree, cam) for cam in cams]


def render(arrays, cams, sh_degree, dyn_idx=None, offsets=None, keep=None, bg=None, want_flags=False):
    """Rendered images [3,H,W] (+ T_final, n_last, flags) for every camera."""
    projs = project_all(arrays, cams, sh_degree, dyn_idx, offsets, keep)
    with torch.no_grad():
        return [comp.render_image(p, cam.width, cam.height, bg=bg, want_flags=want_flags)
                for p, cam in zip(projs, cams)]


def stats_visible(proj, cam):
    """Visibility of a Gaussian in a view for the positional-gradient statistics: in front of
    the near plane, opacity above 1/255, and the square of half-side equal to the footprint
    radius around mean2D overlapping the image [0, W-1] x [0, H-1]."""
    r = footprint_radius(proj["cov2d"], proj["opacity"])
    u, v = proj["mean2d"][:, 0], proj["mean2d"][:, 1]
    return (proj["valid"] & (r > 0) & (u + r >= 0) & (u - r <= cam.width - 1)
            & (v + r >= 0) & (v - r <= cam.height - 1))


def image_vjp(arrays, cams, sh_degree, pixel_grads, dyn_idx=None, offsets=None, keep=None, bg=None):
    """Gradients of sum_c sum_p <dL/dC_c(p), C_c(p)> w.r.t. all parameters.

    pixel_grads: per camera a tuple (px [P], py [P], g [P,3]) of pixel-centre coordinates and
    upstream gradients (any subset of pixels). Returns dict with gradients for means,
    log_scales, quats, opacity_logit, sh (and offsets when given), plus per camera
    dmean2d [N,2] (dL/d mean2D) and visible [N].
    """
    leaves, off = _leaves(arrays, offsets)
    means, s, qn, o = _render_inputs(leaves, off, dyn_idx, keep)
    outs, grads_in, dmean2d, visible = [], [], [], []
    for cam, (px, py, g) in zip(cams, pixel_grads):
        proj = project(means, s, qn, o, leaves["sh"], sh_degree, cam)
        lv = {k: proj[k].detach().clone().requires_grad_(True) for k in ("mean2d", "conic", "opacity", "rgb")}
        lproj = dict(lv, depth=proj["depth"].detach(), valid=proj["valid"])
        order = comp.depth_order(lproj)
        px = t64(px)
        py = t64(py)
        g = t64(g)
        n = order.shape[0]
        chunk = max(1, min(px.shape[0], (1 << 21) // max(1, n)))
        for st in range(0, px.shape[0], chunk):
            r = comp.composite_pixels(lproj, px[st:st + chunk], py[st:st + chunk], bg=bg, order=order,
                                      chunk=chunk)
            (r["color"] * g[st:st + chunk]).sum().backward()
        for k in ("mean2d", "conic", "opacity", "rgb"):
            if lv[k].grad is None:
                lv[k].grad = torch.zeros_like(lv[k])
            outs.append(proj[k])
            grads_in.append(lv[k].grad)
        dmean2d.append(lv["mean2d"].grad.detach().clone())
        with torch.no_grad():
            visible.append(stats_visible(proj, cam))
    torch.autograd.backward(outs, grads_in)
    res = {k: (leaves[k].grad if leaves[k].grad is not None else torch.zeros_like(leaves[k])).detach()
           for k in PARAMS}
    if off is not None:
        res["offsets"] = off.grad.detach() if off.grad is not None else torch.zeros_like(off)
    res["dmean2d"] = dmean2d
    res["visible"] = visible
    return res


def loss_grads(arrays, cams, sh_degree, targets, lam, dyn_idx=None, offsets=None, keep=None, bg=None):
    """Loss (Eq. 3), rendered images, and all parameter gradients for full images."""
    imgs = render(arrays, cams, sh_degree, dyn_idx, offsets, keep, bg)
    images = [r["image"] for r in imgs]
    loss, dimg = loss_and_image_grad(images, [t64(t) for t in targets], lam)
    pg = []
    for cam, gi in zip(cams, dimg):
        px, py = comp.pixel_grid(cam.width, cam.height)
        pg.append((px, py, gi.reshape(3, -1).T))
    res = image_vjp(arrays, cams, sh_degree, pg, dyn_idx, offsets, keep, bg)
    res["loss"] = loss
    res["images"] = images
    res["dimages"] = dimg
    return res


# ------------------------------------------------------------ Sec. 3.2: learned inheritance mask

def ste_keep(m, is_var):
    """Rendering mask of Eq. 1 under the straight-through estimator of App. B.2.

    On var rows m_op = detach(Quant(sigmoid(m)) - sigmoid(m)) + sigmoid(m): its value is
    Quant(sigmoid(m)) (read as [sigmoid(m) > 1/2], i.e. m > 0) and its derivative is that of
    sigmoid(m). Base rows are always rendered (mask 1)."""
    m = t64(m)
    sg = torch.sigmoid(m)
    q = (m > 0).to(DT)
    m_op = (q - sg).detach() + sg
    isv = torch.as_tensor(np.asarray(is_var, dtype=bool))
    return torch.where(isv, m_op, torch.ones_like(m_op))


def inherit_mask_grads(arrays, cams, sh_degree, targets, lam, m, is_var, lam_inher, bg=None):
    """Loss of Eq. 2 and its gradients for the selective-inheritance stage (Sec. 3.2, App. B.2).

    L = (1 - lam) L1 + lam D-SSIM (Eq. 3 over all cameras) + lam_inher * sum_var sigmoid(m).
    The render uses o_r = m_op o and s_r = m_op s (Eq. 1) with m_op from ste_keep. Returns
    loss, d_keep (dL_fidelity/d(mask value) per Gaussian, the derivative of the fidelity loss
    w.r.t. the multiplier of Eq. 1 at its current value) and dm (dL/dm through the STE,
    mask loss included; 0 on base rows)."""
    m_leaf = t64(np.asarray(m, dtype=np.float64)).clone().requires_grad_(True)
    keep = ste_keep(m_leaf, is_var)
    keep.retain_grad()
    imgs = render(arrays, cams, sh_degree, keep=keep.detach(), bg=bg)
    images = [r["image"] for r in imgs]
    fid, dimg = loss_and_image_grad(images, [t64(t) for t in targets], lam)
    pg = []
    for cam, gi in zip(cams, dimg):
        px, py = comp.pixel_grid(cam.width, cam.height)
        pg.append((px, py, gi.reshape(3, -1).T))
    image_vjp(arrays, cams, sh_degree, pg, keep=keep, bg=bg)
    d_keep = keep.grad.detach().clone() if keep.grad is not None else torch.zeros_like(keep)
    isv = torch.as_tensor(np.asarray(is_var, dtype=bool))
    reg = lam_inher * torch.sigmoid(m_leaf[isv]).sum()
    reg.backward()
    dm = m_leaf.grad.detach().clone()
    return {"loss": float(fid) + float(reg.detach()), "fidelity": float(fid), "d_keep": d_keep, "dm": dm,
            "images": images}
