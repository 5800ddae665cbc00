"""Per-Gaussian work of the three DASS stages, FP64 (NumPy / torch CPU).

Test infrastructure (see oracle/__init__.py). References are to arXiv 2411.14847.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .gaussians import DT, alg1_full_projection, quat_mul, quat_to_rotmat, t64


# ------------------------------------------------------------ Sec. 3.3: shift

def shift(means, quats, dyn_idx, offsets):
    """Dynamics-aware shift (Sec. 3.3) applied to the dynamic rows only.

    For each dynamic Gaussian n with offsets (dmu_n, sigma_n):
      p_n' = p_n + dmu_n,   q_n' = norm(q_n) x norm(sigma_n)   (Hamilton product, q on the left).
    Static rows are returned unchanged (their deformation field H_st is outside this path).
    offsets: [N_dyn, 7] = (dmu[3], sigma[4]). Differentiable w.r.t. offsets (and inputs).
    """
    means = t64(means)
    quats = t64(quats)
    offsets = t64(offsets)
    idx = torch.as_tensor(np.asarray(dyn_idx), dtype=torch.long)
    out_m = means.clone()
    out_q = quats.clone()
    if idx.numel() == 0:
        return out_m, out_q
    qn = quats[idx] / torch.linalg.norm(quats[idx], dim=-1, keepdim=True)
    sg = offsets[:, 3:7]
    sn = sg / torch.linalg.norm(sg, dim=-1, keepdim=True)
    out_m = out_m.index_put((idx,), means[idx] + offsets[:, 0:3])
    out_q = out_q.index_put((idx,), quat_mul(qn, sn))
    return out_m, out_q


# ------------------------------------------------------ Sec. 3.2: inheritance

def quant_keep(m):
    """Quant(sigmoid(m)) of Eq. 1 read as 1 iff sigmoid(m) > 0.5, i.e. m > 0 (m = 0 -> 0)."""
    return (np.asarray(m, dtype=np.float64) > 0.0)


def inherit(arrays: dict, is_var, m, t, erase_every=20):
    """Selective inheritance copy (Sec. 3.2, App. B.2).

    G_t starts from every base Gaussian of G_{t-1} (original order) followed by the var
    Gaussians whose quantised mask Quant(sigmoid(m)) is 1 (original order). Every
    `erase_every` timesteps (t % 20 == 0) no var Gaussian is inherited.
    Returns (new arrays, new is_var, old->new index map with -1 for dropped rows).
    `m` is indexed like the rows (entries of base rows are ignored).
    """
    is_var = np.asarray(is_var).astype(bool)
    keep_var = quant_keep(m) & is_var
    if t % erase_every == 0:
        keep_var[:] = False
    base_rows = np.nonzero(~is_var)[0]
    var_rows = np.nonzero(keep_var)[0]
    rows = np.concatenate([base_rows, var_rows])
    remap = np.full(is_var.shape[0], -1, dtype=np.int64)
    remap[rows] = np.arange(rows.shape[0])
    out = {k: np.asarray(v)[rows].copy() for k, v in arrays.items()}
    new_var = np.concatenate([np.zeros(base_rows.shape[0], bool), np.ones(var_rows.shape[0], bool)])
    return out, new_var, remap


def prune_low_opacity(arrays: dict, is_var, min_opacity):
    """Low-opacity pruning of the densification stage (Sec. 3.4): every base row is kept, a var row
    only if its opacity sigmoid(logit) exceeds min_opacity; base rows first, then the kept var rows,
    each group in its original order (the layout of the inheritance copy)."""
    is_var = np.asarray(is_var, dtype=bool)
    o = 1.0 / (1.0 + np.exp(-np.asarray(arrays["opacity_logit"], dtype=np.float64)))
    keep_var = is_var & (o > min_opacity)
    rows = np.concatenate([np.nonzero(~is_var)[0], np.nonzero(keep_var)[0]])
    out = {k: np.asarray(v)[rows].copy() for k, v in arrays.items()}
    new_var = np.concatenate([np.zeros(int((~is_var).sum()), bool), np.ones(int(keep_var.sum()), bool)])
    return out, new_var


# ------------------------------------------------------------ optimiser

def adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15, rows=None):
    """Adam with bias correction on the selected rows only (rows=None: all rows).

    m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
    p <- p - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
    Rows outside `rows` (params, moments) are returned bit-identical. The paper does not
    name its optimiser (3DGS and 3DGStream use Adam).
    """
    p = np.array(param, dtype=np.float64, copy=True)
    g = np.asarray(grad, dtype=np.float64)
    mm = np.array(m, dtype=np.float64, copy=True)
    vv = np.array(v, dtype=np.float64, copy=True)
    sel = slice(None) if rows is None else np.asarray(rows)
    mm[sel] = beta1 * mm[sel] + (1 - beta1) * g[sel]
    vv[sel] = beta2 * vv[sel] + (1 - beta2) * g[sel] ** 2
    mhat = mm[sel] / (1 - beta1 ** step)
    vhat = vv[sel] / (1 - beta2 ** step)
    p[sel] = p[sel] - lr * mhat / (np.sqrt(vhat) + eps)
    return p, mm, vv


# ------------------------------------------------ Sec. 3.4: error guidance

def error_map_f32(image, target):
    """E^c: per-pixel mean over RGB of |render - ground truth| (Sec. 3.4 'comparing').

    Computed in float32 with the operation order ((|dr| + |dg|) + |db|) / 3 because E decides
    the integer bitmap D_err; the CUDA path takes the same decision in the same precision.
    image, target: [3,H,W]. Returns float32 [H,W].
    """
    a = np.asarray(image, dtype=np.float32)
    b = np.asarray(target, dtype=np.float32)
    d = np.abs(a - b)
    return ((d[0] + d[1]) + d[2]) / np.float32(3.0)


def percentile_lower(e, q=0.95):
    """gamma_err: the nearest-rank lower q-quantile, element floor(q (P-1)) of the ascending sort."""
    flat = np.sort(np.asarray(e).reshape(-1), kind="stable")
    k = int(math.floor(q * (flat.shape[0] - 1)))
    return flat[k]


def error_bitmap(e, gamma):
    """D_err^c = 1[e > gamma] (strict)."""
    return np.asarray(e) > gamma


def alg1_pixels(means, cam):
    """Alg. 1: P_hom = [P, 1] T; x_norm = p_x / p_hom, y_norm = p_y / p_hom;
    x_n = Round(0.5((x_norm + 1) W - 1)), y_n = Round(0.5((y_norm + 1) H - 1)).

    Readings: the second line of Alg. 1 uses x_norm for y_n, read as y_norm with H; Round is
    floor(v + 0.5); x is the column (W axis) and y the row (H axis). Returns float64 arrays
    (x_cont, y_cont, p_hom) with the continuous pixel coordinates before rounding.
    """
    T = alg1_full_projection(cam)
    P = np.asarray(means, dtype=np.float64)
    ph = np.concatenate([P, np.ones((P.shape[0], 1))], axis=1) @ T
    with np.errstate(divide="ignore", invalid="ignore"):
        xn = ph[:, 0] / ph[:, 3]
        yn = ph[:, 1] / ph[:, 3]
    xc = 0.5 * ((xn + 1.0) * cam.width - 1.0)
    yc = 0.5 * ((yn + 1.0) * cam.height - 1.0)
    return xc, yc, ph[:, 3]


def error_subset(means, cams, bitmaps, tie_eps=1e-4):
    """S_err = union over views of {n : D_err^c(x_n, y_n) = 1} (Sec. 3.4).

    A Gaussian with p_hom <= 0 or a pixel outside the image is in no S_err^c.
    Returns (s_err bool [N], ambiguous bool [N]); `ambiguous` marks Gaussians whose
    continuous coordinate lies within tie_eps of a rounding boundary in some view
    (FP32 and FP64 may then pick neighbouring pixels; both are correct).
    """
    n = np.asarray(means).shape[0]
    s = np.zeros(n, bool)
    amb = np.zeros(n, bool)
    for cam, D in zip(cams, bitmaps):
        xc, yc, w = alg1_pixels(means, cam)
        ok = w > 0
        with np.errstate(invalid="ignore"):
            xi = np.floor(xc + 0.5)
            yi = np.floor(yc + 0.5)
            near = (np.abs(xc + 0.5 - np.round(xc + 0.5)) < tie_eps) | (np.abs(yc + 0.5 - np.round(yc + 0.5)) < tie_eps)
        inside = ok & (xi >= 0) & (xi < cam.width) & (yi >= 0) & (yi < cam.height)
        hit = np.zeros(n, bool)
        ii = np.nonzero(inside)[0]
        hit[ii] = D[yi[ii].astype(np.int64), xi[ii].astype(np.int64)]
        s |= hit
        amb |= ok & near
    return s, amb


def mean_grad_f32(accum, count):
    """Average view-space positional gradient, float32 division (decides the selection)."""
    a = np.asarray(accum, dtype=np.float32)
    c = np.asarray(count, dtype=np.int64)
    out = np.zeros_like(a)
    nz = c > 0
    out[nz] = a[nz] / c[nz].astype(np.float32)
    return out


def densify_select(grad_mean, s_err, is_base, tau_pos, tau_err, k_max):
    """Eq. 4: S = {n in base : g_n > tau_pos} U (S_err n {n in base : g_n > tau_err}),
    then the at most k_max members with the largest g_n (ties by smaller index).
    Returns the selected indices in ascending index order (the order new rows are appended)."""
    g = np.asarray(grad_mean, dtype=np.float32)
    base = np.asarray(is_base, bool)
    s1 = base & (g > np.float32(tau_pos))
    s2 = np.asarray(s_err, bool) & base & (g > np.float32(tau_err))
    cand = np.nonzero(s1 | s2)[0]
    order = sorted(cand.tolist(), key=lambda n: (-float(g[n]), n))
    return np.asarray(sorted(order[:k_max]), dtype=np.int64)


def spawn(arrays: dict, selected, z, scale_div=1.6):
    """Spawn densification (Sec. 3.4, mechanism not described in the paper; reading):
    one new Gaussian per selected n with mean = mu_n + R_n diag(s_n) z_n, log-scale =
    log(s_n / 1.6); rotation, opacity and SH copied. z: [N_base, 3] standard-normal draws
    indexed by the source Gaussian. Returns the new rows (float64)."""
    sel = np.asarray(selected, dtype=np.int64)
    mu = t64(arrays["means"])[sel]
    ls = t64(arrays["log_scales"])[sel]
    q = t64(arrays["quats"])[sel]
    qn = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    R = quat_to_rotmat(qn)
    s = torch.exp(ls)
    zz = t64(z)[sel]
    new_mu = mu + torch.einsum("nij,nj->ni", R, s * zz)
    out = dict(means=new_mu.numpy(), log_scales=(ls - math.log(scale_div)).numpy(),
               quats=np.asarray(arrays["quats"], np.float64)[sel],
               opacity_logit=np.asarray(arrays["opacity_logit"], np.float64)[sel],
               sh=np.asarray(arrays["sh"], np.float64)[sel])
    return out


def ndc_grad_norm(dmean2d, width, height):
    """|dL/d mean2D_ndc|_2 with dL/du_ndc = dL/du * W/2 and dL/dv_ndc = dL/dv * H/2 (reading of
    the 'view-space positional gradient' of Sec. 3.4)."""
    g = t64(dmean2d)
    return torch.sqrt((g[..., 0] * (width / 2.0)) ** 2 + (g[..., 1] * (height / 2.0)) ** 2)


__all__ = ["shift", "quant_keep", "inherit", "adam", "error_map_f32", "percentile_lower", "error_bitmap",
           "alg1_pixels", "error_subset", "mean_grad_f32", "densify_select", "spawn", "ndc_grad_norm", "DT"]
