"""Gaussian primitives, quaternions, real spherical harmonics and EWA projection (FP64).

Test infrastructure (see oracle/__init__.py). References are to arXiv 2411.14847.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64
NEAR = 0.2           # near-plane cull on camera-space depth (reading of App. A.1; 3DGS convention)
LOW_PASS = 0.3       # added to the diagonal of the 2D covariance (EWA anti-aliasing)


def t64(x):
    """Float64 CPU tensor view of an array-like (keeps autograd leaves as they are)."""
    if isinstance(x, torch.Tensor):
        return x if x.dtype == DT else x.to(DT)
    return torch.as_tensor(np.asarray(x), dtype=DT)


# ----------------------------------------------------------------- activations

def activate(log_scales, quats, opacity_logit, keep=None):
    """Rendering-time attributes: s = exp(log s), o = sigmoid(logit), q_hat = q/|q|.

    With an inheritance mask `keep` (0/1 per Gaussian), Eq. 1 multiplies the
    *activated* opacity and scale by Quant(sigmoid(m)): o_r = keep*o, s_r = keep*s.
    """
    s = torch.exp(log_scales)
    o = torch.sigmoid(opacity_logit)
    qn = quats / torch.linalg.norm(quats, dim=-1, keepdim=True)
    if keep is not None:
        keep = t64(keep)
        o = o * keep
        s = s * keep[:, None]
    return s, qn, o


# ----------------------------------------------------------------- quaternions

def quat_mul(a, b):
    """Hamilton product a x b of (w,x,y,z) quaternions (used by the rotation shift, Sec. 3.3)."""
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], dim=-1)


def quat_to_rotmat(q):
    """Rotation matrix R of a unit (w,x,y,z) quaternion (App. A.1: Sigma = R S S^T R^T)."""
    w, x, y, z = q.unbind(-1)
    r = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ], dim=-1)
    return r.reshape(q.shape[:-1] + (3, 3))


def covariance3d(scales, qhat):
    """Sigma = R S S^T R^T with S = diag(s) (App. A.1)."""
    m = quat_to_rotmat(qhat) * scales[..., None, :]
    return m @ m.transpose(-1, -2)


# ----------------------------------------------------------------- real SH

def _legendre_poly(l):
    """Coefficients (ascending powers of z) of the Legendre polynomial P_l via Rodrigues' formula."""
    p = np.polynomial.polynomial
    c = p.polypow([-1.0, 0.0, 1.0], l) if l > 0 else np.array([1.0])   # (z^2 - 1)^l
    for _ in range(l):
        c = p.polyder(c)
    return c / (2.0 ** l * math.factorial(l))


def _sh_terms(degree):
    """For each basis index k = l*l + l + m: (norm constant, d^|m| P_l / dz^|m| coefficients, m)."""
    terms = []
    for l in range(degree + 1):
        pl = _legendre_poly(l)
        for m in range(-l, l + 1):
            am = abs(m)
            dpl = pl.copy()
            for _ in range(am):
                dpl = np.polynomial.polynomial.polyder(dpl)
            k = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m != 0:
                k *= math.sqrt(2.0)
            terms.append((k, dpl, m))
    return terms


def sh_basis(dirs, degree):
    """Real spherical harmonics Y_k(d), k = l^2 + l + m, for unit directions d [...,3].

    Standard real basis without the Condon-Shortley phase:
      Y_l0 = K_l0 P_l(z);  Y_lm = sqrt2 K_lm P_l^m(z) cos(m phi);  Y_l,-m = sqrt2 K_lm P_l^m(z) sin(m phi)
    with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). On the unit sphere
    P_l^m(z) cos/sin(m phi) = (d^m P_l/dz^m)(z) * Re/Im((x + i y)^m), so the basis is a
    polynomial in (x, y, z) and differentiable everywhere. The paper only says "view-
    dependent color" (App. A.1); degree <= 3 SH is the 3DGS colour model.
    """
    x, y, z = dirs.unbind(-1)
    out = []
    # powers of (x + i y): real and imaginary parts
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for _ in range(degree):
        r, i = re[-1], im[-1]
        re.append(r * x - i * y)
        im.append(r * y + i * x)
    for k, dpl, m in _sh_terms(degree):
        poly = torch.zeros_like(z)
        for j in range(len(dpl) - 1, -1, -1):      # Horner in z
            poly = poly * z + float(dpl[j])
        if m > 0:
            ang = re[m]
        elif m < 0:
            ang = im[-m]
        else:
            ang = torch.ones_like(x)
        out.append(k * poly * ang)
    return torch.stack(out, dim=-1)


def sh_to_rgb(sh, dirs, degree):
    """View-dependent colour: rgb = max(sum_k sh[k] Y_k(d) + 0.5, 0) (3DGS colour convention)."""
    basis = sh_basis(dirs, degree)                    # [N,K]
    col = torch.einsum("nk,nkc->nc", basis, sh[:, : basis.shape[-1], :]) + 0.5
    return torch.clamp_min(col, 0.0)


# ----------------------------------------------------------------- camera / projection

def camera_parts(cam):
    vm = t64(np.asarray(cam.viewmat, dtype=np.float64).astype(np.float32).astype(np.float64))
    return vm[:3, :3], vm[:3, 3]


def camera_center(cam):
    r, t = camera_parts(cam)
    return -(r.T @ t)


def f32(v):
    """A camera scalar as the float32 value the CUDA path receives, widened to float64."""
    return float(np.float32(v))


def project(means, scales, qhat, opacity, sh, sh_degree, cam):
    """Per-Gaussian screen-space attributes for one camera (App. A.1).

    X_c = W p + t (world->camera), cull Z <= 0.2;
    Sigma_2D = J W Sigma W^T J^T + 0.3 I with the EWA Jacobian
      J = [[fx/Z, 0, -fx X/Z^2], [0, fy/Z, -fy Y/Z^2]];
    conic = Sigma_2D^{-1}; mean2D = (fx X/Z + cx, fy Y/Z + cy); depth = Z;
    colour from SH along the unit direction camera-centre -> mean.
    Returns a dict of float64 tensors (differentiable w.r.t. the inputs).
    """
    rw, tw = camera_parts(cam)
    fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    xc = means @ rw.T + tw
    X, Y, Z = xc.unbind(-1)
    valid = Z > NEAR
    Zs = torch.where(valid, Z, torch.ones_like(Z))
    n = means.shape[0]
    J = torch.zeros((n, 2, 3), dtype=DT)
    J = torch.stack([
        torch.stack([fx / Zs, torch.zeros_like(Zs), -fx * X / (Zs * Zs)], dim=-1),
        torch.stack([torch.zeros_like(Zs), fy / Zs, -fy * Y / (Zs * Zs)], dim=-1),
    ], dim=-2)
    T = J @ rw
    sig = covariance3d(scales, qhat)
    s2 = T @ sig @ T.transpose(-1, -2)
    a = s2[:, 0, 0] + LOW_PASS
    b = s2[:, 0, 1]
    c = s2[:, 1, 1] + LOW_PASS
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], dim=-1)
    u = fx * X / Zs + cx
    v = fy * Y / Zs + cy
    dirs = means - camera_center(cam)
    dirs = dirs / torch.linalg.norm(dirs, dim=-1, keepdim=True)
    rgb = sh_to_rgb(sh, dirs, sh_degree)
    return dict(mean2d=torch.stack([u, v], dim=-1), conic=conic, cov2d=torch.stack([a, b, c], dim=-1),
                depth=Z, opacity=opacity, rgb=rgb, valid=valid & (det > 0))


def footprint_radius(cov2d_abc, opacity):
    """Opacity-aware pixel radius of the alpha >= 1/255 footprint (reading of the tile rule).

    A pixel at offset d has alpha = o exp(-d^T Sigma^-1 d / 2) >= 1/255 only if
    d^T Sigma^-1 d <= 2 ln(255 o), which lies inside the disc |d| <= sqrt(2 ln(255 o)) sqrt(lambda_max).
    r = ceil(sqrt(lambda_max) * sqrt(2 ln(255 o) + 0.01)); the 0.01 slack covers FP32 rounding
    of alpha at the footprint edge. r = 0 when 255 o <= 1 (never visible).
    """
    a, b, c = cov2d_abc.unbind(-1)
    mid = 0.5 * (a + c)
    lam = mid + torch.sqrt(torch.clamp_min(mid * mid - (a * c - b * b), 0.0))
    vis = 255.0 * opacity > 1.0
    k2 = 2.0 * torch.log(torch.clamp_min(255.0 * opacity, 1.0)) + 0.01
    r = torch.ceil(torch.sqrt(lam) * torch.sqrt(k2))
    return torch.where(vis, r, torch.zeros_like(r))


def alg1_full_projection(cam, znear=0.01, zfar=100.0):
    """Full 4x4 projection T of the pinhole camera for row vectors, [P,1] T = (p_x, p_y, p_z, p_hom).

    Built so that Alg. 1's pixel mapping 0.5((x_norm + 1) W - 1) equals u = fx X/Z + cx:
    x_norm = (2 (fx X/Z + cx) + 1)/W - 1 and p_hom = Z (camera depth). The z row is a
    standard [znear, zfar] depth map; Alg. 1 never uses it.
    """
    W, H = cam.width, cam.height
    fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    K = np.array([
        [2 * fx / W, 0.0, (2 * cx + 1) / W - 1.0, 0.0],
        [0.0, 2 * fy / H, (2 * cy + 1) / H - 1.0, 0.0],
        [0.0, 0.0, (zfar + znear) / (zfar - znear), -2 * zfar * znear / (zfar - znear)],
        [0.0, 0.0, 1.0, 0.0],
    ])
    vm = np.asarray(cam.viewmat, dtype=np.float64).astype(np.float32).astype(np.float64)
    return (K @ vm).T
