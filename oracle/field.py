"""Hash-encoding deformation field of the dynamics-aware shift, FP64 (torch CPU, autograd).

Test infrastructure (see oracle/__init__.py). References are to arXiv 2411.14847.

Sec. 3.3 / App. B.2 deform each Gaussian with a multiresolution hash-encoding layer (I-NGP)
followed by a small MLP: H_dyn for the dynamic group (T = 2^16 entries, F = 4 features per
entry) and H_st for the static group (T = 2^14, F = 2). The paper fixes T and F only; the
remaining choices (readings) are: positions normalised by a bounding box to [0,1]^3 and clamped;
level l has N_l cells per axis with vertices 0..N_l; a level whose (N_l + 1)^3 vertices fit the
table is indexed densely (i + j (N_l+1) + k (N_l+1)^2), a finer one by the I-NGP spatial hash
(i * 1 XOR j * 2654435761 XOR k * 805459861) mod T; features are trilinearly interpolated and
concatenated over levels; one hidden layer of 64 ReLU units; 7 outputs read as the position
offset and the rotation offset sigma = (1, 0, 0, 0) + out[3:7], both used by the shift
norm(q) x norm(sigma).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
PRIMES = (1, 2654435761, 805459861)


def level_resolutions(levels, n_min=16, n_max=2048):
    """N_l = floor(n_min * b^l) with b = (n_max / n_min)^(1 / (levels - 1)) (geometric growth)."""
    if levels == 1:
        return [int(n_min)]
    b = np.exp((np.log(n_max) - np.log(n_min)) / (levels - 1))
    return [int(np.floor(n_min * b ** l)) for l in range(levels)]


def vertex_index(i, j, k, n_cells, table_size):
    """Table row of vertex (i, j, k) of a level with n_cells per axis (int64 arrays)."""
    v = n_cells + 1
    if v ** 3 <= table_size:
        return i + v * (j + v * k)
    h = (i * PRIMES[0]) ^ ((j * PRIMES[1]) & 0xFFFFFFFF) ^ ((k * PRIMES[2]) & 0xFFFFFFFF)
    return (h & 0xFFFFFFFF) % table_size


def cell_coordinates(means, bbox_min, bbox_max, n, fp32=False):
    """s = x * n with x the box-normalised position clamped to [0, 1]^3 ([N,3] float64 tensor).

    fp32=True takes the steps in FP32 as a single-precision implementation does -- x =
    (p - lo) * (1 / (hi - lo)) and s = x * n, each rounded to FP32 -- because s decides integers
    (the cell, hence which table rows are read) and, through the encoding, the ReLU pattern."""
    if fp32:
        p = np.asarray(means, dtype=np.float32)
        lo = np.asarray(bbox_min, dtype=np.float32)
        hi = np.asarray(bbox_max, dtype=np.float32)
        inv = (np.float32(1.0) / (hi - lo)).astype(np.float32)
        x = np.clip(((p - lo).astype(np.float32) * inv).astype(np.float32), 0.0, 1.0).astype(np.float32)
        return torch.as_tensor((x * np.float32(n)).astype(np.float32).astype(np.float64))
    p = torch.as_tensor(np.asarray(means, dtype=np.float64))
    lo = torch.as_tensor(np.asarray(bbox_min, dtype=np.float64))
    hi = torch.as_tensor(np.asarray(bbox_max, dtype=np.float64))
    return ((p - lo) / (hi - lo)).clamp(0.0, 1.0) * n


def encode(means, table, res, bbox_min, bbox_max, fp32_positions=False):
    """Concatenated trilinear interpolation of every level at the normalised positions.

    means [N,3]; table [L, T, F] (torch, may require grad); returns [N, L*F]."""
    T = table.shape[1]
    npts = np.asarray(means).shape[0]
    out = []
    for l, n in enumerate(res):
        s = cell_coordinates(means, bbox_min, bbox_max, n, fp32_positions)
        cell = torch.clamp(torch.floor(s), max=n - 1).to(torch.int64)
        frac = s - cell.to(DT)
        acc = torch.zeros((npts, table.shape[2]), dtype=DT)
        for c in range(8):
            bits = [(c >> d) & 1 for d in range(3)]
            corner = cell + torch.as_tensor(bits, dtype=torch.int64)
            idx = vertex_index(corner[:, 0].numpy(), corner[:, 1].numpy(), corner[:, 2].numpy(), n, T)
            w = torch.ones(npts, dtype=DT)
            for d in range(3):
                w = w * (frac[:, d] if bits[d] else 1.0 - frac[:, d])
            acc = acc + w[:, None] * table[l][torch.as_tensor(idx, dtype=torch.int64)]
        out.append(acc)
    return torch.cat(out, dim=1)


def field_offsets(means, params, res, bbox_min, bbox_max, fp32_positions=False):
    """Offsets [N,7] = (dmu, sigma) of the deformation field with params {table, w1, b1, w2, b2}."""
    enc = encode(means, params["table"], res, bbox_min, bbox_max, fp32_positions)
    h = torch.relu(enc @ params["w1"].T + params["b1"])
    out = h @ params["w2"].T + params["b2"]
    ident = torch.zeros(7, dtype=DT)
    ident[3] = 1.0
    return out + ident


def field_grads(means, params, res, bbox_min, bbox_max, d_offsets, fp32_positions=False):
    """Gradients of sum(offsets * d_offsets) w.r.t. every parameter (autograd)."""
    leaves = {k: torch.as_tensor(np.asarray(v, dtype=np.float64)).clone().requires_grad_(True)
              for k, v in params.items()}
    off = field_offsets(means, leaves, res, bbox_min, bbox_max, fp32_positions)
    (off * torch.as_tensor(np.asarray(d_offsets, dtype=np.float64))).sum().backward()
    return {k: v.grad.detach().clone() for k, v in leaves.items()}, off.detach()
