"""Buffers and the differentiable render built on the libdass entry points.

PyTorch allocates the device buffers; every computation is a libdass call. The pair
buffer grows on demand: bin/sort reports the exact pair count in counters[0] and an
overflow flag in counters[1]; on overflow the buffer is regrown and binning rerun.
"""
from __future__ import annotations

import math

import torch

from . import dass as D

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh")


def to_device(arrays: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(arrays[k], dtype=torch.float32).contiguous().to(device) for k in PARAM_NAMES}


class Frame:
    """Device buffers for rendering a Gaussian set of size n into a camera set."""

    def __init__(self, cams, n, tile=16, batch=128, pair_capacity=None, device="cuda"):
        self.cams = list(cams)
        self.n = int(n)
        self.tile = tile
        self.batch = batch
        self.device = device
        self.tiles_total, self.pixels = D.tile_layout(self.cams, tile)
        self.n_rec = len(self.cams) * self.n
        self.splats = torch.empty((max(1, self.n_rec), D.SPLAT_FLOATS), dtype=torch.float32, device=device)
        self.splat_grads = torch.empty((max(1, self.n_rec), D.GRAD_FLOATS), dtype=torch.float32, device=device)
        self.tile_ranges = torch.empty((max(1, self.tiles_total), 2), dtype=torch.int32, device=device)
        self.counters = torch.zeros(4, dtype=torch.int64, device=device)
        self.image = torch.empty(3 * self.pixels, dtype=torch.float32, device=device)
        self.T_final = torch.empty(self.pixels, dtype=torch.float32, device=device)
        self.n_last = torch.empty(self.pixels, dtype=torch.int32, device=device)
        cap = pair_capacity if pair_capacity is not None else max(1024, 8 * self.n_rec)
        self._alloc_pairs(cap)

    def _alloc_pairs(self, cap):
        if cap >= 1 << 31:
            raise D.DassError(f"pair buffer of {cap} pairs (sorted-pair positions are 32-bit: at most 2^31 - 1)",
                              D.ERR_INVALID_ARG)
        self.pair_capacity = int(cap)
        self.pair_rec = torch.empty(max(1, self.pair_capacity), dtype=torch.int32, device=self.device)
        ws = D.dass_bin_sort_workspace(self.n_rec, self.pair_capacity, self.tiles_total)
        self.workspace = torch.empty(max(1, ws), dtype=torch.uint8, device=self.device)

    def images(self):
        """Per-camera [3,H,W] views of the planar image buffer."""
        out, off = [], 0
        for c in self.cams:
            sz = 3 * c.width * c.height
            out.append(self.image[off:off + sz].view(3, c.height, c.width))
            off += sz
        return out

    def pixel_views(self, buf):
        out, off = [], 0
        for c in self.cams:
            sz = c.width * c.height
            out.append(buf[off:off + sz].view(c.height, c.width))
            off += sz
        return out

    def project(self, g, keep=None, stream=None):
        D.dass_preprocess(g, self.cams, self.tile, self.splats, keep=keep, stream=stream)

    def bin_sort(self, stream=None, grow=True):
        D.dass_bin_sort(self.splats, self.n, self.cams, self.tile, self.pair_rec, self.tile_ranges, self.counters,
                        self.workspace, stream=stream)
        if grow:
            m, over = (int(v) for v in self.counters[:2].tolist())
            if over:
                self._alloc_pairs(int(math.ceil(m * 1.25)) + 1024)
                D.dass_bin_sort(self.splats, self.n, self.cams, self.tile, self.pair_rec, self.tile_ranges,
                                self.counters, self.workspace, stream=stream)
        return int(self.counters[0].item()) if grow else None

    def render_fwd(self, bg=None, stream=None):
        D.dass_render_fwd(self.splats, self.pair_rec, self.tile_ranges, self.cams, self.tile, self.batch, self.image,
                          self.T_final, self.n_last, bg=bg, stream=stream)

    def render_bwd(self, dL_dimage, bg=None, stream=None):
        D.dass_render_bwd(self.splats, self.pair_rec, self.tile_ranges, self.cams, self.tile, self.batch,
                          self.T_final, self.n_last, dL_dimage, self.splat_grads, bg=bg, stream=stream)

    def render(self, g, keep=None, bg=None):
        self.project(g, keep)
        self.bin_sort()
        self.render_fwd(bg)
        return self.images()


class DassRender(torch.autograd.Function):
    """Differentiable multi-camera render: forward = [shift] -> preprocess -> bin/sort -> composite,
    backward = reverse-order composite backward -> preprocess backward -> [shift backward]. Returns
    the planar image buffer (all cameras concatenated).

    With dyn_idx and offsets ([n_dyn][7] = (dmu, sigma)) the dynamics-aware shift of Sec. 3.3 is
    applied to the dynamic rows before the projection (dass_shift): the offsets receive their
    gradient from dass_shift_bwd, and the means and quaternions of the dynamic rows receive the
    gradient w.r.t. their unshifted values (the mean's is the shifted one's, the quaternion's goes
    through norm(q) x norm(sigma))."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, offsets, frame: Frame, dyn_idx=None, bg=None):
        g = dict(means=means.detach().contiguous(), log_scales=log_scales.detach().contiguous(),
                 quats=quats.detach().contiguous(), opacity_logit=opacity_logit.detach().contiguous(),
                 sh=sh.detach().contiguous())
        gr = g
        off = None
        if offsets is not None:
            off = offsets.detach().contiguous()
            rm, rq = g["means"].clone(), g["quats"].clone()
            D.dass_shift(dyn_idx, off, g["means"], g["quats"], rm, rq)
            gr = dict(g, means=rm, quats=rq)
        frame.project(gr)
        frame.bin_sort()
        frame.render_fwd(bg)
        ctx.frame, ctx.bg, ctx.g, ctx.gr, ctx.off, ctx.dyn_idx = frame, bg, g, gr, off, dyn_idx
        return frame.image.clone()

    @staticmethod
    def backward(ctx, dimage):
        fr = ctx.frame
        fr.render_bwd(dimage.contiguous(), bg=ctx.bg)
        g, gr = ctx.g, ctx.gr
        out = {"d_means": torch.empty_like(g["means"]), "d_log_scales": torch.empty_like(g["log_scales"]),
               "d_quats": torch.empty_like(g["quats"]), "d_opacity_logit": torch.empty_like(g["opacity_logit"]),
               "d_sh": torch.empty_like(g["sh"])}
        D.dass_preprocess_bwd(gr, fr.cams, fr.splats, fr.splat_grads, out, D.GRAD_ALL)
        d_off = None
        if ctx.off is not None:
            idx = ctx.dyn_idx.long()
            dm = out["d_means"][idx].contiguous()
            dq = out["d_quats"][idx].contiguous()
            d_off = torch.empty_like(ctx.off)
            dq_in = torch.empty_like(dq)
            D.dass_shift_bwd(ctx.dyn_idx, ctx.off, g["quats"], dm, dq, d_off, dq_in)
            out["d_quats"][idx] = dq_in
        return (out["d_means"], out["d_log_scales"], out["d_quats"], out["d_opacity_logit"], out["d_sh"], d_off, None,
                None, None)


def render_autograd(params: dict, frame: Frame, bg=None, dyn_idx=None, offsets=None):
    """Differentiable render of params (dict of tensors) into the frame's cameras; with dyn_idx and
    offsets, through the dynamics-aware shift of the dynamic rows."""
    return DassRender.apply(params["means"], params["log_scales"], params["quats"], params["opacity_logit"],
                            params["sh"], offsets, frame, dyn_idx, bg)
