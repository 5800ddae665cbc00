"""Per-timestep driver of the streaming reconstruction on top of libdass.

A timestep (Sec. 3.1) turns G_{t-1} into G_t with the multi-view images of timestep t; the whole
sequence runs inside one C call, dass_timestep (Timestep below):
  1. selective inheritance (Sec. 3.2): s1 iterations learning the var-row mask, then the copy;
  2. dynamics-aware shift stage, s2 iterations (Sec. 3.3);
  3. error pass on the last shift render, Eq. 4 selection and spawn (Sec. 3.4);
  4. densification-stage training of the var rows, s3 iterations, then low-opacity pruning.
The stage classes run one stage through its C stage driver (ShiftStage -> dass_step, InheritStage
-> dass_inherit_step, DensifyStage -> dass_densify_step) over buffers allocated here, so each stage
can be run, timed and checked against the oracle on its own; FieldShiftStage composes the shift
stage with the hash-encoding deformation fields from individual entry points. This module only
allocates buffers (PyTorch) and marshals descriptors.
"""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import dass as D
from .raster import PARAM_NAMES, Frame


# Optimisation steps per timestep of the inheritance, shift and densification stages (Sec. 4.1).
PAPER_SCHEDULE = (20, 100, 60)


def _vp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class _FidelityLoss:
    """Eq. 3 over a fixed target set: the targets' SSIM window statistics are computed once
    (dass_loss_target_stats) and every iteration's loss reads them (dass_loss_cached)."""

    def __init__(self, targets, cams, lam):
        self.targets, self.cams, self.lam = targets, cams, lam
        self.ws = torch.empty(max(1, D.dass_loss_workspace(cams)), dtype=torch.uint8, device=targets.device)
        self.stats = None
        if lam > 0:
            self.stats = torch.empty(2 * targets.numel(), device=targets.device)
            D.dass_loss_target_stats(targets, cams, self.stats)

    def __call__(self, image, dL_dimage, loss):
        if self.stats is None:
            D.dass_loss(image, self.targets, self.cams, self.lam, dL_dimage, loss, self.ws)
        else:
            D.dass_loss_cached(image, self.targets, self.stats, self.cams, self.lam, dL_dimage, loss, self.ws)


class ShiftStage:
    """Buffers and descriptor of one shift-stage optimisation over a fixed Gaussian set."""

    def __init__(self, g, cams, targets, dyn_idx, offsets, tile=16, batch=128, lambda_dssim=0.2, lr_mu=1e-3,
                 lr_sigma=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, pair_capacity=None, stats=True, stream=None):
        self.g = {k: g[k].contiguous() for k in PARAM_NAMES}
        self.cams = list(cams)
        self.n = int(self.g["means"].shape[0])
        self.deg = int(round(math.sqrt(self.g["sh"].shape[1]))) - 1
        self.targets = targets.contiguous()
        self.dyn_idx = dyn_idx.contiguous()
        self.offsets = offsets.contiguous()
        self.n_dyn = int(self.dyn_idx.numel())
        dev = self.g["means"].device
        # per-Gaussian dynamics mask (Sec. 3.3), the dense form of dyn_idx
        self.dyn_mask = torch.zeros(max(1, self.n), dtype=torch.uint8, device=dev)
        if self.n_dyn:
            self.dyn_mask[self.dyn_idx.long()] = 1
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch, pair_capacity=pair_capacity or 1024)
        fr = self.frame
        self.render_means = self.g["means"].clone()
        self.render_quats = self.g["quats"].clone()
        nd = max(1, self.n_dyn)
        self.offset_grad = torch.zeros((nd, 7), device=dev)
        self.adam_m = torch.zeros((nd, 7), device=dev)
        self.adam_v = torch.zeros((nd, 7), device=dev)
        self.adam_step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.d_means_dyn = torch.zeros((nd, 3), device=dev)
        self.d_quats_dyn = torch.zeros((nd, 4), device=dev)
        self.dL_dimage = torch.zeros_like(fr.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self.stat_accum = torch.zeros(self.n, device=dev) if stats else None
        self.stat_count = torch.zeros(self.n, dtype=torch.int32, device=dev) if stats else None
        self.hp = dict(lr_mu=lr_mu, lr_sigma=lr_sigma, beta1=beta1, beta2=beta2, eps=eps, lambda_dssim=lambda_dssim)
        self._cams_arr = D.cameras(self.cams)
        if pair_capacity is None:
            # size the pair buffer from one binning of the unshifted scene (exact count + 25%)
            fr.project(self.g)
            m = fr.bin_sort()
            fr._alloc_pairs(int(m * 1.25) + 4096)
        self._build_desc()

    def _build_desc(self):
        fr = self.frame
        d = D.dass_step_desc()
        d.n, d.sh_degree, d.n_cams = self.n, self.deg, len(self.cams)
        d.means, d.log_scales, d.quats = _vp(self.g["means"]), _vp(self.g["log_scales"]), _vp(self.g["quats"])
        d.opacity_logit, d.sh = _vp(self.g["opacity_logit"]), _vp(self.g["sh"])
        d.cams = C.cast(self._cams_arr, C.c_void_p)
        d.targets = _vp(self.targets)
        d.n_dyn = self.n_dyn
        d.dyn_idx, d.offsets, d.offset_grad = _vp(self.dyn_idx), _vp(self.offsets), _vp(self.offset_grad)
        d.dyn_mask = _vp(self.dyn_mask)
        d.adam_m, d.adam_v, d.adam_step = _vp(self.adam_m), _vp(self.adam_v), _vp(self.adam_step)
        for k, v in self.hp.items():
            setattr(d, k, v)
        d.tile, d.batch = fr.tile, fr.batch
        d.render_means, d.render_quats = _vp(self.render_means), _vp(self.render_quats)
        d.d_means_dyn, d.d_quats_dyn = _vp(self.d_means_dyn), _vp(self.d_quats_dyn)
        d.splats, d.splat_grads = _vp(fr.splats), _vp(fr.splat_grads)
        d.pair_rec, d.pair_capacity = _vp(fr.pair_rec), fr.pair_capacity
        d.tile_ranges, d.counters = _vp(fr.tile_ranges), _vp(fr.counters)
        d.image, d.T_final, d.n_last = _vp(fr.image), _vp(fr.T_final), _vp(fr.n_last)
        d.dL_dimage, d.loss = _vp(self.dL_dimage), _vp(self.loss_buf)
        d.stat_accum, d.stat_count = _vp(self.stat_accum), _vp(self.stat_count)
        d.workspace, d.workspace_bytes = None, 0
        ws = D.dass_step_workspace(d)
        self.workspace = torch.empty(max(1, ws), dtype=torch.uint8, device=self.g["means"].device)
        d.workspace, d.workspace_bytes = _vp(self.workspace), ws
        self.desc = d

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def _snapshot(self):
        return [t.clone() for t in (self.offsets, self.adam_m, self.adam_v, self.adam_step)] + \
               ([self.stat_accum.clone(), self.stat_count.clone()] if self.stat_accum is not None else [])

    def _restore(self, snap):
        dst = [self.offsets, self.adam_m, self.adam_v, self.adam_step]
        if self.stat_accum is not None:
            dst += [self.stat_accum, self.stat_count]
        for d, s in zip(dst, snap):
            d.copy_(s)

    def run(self, n_iters, mode=D.STEP_BATCHED, max_regrow=3):
        """Run n_iters iterations; on pair-buffer overflow regrow and rerun from the saved state."""
        torch.cuda.current_stream().synchronize()
        for _ in range(max_regrow + 1):
            snap = self._snapshot()
            torch.cuda.synchronize()
            st = D.dass_step(self.desc, n_iters, mode, stream=self.stream)
            if st == D.OK:
                return
            m = int(self.frame.counters[0].item())
            self._restore(snap)
            self.frame._alloc_pairs(int(max(m, self.frame.pair_capacity) * 1.5) + 4096)
            self._build_desc()
        raise D.DassError("dass_step", D.ERR_CAPACITY)


def _render_fields(d, fr, dL_dimage, loss_buf):
    d.tile, d.batch = fr.tile, fr.batch
    d.splats, d.splat_grads = _vp(fr.splats), _vp(fr.splat_grads)
    d.pair_rec, d.pair_capacity = _vp(fr.pair_rec), fr.pair_capacity
    d.tile_ranges, d.counters = _vp(fr.tile_ranges), _vp(fr.counters)
    d.image, d.T_final, d.n_last = _vp(fr.image), _vp(fr.T_final), _vp(fr.n_last)
    d.dL_dimage, d.loss = _vp(dL_dimage), _vp(loss_buf)


def _scene_fields(d, g, n, cams_arr, n_cams):
    d.n, d.n_cams = n, n_cams
    d.sh_degree = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    d.means, d.log_scales, d.quats = _vp(g["means"]), _vp(g["log_scales"]), _vp(g["quats"])
    d.opacity_logit, d.sh = _vp(g["opacity_logit"]), _vp(g["sh"])
    d.cams = C.cast(cams_arr, C.c_void_p)


class InheritStage:
    """Selective-inheritance stage (Sec. 3.2, App. B.2) through dass_inherit_step: learns one logit m
    per var Gaussian of G_{t-1} against the images of timestep t, every other parameter fixed.

    One iteration (captured once as a CUDA graph and replayed): keep = Quant(sigmoid(m)) on var rows ->
    projection with opacity and scale multiplied by keep (Eq. 1) -> bin/sort -> forward -> loss of
    Eq. 3 -> backward (full splat gradients for var rows only) -> dL/dkeep -> the straight-through
    gradient with the mask loss of Eq. 2 -> Adam on m. The pair buffer is sized by one binning with
    every var row rendered (the most the stage can render, since a masked row only receives the mask
    loss); an overflow restores m and its Adam state and reruns with a larger buffer.

    The paper fixes neither lambda_inher, the initial logit nor the optimiser of m: m starts at
    m0 > 0 (every var row inherited unless the stage learns otherwise) and takes Adam steps.
    """

    def __init__(self, g, is_var, cams, targets, tile=16, batch=128, lambda_dssim=0.2, lambda_inher=1e-6, m0=0.5,
                 lr=0.05, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
        self.g = {k: g[k].contiguous() for k in PARAM_NAMES}
        self.cams = list(cams)
        self.n = int(self.g["means"].shape[0])
        dev = self.g["means"].device
        self.is_var = is_var[:self.n].contiguous()
        self.var_rows = torch.nonzero(self.is_var).flatten().to(torch.int32).contiguous()
        self.n_var = int(self.var_rows.numel())
        self.targets = targets.contiguous()
        self.m = torch.full((max(1, self.n),), float(m0), device=dev)
        self.keep = torch.ones(max(1, self.n), dtype=torch.uint8, device=dev)
        self.grad = torch.zeros(max(1, self.n), device=dev)
        self.adam_m = torch.zeros(max(1, self.n), device=dev)
        self.adam_v = torch.zeros(max(1, self.n), device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.d_keep = torch.zeros(max(1, self.n_var), device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch)
        self.dL_dimage = torch.zeros_like(self.frame.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self.hp = dict(lr=float(lr), beta1=float(beta1), beta2=float(beta2), eps=float(eps),
                       lambda_dssim=float(lambda_dssim), lambda_inher=float(lambda_inher))
        self._cams_arr = D.cameras(self.cams)
        if self.n:
            self.frame.project(self.g)             # every var row rendered: the stage's largest pair count
            m_pairs = self.frame.bin_sort()
            self.frame._alloc_pairs(int(m_pairs * 1.1) + 4096)
        self._build_desc()

    def _build_desc(self):
        d = D.dass_inherit_step_desc()
        _scene_fields(d, self.g, self.n, self._cams_arr, len(self.cams))
        d.is_var, d.targets = _vp(self.is_var), _vp(self.targets)
        d.n_var, d.var_rows = self.n_var, _vp(self.var_rows)
        d.m, d.keep, d.m_grad = _vp(self.m), _vp(self.keep), _vp(self.grad)
        d.adam_m, d.adam_v, d.adam_step, d.d_keep = _vp(self.adam_m), _vp(self.adam_v), _vp(self.step), _vp(self.d_keep)
        for k, v in self.hp.items():
            setattr(d, k, v)
        _render_fields(d, self.frame, self.dL_dimage, self.loss_buf)
        d.workspace, d.workspace_bytes = None, 0
        ws = D.dass_inherit_step_workspace(d)
        self.workspace = torch.empty(max(1, ws), dtype=torch.uint8, device=self.g["means"].device)
        d.workspace, d.workspace_bytes = _vp(self.workspace), ws
        self.desc = d

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def run(self, n_iters, max_regrow=3):
        """n_iters iterations; returns the learned logits m (var rows meaningful)."""
        if n_iters <= 0 or self.n == 0:
            return self.m
        torch.cuda.current_stream().synchronize()
        for _ in range(max_regrow + 1):
            snap = [t.clone() for t in (self.m, self.adam_m, self.adam_v, self.step)]
            torch.cuda.synchronize()
            if D.dass_inherit_step(self.desc, n_iters, stream=self.stream) == D.OK:
                return self.m
            for dst, src in zip((self.m, self.adam_m, self.adam_v, self.step), snap):
                dst.copy_(src)
            self.frame._alloc_pairs(int(self.frame.pair_capacity * 1.5) + 4096)
            self._build_desc()
        raise D.DassError("dass_inherit_step", D.ERR_CAPACITY)


class DensifyStage:
    """Densification-stage training (Sec. 3.4) through dass_densify_step: s3 iterations of the fidelity
    loss (Eq. 3) over every parameter of the var Gaussians (the new spawns and the inherited var
    rows), base rows fixed.

    The var rows must be the contiguous tail [n_base, n) of the arrays (the layout dass_inherit and
    dass_spawn produce): the backward runs full splat gradients for var rows only, the parameter
    gradients of the tail land in one buffer (per parameter: `grads[name]` views it) and Adam updates
    each parameter slice of the tail. One iteration is captured as a CUDA graph and replayed.

    The paper trains these Gaussians as vanilla 3DGS does and states no learning rates; the 3DGS
    ones are used (positions 1.6e-4 per unit of scene extent, log-scales 5e-3, rotations 1e-3,
    opacity logits 5e-2, SH DC 2.5e-3 and higher bands 2.5e-3 / 20)."""

    def __init__(self, g, n_base, cams, targets, tile=16, batch=128, lambda_dssim=0.2, extent=3.0, lr=None,
                 beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
        self.g = {k: g[k] for k in PARAM_NAMES}
        for k in PARAM_NAMES:
            assert self.g[k].is_contiguous()
        self.cams = list(cams)
        self.n = int(self.g["means"].shape[0])
        self.n_base = int(n_base)
        self.n_var = self.n - self.n_base
        dev = self.g["means"].device
        self.K = int(self.g["sh"].shape[1])
        self.targets = targets.contiguous()
        lr = dict(lr or {})
        self.lr = dict(means=lr.get("means", 1.6e-4 * extent), log_scales=lr.get("log_scales", 5e-3),
                       quats=lr.get("quats", 1e-3), opacity_logit=lr.get("opacity_logit", 5e-2),
                       sh_dc=lr.get("sh_dc", 2.5e-3), sh_rest=lr.get("sh_rest", 2.5e-3 / 20))
        self.betas, self.eps, self.lam = (float(beta1), float(beta2)), float(eps), float(lambda_dssim)
        self.full = torch.zeros(max(1, self.n), dtype=torch.uint8, device=dev)
        self.full[self.n_base:self.n] = 1
        nv = max(1, self.n_var)
        widths = dict(means=3, log_scales=3, quats=4, opacity_logit=1, sh=3 * self.K)
        total = sum(widths.values()) * nv
        self.grad_buf = torch.zeros(total, device=dev)
        self.m_buf = torch.zeros(total, device=dev)
        self.v_buf = torch.zeros(total, device=dev)
        self.grads, off = {}, 0
        for k, w in widths.items():          # parameter-major views of the packed gradient buffer
            self.grads[k] = self.grad_buf[off:off + w * nv].view(nv, w)
            off += w * nv
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch)
        self.dL_dimage = torch.zeros_like(self.frame.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self._cams_arr = D.cameras(self.cams)
        if self.n:
            self.frame.project(self.g)
            m_pairs = self.frame.bin_sort()
            # the var rows move and change size: 50% headroom over the pairs of the starting scene
            self.frame._alloc_pairs(int(m_pairs * 1.5) + 4096)
        self._build_desc()

    def _build_desc(self):
        d = D.dass_densify_step_desc()
        _scene_fields(d, self.g, self.n, self._cams_arr, len(self.cams))
        d.n_base, d.is_var, d.targets = self.n_base, _vp(self.full), _vp(self.targets)
        d.grad, d.adam_m, d.adam_v, d.adam_step = _vp(self.grad_buf), _vp(self.m_buf), _vp(self.v_buf), _vp(self.step)
        d.lr_means, d.lr_log_scales, d.lr_quats = self.lr["means"], self.lr["log_scales"], self.lr["quats"]
        d.lr_opacity, d.lr_sh_dc, d.lr_sh_rest = self.lr["opacity_logit"], self.lr["sh_dc"], self.lr["sh_rest"]
        d.beta1, d.beta2, d.eps, d.lambda_dssim = self.betas[0], self.betas[1], self.eps, self.lam
        _render_fields(d, self.frame, self.dL_dimage, self.loss_buf)
        d.workspace, d.workspace_bytes = None, 0
        ws = D.dass_densify_step_workspace(d)
        self.workspace = torch.empty(max(1, ws), dtype=torch.uint8, device=self.g["means"].device)
        d.workspace, d.workspace_bytes = _vp(self.workspace), ws
        self.desc = d

    def _slice(self, k):
        return self.g[k][self.n_base:self.n].reshape(self.n_var, -1)

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def run(self, n_iters, max_regrow=2):
        """n_iters iterations; on pair-buffer overflow the var rows and optimiser state are restored
        and the stage reruns with a larger pair buffer."""
        if n_iters <= 0 or self.n == 0:
            return
        torch.cuda.current_stream().synchronize()
        for _ in range(max_regrow + 1):
            snap = [self._slice(k).clone() for k in PARAM_NAMES] + [t.clone() for t in (self.m_buf, self.v_buf,
                                                                                         self.step)]
            torch.cuda.synchronize()
            if D.dass_densify_step(self.desc, n_iters, stream=self.stream) == D.OK:
                return
            for k, v in zip(PARAM_NAMES, snap):
                self._slice(k).copy_(v)
            for dst, src in zip((self.m_buf, self.v_buf, self.step), snap[len(PARAM_NAMES):]):
                dst.copy_(src)
            self.frame._alloc_pairs(2 * self.frame.pair_capacity)
            self._build_desc()
        raise D.DassError("dass_densify_step", D.ERR_CAPACITY)


def level_resolutions(levels, n_min=16, n_max=2048):
    """Cells per axis of each hash-grid level: floor(n_min * b^l), b = (n_max / n_min)^(1/(levels-1))."""
    if levels == 1:
        return [int(n_min)]
    b = math.exp((math.log(n_max) - math.log(n_min)) / (levels - 1))
    return [int(math.floor(n_min * b ** l)) for l in range(levels)]


def init_field(levels, features, log2_table, hidden=64, seed=0, device="cuda"):
    """Parameters of a hash-encoding deformation field: table U(-1e-4, 1e-4) (the I-NGP
    initialisation), w1 He-normal, b1 = 0, and a zero output layer so that the field starts as the
    identity deformation (dmu = 0, sigma = (1, 0, 0, 0))."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    T = 1 << log2_table
    n_in = levels * features
    p = {"table": (torch.rand((levels, T, features), generator=gen) * 2e-4 - 1e-4),
         "w1": torch.randn((hidden, n_in), generator=gen) * math.sqrt(2.0 / n_in),
         "b1": torch.zeros(hidden), "w2": torch.zeros((7, hidden)), "b2": torch.zeros(7)}
    return {k: v.to(device=device, dtype=torch.float32).contiguous() for k, v in p.items()}


class FieldShiftStage:
    """Dynamics-aware shift with the paper's hash-encoding deformation fields (Sec. 3.3, App. B.2):
    H_dyn (T = 2^16, F = 4) deforms the dynamic group and the lighter H_st (T = 2^14, F = 2) the
    static group; both are trained with the fidelity loss of Eq. 3.

    One iteration: offsets of both groups (dass_field_fwd) -> shift of every row (dass_shift) ->
    projection -> bin/sort -> forward -> loss -> backward (full splat gradients for every row) ->
    gradients of the shifted means and quaternions per group (dass_preprocess_bwd) -> offset
    gradients (dass_shift_bwd) -> field gradients (dass_field_bwd) -> Adam on every field tensor.
    The first iteration runs eagerly, the rest replay it as a captured CUDA graph. The paper names
    the table sizes and feature widths only; levels (16, resolutions 16..2048), the 64-unit hidden
    layer, the identity initialisation and the Adam learning rate are readings."""

    def __init__(self, g, cams, targets, dyn_idx, tile=16, batch=128, lambda_dssim=0.2, levels=16, bbox=None,
                 lr=1e-3, dyn_spec=(4, 16), st_spec=(2, 14), beta1=0.9, beta2=0.999, eps=1e-15, seed=0):
        self.g = {k: g[k].contiguous() for k in PARAM_NAMES}
        self.cams = list(cams)
        self.n = int(self.g["means"].shape[0])
        dev = self.g["means"].device
        self.targets = targets.contiguous()
        self.lam = float(lambda_dssim)
        self.lr, self.betas, self.eps = float(lr), (float(beta1), float(beta2)), float(eps)
        mask = torch.zeros(self.n, dtype=torch.bool, device=dev)
        mask[dyn_idx.long()] = True
        self.groups = []
        if bbox is None:
            lo = self.g["means"].min(0).values.cpu().numpy() - 1e-3
            hi = self.g["means"].max(0).values.cpu().numpy() + 1e-3
        else:
            lo, hi = bbox
        for gi, (rows, (feats, log2t)) in enumerate(((torch.nonzero(mask).flatten(), dyn_spec),
                                                     (torch.nonzero(~mask).flatten(), st_spec))):
            rows = rows.to(torch.int32).contiguous()
            nr = int(rows.numel())
            prm = init_field(levels, feats, log2t, seed=seed + gi, device=dev)
            res = level_resolutions(levels)
            grp = {"rows": rows, "n": nr, "params": prm, "res": res, "log2t": log2t,
                   "field": D.field_struct(prm, res, log2t, lo, hi),
                   "grads": {k: torch.zeros_like(v) for k, v in prm.items()},
                   "m": {k: torch.zeros_like(v) for k, v in prm.items()},
                   "v": {k: torch.zeros_like(v) for k, v in prm.items()},
                   "offsets": torch.zeros((max(1, nr), 7), device=dev),
                   "d_offsets": torch.zeros((max(1, nr), 7), device=dev),
                   "d_means": torch.zeros((max(1, nr), 3), device=dev),
                   "d_quats": torch.zeros((max(1, nr), 4), device=dev)}
            self.groups.append(grp)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.render_means = self.g["means"].clone()
        self.render_quats = self.g["quats"].clone()
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch)
        self.dL_dimage = torch.zeros_like(self.frame.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self.overflow = torch.zeros(1, dtype=torch.int64, device=dev)
        self.fidelity = _FidelityLoss(self.targets, self.cams, self.lam)
        self.graph = None

    def _render_g(self):
        return dict(self.g, means=self.render_means, quats=self.render_quats)

    def _iteration(self, eager=False):
        fr = self.frame
        for grp in self.groups:
            if grp["n"]:
                D.dass_field_fwd(grp["field"], self.g["means"], grp["offsets"], rows=grp["rows"])
                D.dass_shift(grp["rows"], grp["offsets"], self.g["means"], self.g["quats"], self.render_means,
                             self.render_quats)
        gr = self._render_g()
        fr.project(gr)
        if eager:
            fr.bin_sort()
        else:
            fr.bin_sort(grow=False)
            torch.maximum(self.overflow, fr.counters[1:2], out=self.overflow)
        fr.render_fwd()
        self.loss_buf.zero_()
        self.fidelity(fr.image, self.dL_dimage, self.loss_buf)
        fr.render_bwd(self.dL_dimage)
        b1, b2 = self.betas
        last = max(i for i, grp in enumerate(self.groups) if grp["n"]) if any(g_["n"] for g_ in self.groups) else -1
        for gi, grp in enumerate(self.groups):
            if not grp["n"]:
                continue
            D.dass_preprocess_bwd(gr, self.cams, fr.splats, fr.splat_grads,
                                  {"d_means": grp["d_means"], "d_quats": grp["d_quats"]},
                                  D.GRAD_MEANS | D.GRAD_QUATS, rows=grp["rows"])
            D.dass_shift_bwd(grp["rows"], grp["offsets"], self.g["quats"], grp["d_means"], grp["d_quats"],
                             grp["d_offsets"])
            for t in grp["grads"].values():
                t.zero_()
            D.dass_field_bwd(grp["field"], self.g["means"], grp["d_offsets"], grp["grads"], rows=grp["rows"])
            names = list(grp["params"].keys())
            for i, k in enumerate(names):
                p_, g_ = grp["params"][k], grp["grads"][k]
                w = 16 if p_.numel() % 16 == 0 else 1
                D.dass_adam(p_.view(-1, w), g_.view(-1, w), grp["m"][k].view(-1, w), grp["v"][k].view(-1, w),
                            self.step, [self.lr] * w, b1, b2, self.eps,
                            increment_step=(gi == last and i == len(names) - 1))

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def run(self, n_iters):
        if n_iters <= 0 or self.n == 0:
            return
        replays = n_iters
        if self.graph is None:
            self._iteration(eager=True)
            replays -= 1
            if replays > 0:
                m_pairs = int(self.frame.counters[0].item())
                if self.frame.pair_capacity < int(m_pairs * 1.25) + 4096:
                    self.frame._alloc_pairs(int(m_pairs * 1.25) + 4096)
                torch.cuda.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self._iteration()
        for _ in range(replays):
            self.graph.replay()
        if replays > 0 and int(self.overflow.item()):
            raise D.DassError("field shift stage bin_sort", D.ERR_CAPACITY)


class Timestep:
    """One full timestep t of the streaming pipeline (dass_timestep) over resident device buffers.

    The scene arrays have room for `n_max` rows; `n` tracks the live count. Hyper-parameters (paper
    readings where the paper states none): lambda = 0.2, inheritance logits start at 0.5 with Adam
    lr 0.05 and lambda_inher = 1e-6, offsets Adam lr 1e-3, error quantile 0.95, tau_pos = 2e-4,
    tau_err = 1e-4, at most 5000 spawns, erase every 20 timesteps, prune below opacity 0.005, and the
    3DGS learning rates in the densification stage. A pair overflow in any stage leaves G_{t-1}
    untouched; the pair buffer is then regrown from the reported count and the timestep rerun."""

    def __init__(self, cams, n_max, sh_degree, tile=16, batch=128, lambda_dssim=0.2, n_shift=100,
                 quantile=0.95, tau_pos=2e-4, tau_err=1e-4, k_max=5000, erase_every=20, n_inherit=0,
                 lambda_inher=1e-6, n_densify=0, prune_opacity=0.005, extent=3.0, device="cuda", stream=None):
        self.cams = list(cams)
        self.n_max = int(n_max)
        self.deg = sh_degree
        self.K = (sh_degree + 1) ** 2
        self.tile, self.batch = tile, batch
        self.device = device
        self.hp = dict(lambda_dssim=float(lambda_dssim), lambda_inher=float(lambda_inher), inherit_m0=0.5,
                       quantile=float(quantile), tau_pos=float(tau_pos), tau_err=float(tau_err),
                       prune_opacity=float(prune_opacity), lr_inherit=0.05, lr_mu=1e-3, lr_sigma=1e-3,
                       lr_means=1.6e-4 * extent, lr_log_scales=5e-3, lr_quats=1e-3, lr_opacity=5e-2,
                       lr_sh_dc=2.5e-3, lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15)
        self.sched = dict(n_inherit=int(n_inherit), n_shift=int(n_shift), n_densify=int(n_densify),
                          k_max=int(k_max), erase_every=int(erase_every))
        self.k_max = int(k_max)
        shapes = dict(means=(3,), log_scales=(3,), quats=(4,), opacity_logit=(), sh=(self.K, 3))
        self.bufs = {k: torch.zeros((self.n_max,) + s, device=device) for k, s in shapes.items()}
        self.is_var = torch.zeros(self.n_max, dtype=torch.uint8, device=device)
        self.n = 0
        self._n_host = C.c_int64(0)
        self._cams_arr = D.cameras(self.cams)
        self.tiles_total, self.pixels = D.tile_layout(self.cams, tile)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.pair_capacity = None
        self.workspace = None
        self.last_stats = None

    def load(self, arrays: dict, is_var=None):
        n = int(arrays["means"].shape[0])
        assert n + self.k_max <= self.n_max
        for k in PARAM_NAMES:
            self.bufs[k][:n].copy_(torch.as_tensor(arrays[k], dtype=torch.float32))
        self.is_var.zero_()
        if is_var is not None:
            self.is_var[:n].copy_(torch.as_tensor(is_var, dtype=torch.uint8))
        self.n = n

    def view(self):
        return {k: v[:self.n] for k, v in self.bufs.items()}

    def _size_pairs(self):
        """Pair buffer from one binning of the current scene (all views), with headroom for the
        spawned and moving Gaussians of the coming timesteps."""
        fr = Frame(self.cams, self.n, tile=self.tile, batch=self.batch)
        fr.project(self.view())
        return int(fr.bin_sort() * 1.3) + (1 << 16)

    def _alloc(self, n_dyn):
        d = self._desc_template(n_dyn)
        ws = D.dass_timestep_workspace(d)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def _desc_template(self, n_dyn):
        d = D.dass_timestep_desc()
        d.n_max, d.sh_degree, d.n_cams = self.n_max, self.deg, len(self.cams)
        for k in PARAM_NAMES:
            setattr(d, k, _vp(self.bufs[k]))
        d.is_var, d.n, d.cams = _vp(self.is_var), C.cast(C.pointer(self._n_host), C.c_void_p), \
            C.cast(self._cams_arr, C.c_void_p)
        d.n_dyn = n_dyn
        d.tile, d.batch, d.pair_capacity = self.tile, self.batch, self.pair_capacity
        for k, v in self.sched.items():
            setattr(d, k, v)
        for k, v in self.hp.items():
            setattr(d, k, v)
        return d

    def run(self, t, targets, dyn_idx, offsets, z=None, targets_host=None, host_out=None, max_regrow=3,
            next_targets_host=None, next_targets=None):
        """Reconstruct timestep t from the images `targets` (device; with targets_host (pinned host
        tensor) the call first uploads it into `targets`). `offsets` ([n_dyn][7], device) gives the
        initial offsets and receives the learned ones. host_out (optional dict of pinned host tensors
        like `bufs` plus is_var) receives G_t. With next_targets_host (pinned host tensor) and
        next_targets (a second device image buffer), the next timestep's images are uploaded while
        this one trains; the next call then takes next_targets as its `targets`. Returns a dict of
        what the timestep did."""
        if (next_targets_host is None) != (next_targets is None):
            raise ValueError("next_targets_host and next_targets go together")
        n_dyn = int(dyn_idx.numel())
        dyn_idx = dyn_idx.contiguous()
        off_init = offsets.contiguous().clone()
        if z is None:
            z = torch.zeros((self.n_max, 3), device=self.device)
        if self.pair_capacity is None:
            self.pair_capacity = self._size_pairs()
            self._alloc(n_dyn)
        torch.cuda.current_stream().synchronize()
        for _ in range(max_regrow + 1):
            d = self._desc_template(n_dyn)
            self._n_host.value = self.n
            d.targets, d.targets_host = _vp(targets), (C.c_void_p(targets_host.data_ptr())
                                                       if targets_host is not None else None)
            if next_targets is not None:
                d.next_targets_host, d.next_targets = C.c_void_p(next_targets_host.data_ptr()), _vp(next_targets)
            d.t = int(t)
            d.dyn_idx, d.offsets_init, d.offsets, d.z = _vp(dyn_idx), _vp(off_init), _vp(offsets), _vp(z)
            need = D.dass_timestep_workspace(d)
            if self.workspace is None or self.workspace.numel() < need:
                self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            d.workspace, d.workspace_bytes = _vp(self.workspace), self.workspace.numel()
            if host_out is not None:
                for k in PARAM_NAMES:
                    setattr(d, "host_" + k, C.c_void_p(host_out[k].data_ptr()))
                d.host_is_var = C.c_void_p(host_out["is_var"].data_ptr())
            st, stats = D.dass_timestep(d, stream=self.stream)
            if st == D.OK:
                self.n = int(self._n_host.value)
                self.last_stats = stats.as_dict()
                s = self.last_stats
                return dict(loss=s["loss_shift"], n=self.n, spawned=s["n_spawned"],
                            densify_loss=s["loss_densify"] if s["n_var_trained"] else None,
                            pruned=s["n_inherited"] + s["n_spawned"] - s["n_out"] if s["n_var_trained"] else 0,
                            inherit_loss=s["loss_inherit"] if s["inherit_ran"] else None, stats=s)
            # a stage overflowed the pair buffer: G_{t-1} is unchanged, regrow and rerun
            self.pair_capacity = min((1 << 31) - 1, int(max(stats.pairs_max, self.pair_capacity) * 1.25) + 4096)
            self.workspace = None
        raise D.DassError("dass_timestep", D.ERR_CAPACITY)
