"""Per-timestep driver of the streaming reconstruction on top of libdass.

A timestep (Sec. 3.1) turns G_{t-1} into G_t with the multi-view images of timestep t:
  1. selective inheritance (Sec. 3.2): s1 iterations learning the var-row mask (InheritStage:
     dass_inherit_keep, dass_keep_grad, dass_inherit_mask_grad, dass_adam), then the copy
                                                           -> dass_inherit
  2. dynamics-aware shift stage, n_shift iterations (Sec. 3.3) -> dass_step (graph replay)
  3. error pass on the last shift render, Eq. 4 selection and spawn (Sec. 3.4)
                                                           -> dass_error_pass, dass_densify_select, dass_spawn
  4. densification-stage training of the var rows, s3 iterations (DensifyStage: dass_preprocess_bwd
     over the var tail, dass_adam), then low-opacity pruning -> dass_prune_logits, dass_inherit
This module only allocates buffers (PyTorch) and sequences the calls.
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


class InheritStage:
    """Selective-inheritance stage (Sec. 3.2, App. B.2): learns one logit m per var Gaussian of
    G_{t-1} against the images of timestep t, every other parameter fixed.

    One iteration: keep = Quant(sigmoid(m)) on var rows (dass_inherit_keep) -> projection with
    opacity and scale multiplied by keep (Eq. 1) -> bin/sort -> forward -> loss of Eq. 3 ->
    backward (full splat gradients for var rows only) -> dL/dkeep (dass_keep_grad) -> the
    straight-through gradient with the mask loss of Eq. 2 (dass_inherit_mask_grad) -> Adam on m.
    The first iteration runs eagerly (it sizes the pair buffer with every var row rendered, the
    most the stage can render since a masked row only receives the mask loss); the others replay
    it as one captured CUDA graph.

    The paper fixes neither lambda_inher, the initial logit nor the optimiser of m: m starts at
    m0 > 0 (every var row inherited unless the stage learns otherwise) and takes Adam steps.
    """

    def __init__(self, g, is_var, cams, targets, tile=16, batch=128, lambda_dssim=0.2, lambda_inher=1e-6, m0=0.5,
                 lr=0.05, beta1=0.9, beta2=0.999, eps=1e-15):
        self.g = {k: g[k].contiguous() for k in PARAM_NAMES}
        self.cams = list(cams)
        self.n = int(self.g["means"].shape[0])
        dev = self.g["means"].device
        self.is_var = is_var[:self.n].contiguous()
        self.var_rows = torch.nonzero(self.is_var).flatten().to(torch.int32).contiguous()
        self.n_var = int(self.var_rows.numel())
        self.targets = targets.contiguous()
        self.lam, self.lam_inher = float(lambda_dssim), float(lambda_inher)
        self.lr, self.betas, self.eps = float(lr), (float(beta1), float(beta2)), float(eps)
        self.m = torch.full((max(1, self.n),), float(m0), device=dev)
        self.keep = torch.ones(max(1, self.n), dtype=torch.uint8, device=dev)
        self.grad = torch.zeros(max(1, self.n), device=dev)
        self.adam_m = torch.zeros(max(1, self.n), device=dev)
        self.adam_v = torch.zeros(max(1, self.n), device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.d_keep = torch.zeros(max(1, self.n_var), device=dev)
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch)
        self.dL_dimage = torch.zeros_like(self.frame.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self.overflow = torch.zeros(1, dtype=torch.int64, device=dev)
        self.fidelity = _FidelityLoss(self.targets, self.cams, self.lam)
        self.graph = None

    def _iteration(self, eager=False):
        fr = self.frame
        D.dass_inherit_keep(self.is_var, self.m, self.keep)
        fr.project(self.g, keep=self.keep)
        if eager:
            fr.bin_sort()
        else:
            fr.bin_sort(grow=False)
            torch.maximum(self.overflow, fr.counters[1:2], out=self.overflow)
        fr.render_fwd()
        self.loss_buf.zero_()
        self.fidelity(fr.image, self.dL_dimage, self.loss_buf)
        D.dass_render_bwd(fr.splats, fr.pair_rec, fr.tile_ranges, self.cams, fr.tile, fr.batch, fr.T_final,
                          fr.n_last, self.dL_dimage, fr.splat_grads, full_grad=self.is_var, rec_stride=self.n)
        if self.n_var:
            D.dass_keep_grad(self.g, self.cams, fr.splats, fr.splat_grads, self.d_keep, keep=self.keep,
                             rows=self.var_rows)
            D.dass_inherit_mask_grad(self.var_rows, self.m, self.d_keep, self.lam_inher, self.grad, self.loss_buf)
            D.dass_adam(self.m.view(-1, 1), self.grad.view(-1, 1), self.adam_m.view(-1, 1), self.adam_v.view(-1, 1),
                        self.step, [self.lr], self.betas[0], self.betas[1], self.eps, rows=self.var_rows)

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def run(self, n_iters):
        """n_iters iterations; returns the learned logits m (var rows meaningful)."""
        if n_iters <= 0 or self.n == 0:
            return self.m
        replays = n_iters
        if self.graph is None:
            self._iteration(eager=True)
            replays -= 1
            if replays > 0:
                # the pair buffer now holds the exact count with every var row rendered (+ margin)
                m_pairs = int(self.frame.counters[0].item())
                if self.frame.pair_capacity < m_pairs * 1.05 + 1024:
                    self.frame._alloc_pairs(int(m_pairs * 1.1) + 1024)
                torch.cuda.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self._iteration()
        for _ in range(replays):
            self.graph.replay()
        if replays > 0 and int(self.overflow.item()):
            raise D.DassError("inherit stage bin_sort", D.ERR_CAPACITY)
        return self.m


class DensifyStage:
    """Densification-stage training (Sec. 3.4): s3 iterations of the fidelity loss (Eq. 3) over every
    parameter of the var Gaussians (the new spawns and the inherited var rows), base rows fixed.

    The var rows must be the contiguous tail [n_base, n) of the arrays (the layout dass_inherit and
    dass_spawn produce), so each parameter's var part is a slice: the backward runs full splat
    gradients for var rows only (dass_render_bwd full_grad), dass_preprocess_bwd with rows = the
    tail gives compact gradients of exactly those slices, and dass_adam updates the slices. One
    iteration runs eagerly, the rest replay it as a captured CUDA graph.

    The paper trains these Gaussians as vanilla 3DGS does and states no learning rates; the 3DGS
    ones are used (positions 1.6e-4 per unit of scene extent, log-scales 5e-3, rotations 1e-3,
    opacity logits 5e-2, SH DC 2.5e-3 and higher bands 2.5e-3 / 20)."""

    def __init__(self, g, n_base, cams, targets, tile=16, batch=128, lambda_dssim=0.2, extent=3.0, lr=None,
                 beta1=0.9, beta2=0.999, eps=1e-15):
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
        self.lam = float(lambda_dssim)
        lr = dict(lr or {})
        self.lr = dict(means=lr.get("means", 1.6e-4 * extent), log_scales=lr.get("log_scales", 5e-3),
                       quats=lr.get("quats", 1e-3), opacity_logit=lr.get("opacity_logit", 5e-2),
                       sh_dc=lr.get("sh_dc", 2.5e-3), sh_rest=lr.get("sh_rest", 2.5e-3 / 20))
        self.betas, self.eps = (float(beta1), float(beta2)), float(eps)
        self.rows = torch.arange(self.n_base, self.n, dtype=torch.int32, device=dev)
        self.full = torch.zeros(max(1, self.n), dtype=torch.uint8, device=dev)
        self.full[self.n_base:self.n] = 1
        nv = max(1, self.n_var)
        widths = dict(means=3, log_scales=3, quats=4, opacity_logit=1, sh=3 * self.K)
        self.grads = {k: torch.zeros((nv, w), device=dev) for k, w in widths.items()}
        self.adam_m = {k: torch.zeros((nv, w), device=dev) for k, w in widths.items()}
        self.adam_v = {k: torch.zeros((nv, w), device=dev) for k, w in widths.items()}
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        band = torch.arange(max(1, self.n_var) * self.K, device=dev) % self.K
        self.sh_dc_rows = torch.nonzero(band == 0).flatten().to(torch.int32).contiguous()
        self.sh_rest_rows = torch.nonzero(band > 0).flatten().to(torch.int32).contiguous()
        self.frame = Frame(self.cams, self.n, tile=tile, batch=batch)
        self.dL_dimage = torch.zeros_like(self.frame.image)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        self.overflow = torch.zeros(1, dtype=torch.int64, device=dev)
        self.fidelity = _FidelityLoss(self.targets, self.cams, self.lam)
        self.graph = None

    def _slice(self, k):
        return self.g[k][self.n_base:self.n].reshape(self.n_var, -1)

    def _iteration(self, eager=False):
        fr = self.frame
        fr.project(self.g)
        if eager:
            fr.bin_sort()
        else:
            fr.bin_sort(grow=False)
            torch.maximum(self.overflow, fr.counters[1:2], out=self.overflow)
        fr.render_fwd()
        self.loss_buf.zero_()
        self.fidelity(fr.image, self.dL_dimage, self.loss_buf)
        D.dass_render_bwd(fr.splats, fr.pair_rec, fr.tile_ranges, self.cams, fr.tile, fr.batch, fr.T_final,
                          fr.n_last, self.dL_dimage, fr.splat_grads, full_grad=self.full, rec_stride=self.n)
        if self.n_var == 0:
            return
        out = {"d_means": self.grads["means"], "d_log_scales": self.grads["log_scales"],
               "d_quats": self.grads["quats"], "d_opacity_logit": self.grads["opacity_logit"],
               "d_sh": self.grads["sh"]}
        D.dass_preprocess_bwd(self.g, self.cams, fr.splats, fr.splat_grads, out, D.GRAD_ALL, rows=self.rows)
        b1, b2 = self.betas
        for k in ("means", "log_scales", "quats", "opacity_logit"):
            D.dass_adam(self._slice(k), self.grads[k], self.adam_m[k], self.adam_v[k], self.step,
                        [self.lr[k]] * self.grads[k].shape[1], b1, b2, self.eps, increment_step=False)
        # SH as [rows * K, 3]: the DC band and the higher bands take their own learning rates
        sh = self.g["sh"][self.n_base:self.n].reshape(-1, 3)
        gs, ms, vs = (t.view(-1, 3) for t in (self.grads["sh"], self.adam_m["sh"], self.adam_v["sh"]))
        D.dass_adam(sh, gs, ms, vs, self.step, [self.lr["sh_dc"]] * 3, b1, b2, self.eps, rows=self.sh_dc_rows,
                    increment_step=self.K == 1)
        if self.K > 1:
            D.dass_adam(sh, gs, ms, vs, self.step, [self.lr["sh_rest"]] * 3, b1, b2, self.eps,
                        rows=self.sh_rest_rows, increment_step=True)

    @property
    def loss(self):
        return float(self.loss_buf.item())

    def run(self, n_iters, max_regrow=2):
        """n_iters iterations; on pair-buffer overflow the var rows and optimiser state are restored
        and the stage reruns with twice the pair capacity."""
        snap = [self._slice(k).clone() for k in PARAM_NAMES]
        for _ in range(max_regrow + 1):
            try:
                self._run(n_iters)
                return
            except D.DassError as e:
                if e.status != D.ERR_CAPACITY:
                    raise
                for k, v in zip(PARAM_NAMES, snap):
                    self._slice(k).copy_(v)
                for d in (self.adam_m, self.adam_v):
                    for t in d.values():
                        t.zero_()
                self.step.zero_()
                self.overflow.zero_()
                self.frame._alloc_pairs(2 * self.frame.pair_capacity)
                self.graph = None
        raise D.DassError("densify stage bin_sort", D.ERR_CAPACITY)

    def _run(self, n_iters):
        if n_iters <= 0 or self.n == 0:
            return
        replays = n_iters
        if self.graph is None:
            self._iteration(eager=True)
            replays -= 1
            if replays > 0:
                m_pairs = int(self.frame.counters[0].item())
                # the var rows move and change size: keep 50% headroom over the pairs of the first render
                if self.frame.pair_capacity < int(m_pairs * 1.5) + 4096:
                    self.frame._alloc_pairs(int(m_pairs * 1.5) + 4096)
                torch.cuda.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self._iteration()
        for _ in range(replays):
            self.graph.replay()
        if replays > 0 and int(self.overflow.item()):
            raise D.DassError("densify stage bin_sort", D.ERR_CAPACITY)


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
    """One full timestep t of the streaming pipeline over resident device buffers.

    Scene arrays are allocated with room for `n_max` rows; `n` tracks the live count."""

    def __init__(self, cams, n_max, sh_degree, tile=16, batch=128, lambda_dssim=0.2, n_shift=100,
                 quantile=0.95, tau_pos=2e-4, tau_err=1e-4, k_max=5000, erase_every=20, n_inherit=0,
                 lambda_inher=1e-6, n_densify=0, prune_opacity=0.005, device="cuda"):
        self.cams = list(cams)
        self.n_max = int(n_max)
        self.deg = sh_degree
        self.tile, self.batch = tile, batch
        self.lambda_dssim = lambda_dssim
        self.n_shift = n_shift
        self.quantile, self.tau_pos, self.tau_err, self.k_max = quantile, tau_pos, tau_err, k_max
        self.erase_every = erase_every
        self.n_inherit, self.lambda_inher = int(n_inherit), float(lambda_inher)   # s1 of the inheritance stage
        self.n_densify, self.prune_opacity = int(n_densify), float(prune_opacity)  # s3 of the densification stage
        self.device = device
        K = (sh_degree + 1) ** 2
        shapes = dict(means=(3,), log_scales=(3,), quats=(4,), opacity_logit=(), sh=(K, 3))
        self.bufs = [{k: torch.zeros((self.n_max,) + s, device=device) for k, s in shapes.items()} for _ in range(2)]
        self.is_var = [torch.zeros(self.n_max, dtype=torch.uint8, device=device) for _ in range(2)]
        self.cur = 0
        self.n = 0

    def load(self, arrays: dict, is_var=None):
        n = int(arrays["means"].shape[0])
        assert n + self.k_max <= self.n_max
        for k in PARAM_NAMES:
            self.bufs[self.cur][k][:n].copy_(torch.as_tensor(arrays[k], dtype=torch.float32))
        self.is_var[self.cur].zero_()
        if is_var is not None:
            self.is_var[self.cur][:n].copy_(torch.as_tensor(is_var, dtype=torch.uint8))
        self.n = n

    def view(self, which=None):
        b = self.bufs[self.cur if which is None else which]
        return {k: v[:self.n] for k, v in b.items()}

    def run(self, t, targets, dyn_idx, offsets, inherit_logits=None, z=None, mode=D.STEP_BATCHED):
        """Reconstruct timestep t. Returns dict of per-stage results (loss, #Gaussians, #spawned)."""
        dev = self.device
        src, dst = self.cur, 1 - self.cur
        n = self.n
        # 1) selective inheritance (Sec. 3.2): learn the mask over the var rows (s1 iterations),
        #    unless the logits are given or this timestep erases every var row (App. B.2)
        erase = t % self.erase_every == 0
        if inherit_logits is None and self.n_inherit > 0 and not erase and n > 0 and bool(self.is_var[src][:n].any()):
            stage1 = InheritStage(self.view(src), self.is_var[src][:n], self.cams, targets, tile=self.tile,
                                  batch=self.batch, lambda_dssim=self.lambda_dssim, lambda_inher=self.lambda_inher)
            inherit_logits = stage1.run(self.n_inherit)[:n]
        m = inherit_logits if inherit_logits is not None else torch.ones(n, device=dev)
        ws = torch.empty(max(1, D.dass_inherit_workspace(n)), dtype=torch.uint8, device=dev)
        remap = torch.empty(max(1, n), dtype=torch.int32, device=dev)
        n_out = torch.zeros(1, dtype=torch.int64, device=dev)
        out = {k: v for k, v in self.bufs[dst].items()}
        D.dass_inherit(self.view(src), self.is_var[src][:n], m[:n].contiguous(), erase, out,
                       self.is_var[dst], remap, n_out, ws)
        self.cur = dst
        self.n = int(n_out.item())
        g = self.view()
        # dynamic rows follow the inherited layout (base rows keep their indices)
        dyn = dyn_idx
        # 2) shift stage
        stage = ShiftStage(g, self.cams, targets, dyn, offsets, tile=self.tile, batch=self.batch,
                           lambda_dssim=self.lambda_dssim)
        stage.run(self.n_shift, mode)
        # commit the shift into the scene (the learned offsets move the dynamic rows)
        D.dass_shift(dyn, stage.offsets, g["means"].clone(), g["quats"].clone(), g["means"], g["quats"])
        # 3) error-guided densification statistics, selection and spawn (Sec. 3.4)
        n = self.n
        s_err = torch.zeros(n, dtype=torch.uint8, device=dev)
        ews = torch.empty(D.dass_error_pass_workspace(self.cams), dtype=torch.uint8, device=dev)
        D.dass_error_pass(stage.frame.image, targets, self.cams, self.quantile, g["means"], self.is_var[self.cur][:n],
                          s_err, ews)
        sel = torch.empty(max(1, self.k_max), dtype=torch.int32, device=dev)
        nsel = torch.zeros(1, dtype=torch.int32, device=dev)
        sws = torch.empty(D.dass_densify_select_workspace(n), dtype=torch.uint8, device=dev)
        D.dass_densify_select(stage.stat_accum, stage.stat_count, s_err, self.is_var[self.cur][:n], self.tau_pos,
                              self.tau_err, self.k_max, sel, nsel, sws)
        if z is None:
            z = torch.zeros((n, 3), device=dev)
        n_total = torch.zeros(1, dtype=torch.int64, device=dev)
        D.dass_spawn({k: v for k, v in self.bufs[self.cur].items()}, n, self.is_var[self.cur], sel, nsel,
                     self.k_max, z[:n].contiguous(), n_total)
        self.n = int(n_total.item())
        spawned = int(nsel.item())
        out = dict(loss=stage.loss, n=self.n, spawned=spawned, stage=stage)
        # 4) densification-stage training of the var rows (Sec. 3.4, s3 iterations), then the
        #    low-opacity pruning of the var rows
        if self.n_densify > 0:
            out.update(self._densify(targets))
        return out

    def _densify(self, targets):
        n = self.n
        isv = self.is_var[self.cur][:n]
        n_base = int((isv == 0).sum().item())
        if n == n_base:
            return dict(densify_loss=None, pruned=0)
        if bool(isv[:n_base].any()) or not bool(isv[n_base:].all()):
            raise ValueError("densification stage needs the var rows as the contiguous tail of the arrays")
        stage3 = DensifyStage(self.view(), n_base, self.cams, targets, tile=self.tile, batch=self.batch,
                              lambda_dssim=self.lambda_dssim)
        stage3.run(self.n_densify)
        dev = self.device
        g = self.view()
        m = torch.empty(n, device=dev)
        D.dass_prune_logits(g["opacity_logit"], self.prune_opacity, m)
        src, dst = self.cur, 1 - self.cur
        ws = torch.empty(max(1, D.dass_inherit_workspace(n)), dtype=torch.uint8, device=dev)
        remap = torch.empty(n, dtype=torch.int32, device=dev)
        n_out = torch.zeros(1, dtype=torch.int64, device=dev)
        D.dass_inherit(g, isv, m, False, {k: v for k, v in self.bufs[dst].items()}, self.is_var[dst], remap, n_out, ws)
        self.cur = dst
        self.n = int(n_out.item())
        return dict(densify_loss=stage3.loss, pruned=n - self.n, n=self.n, densify_stage=stage3)
