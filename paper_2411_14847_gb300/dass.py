"""ctypes binding of libdass (include/dass.h): argument marshalling only.

Every function below has the name of its C entry point, takes torch CUDA tensors for the
device arrays and plain Python values for the rest, and raises DassError on a non-zero
status. All compute happens in libdass; torch only provides device memory and streams.
The library is loaded on first use; if it is missing the call fails (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdass.so")
_lib = None

MAX_CAMERAS = 64
GRAD_MEANS, GRAD_SCALES, GRAD_QUATS, GRAD_OPACITY, GRAD_SH = 1, 2, 4, 8, 16
GRAD_ALL = 31
STEP_BATCHED, STEP_PLAIN = 0, 1
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
SPLAT_FLOATS = 12   # sizeof(dass_splat) / 4
GRAD_FLOATS = 12    # sizeof(dass_splat_grad) / 4


class DassError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        detail = ""
        if _lib is not None:
            detail = _lib.dass_last_error().decode()
            name = _lib.dass_status_string(status).decode()
        else:
            name = str(status)
        super().__init__(f"{fn} failed: {name} ({status}) {detail}".strip())


class dass_camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class dass_step_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("sh_degree", C.c_int32), ("n_cams", C.c_int32),
        ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
        ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("cams", C.c_void_p), ("targets", C.c_void_p),
        ("n_dyn", C.c_int64), ("dyn_idx", C.c_void_p), ("dyn_mask", C.c_void_p), ("offsets", C.c_void_p),
        ("offset_grad", C.c_void_p),
        ("adam_m", C.c_void_p), ("adam_v", C.c_void_p), ("adam_step", C.c_void_p),
        ("lr_mu", C.c_float), ("lr_sigma", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
        ("eps", C.c_float), ("lambda_dssim", C.c_float),
        ("tile", C.c_int32), ("batch", C.c_int32),
        ("render_means", C.c_void_p), ("render_quats", C.c_void_p), ("d_means_dyn", C.c_void_p),
        ("d_quats_dyn", C.c_void_p), ("splats", C.c_void_p), ("splat_grads", C.c_void_p),
        ("pair_rec", C.c_void_p), ("pair_capacity", C.c_int64), ("tile_ranges", C.c_void_p),
        ("counters", C.c_void_p), ("image", C.c_void_p), ("T_final", C.c_void_p), ("n_last", C.c_void_p),
        ("dL_dimage", C.c_void_p), ("loss", C.c_void_p), ("stat_accum", C.c_void_p), ("stat_count", C.c_void_p),
        ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
    ]


_V, _F, _I32, _I64 = C.c_void_p, C.c_float, C.c_int32, C.c_int64
_RENDER_FIELDS = [("tile", _I32), ("batch", _I32), ("splats", _V), ("splat_grads", _V), ("pair_rec", _V),
                  ("pair_capacity", _I64), ("tile_ranges", _V), ("counters", _V), ("image", _V), ("T_final", _V),
                  ("n_last", _V), ("dL_dimage", _V), ("loss", _V), ("workspace", _V), ("workspace_bytes", C.c_size_t)]
_SCENE_FIELDS = [("n", _I64), ("sh_degree", _I32), ("n_cams", _I32), ("means", _V), ("log_scales", _V),
                 ("quats", _V), ("opacity_logit", _V), ("sh", _V)]


class dass_inherit_step_desc(C.Structure):
    _fields_ = _SCENE_FIELDS + [
        ("is_var", _V), ("cams", _V), ("targets", _V), ("n_var", _I64), ("var_rows", _V), ("m", _V), ("keep", _V),
        ("m_grad", _V), ("adam_m", _V), ("adam_v", _V), ("adam_step", _V), ("d_keep", _V),
        ("lr", _F), ("beta1", _F), ("beta2", _F), ("eps", _F), ("lambda_dssim", _F), ("lambda_inher", _F),
    ] + _RENDER_FIELDS


class dass_densify_step_desc(C.Structure):
    _fields_ = _SCENE_FIELDS + [
        ("n_base", _I64), ("is_var", _V), ("cams", _V), ("targets", _V), ("grad", _V), ("adam_m", _V),
        ("adam_v", _V), ("adam_step", _V),
        ("lr_means", _F), ("lr_log_scales", _F), ("lr_quats", _F), ("lr_opacity", _F), ("lr_sh_dc", _F),
        ("lr_sh_rest", _F), ("beta1", _F), ("beta2", _F), ("eps", _F), ("lambda_dssim", _F),
    ] + _RENDER_FIELDS


class dass_timestep_desc(C.Structure):
    _fields_ = [
        ("n_max", _I64), ("sh_degree", _I32), ("n_cams", _I32), ("means", _V), ("log_scales", _V), ("quats", _V),
        ("opacity_logit", _V), ("sh", _V), ("is_var", _V), ("n", _V), ("cams", _V), ("targets", _V),
        ("targets_host", _V), ("t", _I32), ("erase_every", _I32), ("n_dyn", _I64), ("dyn_idx", _V),
        ("offsets_init", _V), ("offsets", _V), ("z", _V),
        ("n_inherit", _I32), ("n_shift", _I32), ("n_densify", _I32), ("k_max", _I32), ("tile", _I32), ("batch", _I32),
        ("lambda_dssim", _F), ("lambda_inher", _F), ("inherit_m0", _F), ("quantile", _F), ("tau_pos", _F),
        ("tau_err", _F), ("prune_opacity", _F), ("lr_inherit", _F), ("lr_mu", _F), ("lr_sigma", _F),
        ("lr_means", _F), ("lr_log_scales", _F), ("lr_quats", _F), ("lr_opacity", _F), ("lr_sh_dc", _F),
        ("lr_sh_rest", _F), ("beta1", _F), ("beta2", _F), ("eps", _F),
        ("pair_capacity", _I64), ("workspace", _V), ("workspace_bytes", C.c_size_t),
        ("host_means", _V), ("host_log_scales", _V), ("host_quats", _V), ("host_opacity_logit", _V),
        ("host_sh", _V), ("host_is_var", _V), ("next_targets_host", _V), ("next_targets", _V),
    ]


class dass_timestep_stats(C.Structure):
    _fields_ = [("n_in", _I64), ("n_var_in", _I64), ("n_inherited", _I64), ("n_spawned", _I64),
                ("n_var_trained", _I64), ("n_out", _I64), ("pairs_max", _I64), ("erased", _I32),
                ("inherit_ran", _I32), ("loss_inherit", C.c_double), ("loss_shift", C.c_double),
                ("loss_densify", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dass_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("pad", C.c_int32), ("means", C.c_void_p),
                ("log_scales", C.c_void_p), ("quats", C.c_void_p), ("opacity_logit", C.c_void_p),
                ("sh", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "dass_version": (C.c_int, []),
    "dass_status_string": (C.c_char_p, [C.c_int]),
    "dass_last_error": (C.c_char_p, []),
    "dass_kernel_launches": (C.c_int64, []),
    "dass_tile_layout": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "dass_render_work": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P]),
    "dass_preprocess": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, C.c_int, C.c_int, _P, _P]),
    "dass_preprocess_scenes": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int64, _P, _P]),
    "dass_preprocess_scenes_packed": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P]),
    "dass_bin_sort_workspace": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, _P]),
    "dass_bin_sort_packed": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P, C.c_size_t, _P]),
    "dass_bin_sort": (C.c_int, [_P, C.c_int64, _P, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P, C.c_size_t, _P]),
    "dass_bin_sort_static": (C.c_int, [_P, C.c_int64, _P, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P]),
    "dass_bin_sort_split_workspace": (C.c_int, [C.c_int64, C.c_int, C.c_int64, _P]),
    "dass_bin_sort_split": (C.c_int, [_P, C.c_int64, _P, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P, _P,
                                      _P, _P, _P, C.c_size_t, _P]),
    "dass_bin_sort_merge_workspace": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, _P]),
    "dass_bin_sort_merge": (C.c_int, [_P, C.c_int64, _P, C.c_int, C.c_int, _P, _P, C.c_int64, _P, _P, _P, _P, _P,
                                      C.c_int64, _P, _P, _P, C.c_size_t, _P]),
    "dass_render_fwd": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]),
    "dass_tile_order": (C.c_int, [_P, C.c_int, _P, _P]),
    "dass_render_bwd": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, C.c_int64,
                                  _P, _P, _P]),
    "dass_preprocess_bwd": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P,
                                      C.c_int64, C.c_uint32, C.c_int, _P, _P, _P, _P, _P, _P]),
    "dass_keep_grad": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P, C.c_int64,
                                 _P, _P]),
    "dass_densify_stats": (C.c_int, [C.c_int64, _P, _P, _P, C.c_int, _P, _P, _P]),
    "dass_inherit_keep": (C.c_int, [C.c_int64, _P, _P, _P, _P]),
    "dass_field_fwd": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "dass_render_features": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, _P, C.c_int, C.c_int64, _P, _P]),
    "dass_object_ids": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P, C.c_int, _P, _P]),
    "dass_dynamic_objects": (C.c_int, [_P, _P, C.c_int64, C.c_int, C.c_uint32, _P, _P, _P]),
    "dass_dynamic_gaussians": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P, C.c_int, _P, _P, _P]),
    "dass_mask_rows_workspace": (C.c_int, [C.c_int64, _P]),
    "dass_mask_rows": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_size_t, _P]),
    "dass_field_bwd": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dass_prune_logits": (C.c_int, [C.c_int64, _P, C.c_float, _P, _P]),
    "dass_inherit_mask_grad": (C.c_int, [C.c_int64, _P, _P, _P, C.c_float, _P, _P, _P]),
    "dass_shift": (C.c_int, [C.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "dass_shift_bwd": (C.c_int, [C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dass_adam": (C.c_int, [C.c_int64, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_float, C.c_float,
                            C.c_float, C.c_int, _P]),
    "dass_loss_workspace": (C.c_int, [_P, C.c_int, _P]),
    "dass_loss": (C.c_int, [_P, _P, _P, C.c_int, C.c_float, _P, _P, _P, C.c_size_t, _P]),
    "dass_loss_target_stats": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "dass_loss_cached": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_float, _P, _P, _P, C.c_size_t, _P]),
    "dass_inherit_workspace": (C.c_int, [C.c_int64, _P]),
    "dass_inherit": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P, _P, _P, _P,
                               _P, _P, _P, C.c_size_t, _P]),
    "dass_error_pass_workspace": (C.c_int, [_P, C.c_int, _P]),
    "dass_error_pass": (C.c_int, [_P, _P, _P, C.c_int, C.c_float, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_size_t,
                                  _P]),
    "dass_densify_select_workspace": (C.c_int, [C.c_int64, _P]),
    "dass_densify_select": (C.c_int, [C.c_int64, _P, _P, _P, _P, C.c_float, C.c_float, C.c_int32, _P, _P, _P,
                                      C.c_size_t, _P]),
    "dass_spawn": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "dass_step_workspace": (C.c_int, [_P, _P]),
    "dass_step": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "dass_inherit_step_workspace": (C.c_int, [_P, _P]),
    "dass_inherit_step": (C.c_int, [_P, C.c_int, _P]),
    "dass_densify_step_workspace": (C.c_int, [_P, _P]),
    "dass_densify_step": (C.c_int, [_P, C.c_int, _P]),
    "dass_timestep_workspace": (C.c_int, [_P, _P]),
    "dass_timestep": (C.c_int, [_P, _P, _P]),
}


def load():
    """Open libdass.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdass.so not found at {LIB_PATH}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS.keys())


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != OK:
        raise DassError(name, st)
    return st


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


# Feature widths dass_render_features, dass_object_ids and dass_dynamic_gaussians accept.
FEATURE_WIDTHS = (4, 8, 16, 32)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def cameras(cams):
    """ctypes array of dass_camera from objects with viewmat/fx/fy/cx/cy/width/height; an array
    already built by this function is returned as it is (callers that issue several calls for the
    same cameras marshal them once)."""
    if isinstance(cams, C.Array) and getattr(cams, "_type_", None) is dass_camera:
        return cams
    arr = (dass_camera * len(cams))()
    for i, c in enumerate(cams):
        vm = np.asarray(c.viewmat, dtype=np.float32).reshape(-1)
        arr[i].viewmat[:] = [float(v) for v in vm]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def tile_layout(cams, tile):
    arr = cameras(cams)
    t = C.c_int32()
    p = C.c_int64()
    _call("dass_tile_layout", arr, len(cams), tile, C.byref(t), C.byref(p))
    return t.value, p.value


# ----------------------------------------------------------------- raw entry points

F32, I32, U8, I64, F64 = torch.float32, torch.int32, torch.uint8, torch.int64, torch.float64


def dass_preprocess(g, cams, tile, splats, keep=None, stream=None):
    n = g["means"].shape[0]
    deg = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    arr = cameras(cams)
    _call("dass_preprocess", n, deg, _ptr(g["means"], F32), _ptr(g["log_scales"], F32), _ptr(g["quats"], F32),
          _ptr(g["opacity_logit"], F32), _ptr(g["sh"], F32), _ptr(keep, U8), arr, len(cams), tile,
          _ptr(splats, F32), _stream(stream))


def dass_preprocess_scenes(scenes, cams, tile, rec_stride, splats, stream=None):
    """scenes: one dict of Gaussian tensors per camera (same SH degree)."""
    _call("dass_preprocess_scenes", _scene_array(scenes), cameras(cams), len(cams), tile, rec_stride,
          _ptr(splats, F32), _stream(stream))


def _scene_array(scenes):
    arr = (dass_scene * len(scenes))()
    for i, g in enumerate(scenes):
        arr[i].n = g["means"].shape[0]
        arr[i].sh_degree = int(round(math.sqrt(g["sh"].shape[1]))) - 1
        for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            setattr(arr[i], name, _ptr(g[name], F32).value)
    return arr


def record_offsets(scenes):
    """Host int64 array [len(scenes) + 1] of packed record segments: 0, n_0, n_0 + n_1, ..."""
    off = (C.c_int64 * (len(scenes) + 1))()
    for i, g in enumerate(scenes):
        off[i + 1] = off[i] + int(g["means"].shape[0])
    return off


def dass_preprocess_scenes_packed(scenes, cams, tile, rec_offsets, splats, stream=None):
    """scenes: one dict of Gaussian tensors per camera; rec_offsets from record_offsets(scenes)."""
    _call("dass_preprocess_scenes_packed", _scene_array(scenes), cameras(cams), len(cams), tile, rec_offsets,
          _ptr(splats, F32), _stream(stream))


def dass_bin_sort_packed(splats, rec_offsets, cams, tile, pair_rec, tile_ranges, counters, workspace, stream=None):
    _call("dass_bin_sort_packed", _ptr(splats, F32), rec_offsets, cameras(cams), len(cams), tile,
          _ptr(pair_rec, I32), pair_rec.numel(), _ptr(tile_ranges, I32), _ptr(counters, I64), _ptr(workspace, U8),
          workspace.numel(), _stream(stream))


def dass_bin_sort_workspace(n_records, pair_capacity, tiles_total):
    b = C.c_size_t()
    _call("dass_bin_sort_workspace", n_records, pair_capacity, tiles_total, C.byref(b))
    return b.value


def dass_bin_sort(splats, rec_stride, cams, tile, pair_rec, tile_ranges, counters, workspace, stream=None):
    arr = cameras(cams)
    _call("dass_bin_sort", _ptr(splats, F32), rec_stride, arr, len(cams), tile, _ptr(pair_rec, I32),
          pair_rec.numel(), _ptr(tile_ranges, I32), _ptr(counters, I64), _ptr(workspace, U8), workspace.numel(),
          _stream(stream))


def dass_bin_sort_static(splats, rec_stride, cams, tile, pair_rec, tile_ranges, counters, stream=None):
    """dass_bin_sort without a workspace (static device scratch; see include/dass.h)."""
    arr = cameras(cams)
    _call("dass_bin_sort_static", _ptr(splats, F32), rec_stride, arr, len(cams), tile, _ptr(pair_rec, I32),
          pair_rec.numel(), _ptr(tile_ranges, I32), _ptr(counters, I64), _stream(stream))


def dass_bin_sort_split_workspace(n_rows, n_cams, pair_capacity):
    b = C.c_size_t(0)
    _call("dass_bin_sort_split_workspace", n_rows, n_cams, pair_capacity, C.byref(b))
    return b.value


def dass_bin_sort_split(splats, n_rows, cams, tile, moving, static_rec, static_depth, tile_start, static_counters,
                        moving_rec, n_moving_rec, moving_rows, n_moving_rows, workspace, stream=None):
    """Static lists of an incremental binning (every row not flagged in `moving`); see include/dass.h."""
    _call("dass_bin_sort_split", _ptr(splats, F32), n_rows, cameras(cams), len(cams), tile, _ptr(moving, U8),
          static_rec.numel(), _ptr(static_rec, I32), _ptr(static_depth, I32), _ptr(tile_start, I32),
          _ptr(static_counters, I64), _ptr(moving_rec, I32), _ptr(n_moving_rec, I64), _ptr(moving_rows, I32),
          _ptr(n_moving_rows, I64), _ptr(workspace, U8), workspace.numel(), _stream(stream))


def dass_bin_sort_merge_workspace(moving_capacity, pair_capacity, tiles_total):
    b = C.c_size_t(0)
    _call("dass_bin_sort_merge_workspace", moving_capacity, pair_capacity, tiles_total, C.byref(b))
    return b.value


def dass_bin_sort_merge(splats, n_rows, cams, tile, moving_rec, n_moving_rec, moving_capacity, static_rec,
                        static_depth, tile_start, static_counters, pair_rec, tile_ranges, counters, workspace,
                        stream=None):
    """The moving rows' pairs merged into the static lists: dass_bin_sort's outputs; see include/dass.h."""
    _call("dass_bin_sort_merge", _ptr(splats, F32), n_rows, cameras(cams), len(cams), tile, _ptr(moving_rec, I32),
          _ptr(n_moving_rec, I64), moving_capacity, _ptr(static_rec, I32), _ptr(static_depth, I32),
          _ptr(tile_start, I32), _ptr(static_counters, I64), _ptr(pair_rec, I32), pair_rec.numel(),
          _ptr(tile_ranges, I32), _ptr(counters, I64), _ptr(workspace, U8), workspace.numel(), _stream(stream))


def dass_render_fwd(splats, pair_rec, tile_ranges, cams, tile, batch, image, T_final, n_last, bg=None, order=None,
                    stream=None):
    arr = cameras(cams)
    bgp = (C.c_float * 3)(*bg) if bg is not None else None
    _call("dass_render_fwd", _ptr(splats, F32), _ptr(pair_rec, I32), _ptr(tile_ranges, I32), arr, len(cams), tile,
          batch, bgp, _ptr(image, F32), _ptr(T_final, F32), _ptr(n_last, I32), _ptr(order, I32), _stream(stream))


def dass_tile_order(tile_ranges, order, stream=None):
    """order: int32 CUDA tensor of tile_ranges.shape[0] entries (a permutation, longest lists first)."""
    _call("dass_tile_order", _ptr(tile_ranges, I32), int(order.numel()), _ptr(order, I32), _stream(stream))


def dass_kernel_launches():
    return int(load().dass_kernel_launches())


def dass_render_work(splats, pair_rec, tile_ranges, cams, tile, batch, image, T_final, n_last, work, full_grad=None,
                     rec_stride=0, stream=None):
    """work: int64 CUDA tensor of 5 (counts, see include/dass.h)."""
    arr = cameras(cams)
    _call("dass_render_work", _ptr(splats, F32), _ptr(pair_rec, I32), _ptr(tile_ranges, I32), arr, len(cams), tile,
          batch, _ptr(full_grad, U8), rec_stride, _ptr(image, F32), _ptr(T_final, F32), _ptr(n_last, I32),
          _ptr(work, I64), _stream(stream))


def dass_render_bwd(splats, pair_rec, tile_ranges, cams, tile, batch, T_final, n_last, dL_dimage, splat_grads,
                    bg=None, full_grad=None, rec_stride=0, order=None, stream=None):
    arr = cameras(cams)
    bgp = (C.c_float * 3)(*bg) if bg is not None else None
    _call("dass_render_bwd", _ptr(splats, F32), splat_grads.numel() // GRAD_FLOATS, _ptr(pair_rec, I32),
          _ptr(tile_ranges, I32), arr, len(cams), tile, batch, bgp, _ptr(T_final, F32), _ptr(n_last, I32),
          _ptr(dL_dimage, F32), _ptr(full_grad, U8), rec_stride, _ptr(splat_grads, F32), _ptr(order, I32),
          _stream(stream))


def dass_preprocess_bwd(g, cams, splats, splat_grads, out, grad_flags=GRAD_ALL, rows=None, accumulate=False,
                        keep=None, stream=None):
    """out: dict with any of d_means, d_log_scales, d_quats, d_opacity_logit, d_sh tensors."""
    n = g["means"].shape[0]
    deg = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    arr = cameras(cams)
    n_rows = rows.numel() if rows is not None else n
    _call("dass_preprocess_bwd", n, deg, _ptr(g["means"], F32), _ptr(g["log_scales"], F32), _ptr(g["quats"], F32),
          _ptr(g["opacity_logit"], F32), _ptr(g["sh"], F32), _ptr(keep, U8), arr, len(cams), _ptr(splats, F32),
          _ptr(splat_grads, F32), _ptr(rows, I32), n_rows, grad_flags, int(bool(accumulate)),
          _ptr(out.get("d_means"), F32), _ptr(out.get("d_log_scales"), F32), _ptr(out.get("d_quats"), F32),
          _ptr(out.get("d_opacity_logit"), F32), _ptr(out.get("d_sh"), F32), _stream(stream))


def dass_keep_grad(g, cams, splats, splat_grads, d_keep, keep=None, rows=None, stream=None):
    """dL/dkeep of the inheritance mask per row (compact [n_rows] when rows is given)."""
    n = g["means"].shape[0]
    deg = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    arr = cameras(cams)
    n_rows = rows.numel() if rows is not None else n
    _call("dass_keep_grad", n, deg, _ptr(g["means"], F32), _ptr(g["log_scales"], F32), _ptr(g["quats"], F32),
          _ptr(g["opacity_logit"], F32), _ptr(g["sh"], F32), _ptr(keep, U8), arr, len(cams), _ptr(splats, F32),
          _ptr(splat_grads, F32), _ptr(rows, I32), n_rows, _ptr(d_keep, F32), _stream(stream))


def dass_render_features(splats, pair_rec, tile_ranges, cams, tile, features, rec_stride, out, stream=None):
    """features: [n, F] per Gaussian (F in 4, 8, 16, 32); out: [pixels_total, F]."""
    arr = cameras(cams)
    _call("dass_render_features", _ptr(splats, F32), _ptr(pair_rec, I32), _ptr(tile_ranges, I32), arr, len(cams),
          tile, _ptr(features, F32), int(features.shape[1]), rec_stride, _ptr(out, F32), _stream(stream))


def dass_object_ids(x, W, b, ids, stream=None):
    _call("dass_object_ids", _ptr(x, F32), x.shape[0], int(x.shape[1]), _ptr(W, F32), _ptr(b, F32), int(W.shape[0]),
          _ptr(ids, I32), _stream(stream))


def dass_dynamic_objects(ids, dyn_area, n_classes, min_pixels, obj_mask, hist, stream=None):
    _call("dass_dynamic_objects", _ptr(ids, I32), _ptr(dyn_area, U8), ids.numel(), int(n_classes), int(min_pixels),
          _ptr(obj_mask, U8), _ptr(hist, I32), _stream(stream))


def dass_dynamic_gaussians(features, W, b, obj_mask, dyn_mask, stream=None):
    _call("dass_dynamic_gaussians", _ptr(features, F32), features.shape[0], int(features.shape[1]), _ptr(W, F32),
          _ptr(b, F32), int(W.shape[0]), _ptr(obj_mask, U8), _ptr(dyn_mask, U8), _stream(stream))


def dass_mask_rows_workspace(n):
    b = C.c_size_t()
    _call("dass_mask_rows_workspace", n, C.byref(b))
    return b.value


def dass_mask_rows(mask, rows, count, workspace, stream=None):
    _call("dass_mask_rows", _ptr(mask, U8), mask.numel(), _ptr(rows, I32), _ptr(count, I64), _ptr(workspace, U8),
          workspace.numel(), _stream(stream))


class dass_field(C.Structure):
    _fields_ = [("levels", C.c_int32), ("features", C.c_int32), ("log2_table", C.c_int32), ("hidden", C.c_int32),
                ("res", C.c_int32 * 16), ("bbox_min", C.c_float * 3), ("bbox_max", C.c_float * 3),
                ("table", C.c_void_p), ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p),
                ("b2", C.c_void_p)]


def field_struct(p: dict, res, log2_table, bbox_min, bbox_max):
    """dass_field over parameter tensors p = {table [L][T][F], w1 [H][L*F], b1 [H], w2 [7][H], b2 [7]}."""
    f = dass_field()
    f.levels, f.features = int(p["table"].shape[0]), int(p["table"].shape[2])
    f.log2_table, f.hidden = int(log2_table), int(p["w1"].shape[0])
    for i, r in enumerate(res):
        f.res[i] = int(r)
    for d in range(3):
        f.bbox_min[d], f.bbox_max[d] = float(bbox_min[d]), float(bbox_max[d])
    for k in ("table", "w1", "b1", "w2", "b2"):
        assert p[k].is_cuda and p[k].dtype == torch.float32 and p[k].is_contiguous(), k
        setattr(f, k, p[k].data_ptr())
    return f


def dass_field_fwd(field, means, offsets, rows=None, stream=None):
    n_rows = rows.numel() if rows is not None else means.shape[0]
    _call("dass_field_fwd", C.byref(field), n_rows, _ptr(rows, I32), _ptr(means, F32), _ptr(offsets, F32),
          _stream(stream))


def dass_field_bwd(field, means, d_offsets, grads, rows=None, stream=None):
    """grads: dict of tensors table, w1, b1, w2, b2 (accumulated into)."""
    n_rows = rows.numel() if rows is not None else means.shape[0]
    _call("dass_field_bwd", C.byref(field), n_rows, _ptr(rows, I32), _ptr(means, F32), _ptr(d_offsets, F32),
          _ptr(grads["table"], F32), _ptr(grads["w1"], F32), _ptr(grads["b1"], F32), _ptr(grads["w2"], F32),
          _ptr(grads["b2"], F32), _stream(stream))


def dass_prune_logits(opacity_logit, min_opacity, m, stream=None):
    _call("dass_prune_logits", opacity_logit.numel(), _ptr(opacity_logit, F32), float(min_opacity), _ptr(m, F32),
          _stream(stream))


def dass_inherit_keep(is_var, m, keep, stream=None):
    _call("dass_inherit_keep", is_var.numel(), _ptr(is_var, U8), _ptr(m, F32), _ptr(keep, U8), _stream(stream))


def dass_inherit_mask_grad(rows, m, d_keep, lambda_inher, grad, loss=None, stream=None):
    n_rows = rows.numel() if rows is not None else m.numel()
    _call("dass_inherit_mask_grad", n_rows, _ptr(rows, I32), _ptr(m, F32), _ptr(d_keep, F32), float(lambda_inher),
          _ptr(grad, F32), _ptr(loss, F64), _stream(stream))


def dass_densify_stats(n, splats, splat_grads, cams, accum, count, stream=None):
    arr = cameras(cams)
    _call("dass_densify_stats", n, _ptr(splats, F32), _ptr(splat_grads, F32), arr, len(cams), _ptr(accum, F32),
          _ptr(count, I32), _stream(stream))


def dass_shift(dyn_idx, offsets, means, quats, out_means, out_quats, stream=None):
    _call("dass_shift", dyn_idx.numel(), _ptr(dyn_idx, I32), _ptr(offsets, F32), _ptr(means, F32), _ptr(quats, F32),
          _ptr(out_means, F32), _ptr(out_quats, F32), _stream(stream))


def dass_shift_bwd(dyn_idx, offsets, quats, d_out_means, d_out_quats, d_offsets, d_quats=None, stream=None):
    _call("dass_shift_bwd", dyn_idx.numel(), _ptr(dyn_idx, I32), _ptr(offsets, F32), _ptr(quats, F32),
          _ptr(d_out_means, F32), _ptr(d_out_quats, F32), _ptr(d_offsets, F32), _ptr(d_quats, F32), _stream(stream))


def dass_adam(param, grad, m, v, step_dev, lr, beta1=0.9, beta2=0.999, eps=1e-15, rows=None, increment_step=True,
              stream=None):
    """param/grad/m/v: [n_rows, width]; lr: list of width learning rates."""
    n_rows, width = param.shape
    lra = (C.c_float * width)(*[float(x) for x in lr])
    _call("dass_adam", n_rows, width, _ptr(rows, I32), rows.numel() if rows is not None else n_rows,
          _ptr(param, F32), _ptr(grad, F32), _ptr(m, F32), _ptr(v, F32), _ptr(step_dev, I32), lra, beta1, beta2, eps,
          int(bool(increment_step)), _stream(stream))


def dass_loss_workspace(cams):
    arr = cameras(cams)
    b = C.c_size_t()
    _call("dass_loss_workspace", arr, len(cams), C.byref(b))
    return b.value


def dass_loss(image, target, cams, lam, dL_dimage, loss, workspace, stream=None):
    arr = cameras(cams)
    _call("dass_loss", _ptr(image, F32), _ptr(target, F32), arr, len(cams), lam, _ptr(dL_dimage, F32),
          _ptr(loss, F64), _ptr(workspace, U8), workspace.numel() if workspace is not None else 0, _stream(stream))


def dass_loss_target_stats(target, cams, stats, stream=None):
    arr = cameras(cams)
    _call("dass_loss_target_stats", _ptr(target, F32), arr, len(cams), _ptr(stats, F32), _stream(stream))


def dass_loss_cached(image, target, target_stats, cams, lam, dL_dimage, loss, workspace, stream=None):
    arr = cameras(cams)
    _call("dass_loss_cached", _ptr(image, F32), _ptr(target, F32), _ptr(target_stats, F32), arr, len(cams), lam,
          _ptr(dL_dimage, F32), _ptr(loss, F64), _ptr(workspace, U8), workspace.numel() if workspace is not None else 0,
          _stream(stream))


def dass_inherit_workspace(n):
    b = C.c_size_t()
    _call("dass_inherit_workspace", n, C.byref(b))
    return b.value


def dass_inherit(g, is_var, m, erase, out, is_var_out, remap, n_out, workspace, stream=None):
    n = g["means"].shape[0]
    deg = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    _call("dass_inherit", n, deg, _ptr(g["means"], F32), _ptr(g["log_scales"], F32), _ptr(g["quats"], F32),
          _ptr(g["opacity_logit"], F32), _ptr(g["sh"], F32), _ptr(is_var, U8), _ptr(m, F32), int(bool(erase)),
          _ptr(out["means"], F32), _ptr(out["log_scales"], F32), _ptr(out["quats"], F32),
          _ptr(out["opacity_logit"], F32), _ptr(out["sh"], F32), _ptr(is_var_out, U8), _ptr(remap, I32),
          _ptr(n_out, I64), _ptr(workspace, U8), workspace.numel(), _stream(stream))


def dass_error_pass_workspace(cams):
    arr = cameras(cams)
    b = C.c_size_t()
    _call("dass_error_pass_workspace", arr, len(cams), C.byref(b))
    return b.value


def dass_error_pass(image, target, cams, quantile, means, is_var, s_err, workspace, error_map=None, gamma=None,
                    stream=None):
    arr = cameras(cams)
    n = means.shape[0] if means is not None else 0
    _call("dass_error_pass", _ptr(image, F32), _ptr(target, F32), arr, len(cams), quantile, n, _ptr(means, F32),
          _ptr(is_var, U8), _ptr(error_map, F32), _ptr(gamma, F32), _ptr(s_err, U8), _ptr(workspace, U8),
          workspace.numel(), _stream(stream))


def dass_densify_select_workspace(n):
    b = C.c_size_t()
    _call("dass_densify_select_workspace", n, C.byref(b))
    return b.value


def dass_densify_select(accum, count, s_err, is_var, tau_pos, tau_err, k_max, selected, n_selected, workspace,
                        stream=None):
    _call("dass_densify_select", accum.numel(), _ptr(accum, F32), _ptr(count, I32), _ptr(s_err, U8),
          _ptr(is_var, U8), tau_pos, tau_err, k_max, _ptr(selected, I32), _ptr(n_selected, I32),
          _ptr(workspace, U8), workspace.numel(), _stream(stream))


def dass_spawn(g, n, is_var, selected, n_selected, k_max, z, n_total, stream=None):
    deg = int(round(math.sqrt(g["sh"].shape[1]))) - 1
    _call("dass_spawn", n, deg, _ptr(g["means"], F32), _ptr(g["log_scales"], F32), _ptr(g["quats"], F32),
          _ptr(g["opacity_logit"], F32), _ptr(g["sh"], F32), _ptr(is_var, U8), _ptr(selected, I32),
          _ptr(n_selected, I32), k_max, _ptr(z, F32), _ptr(n_total, I64), _stream(stream))


def dass_step_workspace(desc):
    b = C.c_size_t()
    _call("dass_step_workspace", C.byref(desc), C.byref(b))
    return b.value


def dass_step(desc, n_iters, mode=STEP_BATCHED, stream=None):
    lib = load()
    st = lib.dass_step(C.byref(desc), n_iters, mode, _stream(stream))
    if st not in (OK, ERR_CAPACITY):
        raise DassError("dass_step", st)
    return st


def dass_inherit_step_workspace(desc):
    b = C.c_size_t()
    _call("dass_inherit_step_workspace", C.byref(desc), C.byref(b))
    return b.value


def dass_inherit_step(desc, n_iters, stream=None):
    """Returns OK or ERR_CAPACITY (pair overflow in some iteration); raises on other errors."""
    st = load().dass_inherit_step(C.byref(desc), n_iters, _stream(stream))
    if st not in (OK, ERR_CAPACITY):
        raise DassError("dass_inherit_step", st)
    return st


def dass_densify_step_workspace(desc):
    b = C.c_size_t()
    _call("dass_densify_step_workspace", C.byref(desc), C.byref(b))
    return b.value


def dass_densify_step(desc, n_iters, stream=None):
    """Returns OK or ERR_CAPACITY (pair overflow in some iteration); raises on other errors."""
    st = load().dass_densify_step(C.byref(desc), n_iters, _stream(stream))
    if st not in (OK, ERR_CAPACITY):
        raise DassError("dass_densify_step", st)
    return st


def dass_timestep_workspace(desc):
    b = C.c_size_t()
    _call("dass_timestep_workspace", C.byref(desc), C.byref(b))
    return b.value


def dass_timestep(desc, stream=None):
    """Returns (status, stats): status OK or ERR_CAPACITY (G_{t-1} left unchanged); raises on other
    errors."""
    stats = dass_timestep_stats()
    st = load().dass_timestep(C.byref(desc), C.byref(stats), _stream(stream))
    if st not in (OK, ERR_CAPACITY):
        raise DassError("dass_timestep", st)
    return st, stats
