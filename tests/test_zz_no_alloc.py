"""dass_bin_sort_static: binning for callers that cannot allocate device memory.

Some callers own every device allocation through their own pool, or cannot afford an
allocation on their calling path; for them dass_bin_sort_static takes the same inputs and
outputs as dass_bin_sort but keeps its scratch in a fixed device array inside the library.
This file checks, through the C ABI, that two calls in a row give exactly the outputs of
dass_bin_sort with a caller-provided workspace (tile lists are integer work: bit-exact), and
that a request larger than the static array is refused without launching.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_14847_gb300 import synth

pytestmark = pytest.mark.gpu


def _records(n_cams, n, seed, width, height):
    rng = np.random.default_rng(seed)
    R = n_cams * n
    rec = np.zeros((R, 12), np.float32)
    rec[:, 0] = rng.uniform(-20, width + 20, R)
    rec[:, 1] = rng.uniform(-20, height + 20, R)
    sx, sy = rng.uniform(0.5, 7.0, R), rng.uniform(0.5, 7.0, R)      # footprint axes in pixels
    th = rng.uniform(0, np.pi, R)
    c, s = np.cos(th), np.sin(th)
    cxx, cyy = c * c * sx * sx + s * s * sy * sy, s * s * sx * sx + c * c * sy * sy
    cxy = c * s * (sx * sx - sy * sy)
    det = cxx * cyy - cxy * cxy
    rec[:, 2], rec[:, 3], rec[:, 4] = cyy / det, -cxy / det, cxx / det   # conic = covariance^-1
    rec[:, 5] = rng.uniform(0.05, 1.0, R)                              # opacity
    rec[:, 9] = rng.integers(1, 200, R).astype(np.float32) * 0.05        # depth ties included
    rad = np.full(R, 30, np.int32)
    rad[rng.uniform(size=R) < 0.1] = 0
    rec[:, 10] = rad.view(np.float32)
    return torch.from_numpy(rec).cuda()


def _outputs(cap, tiles_total):
    return (torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
            torch.full((tiles_total, 2), -7, dtype=torch.int32, device="cuda"),
            torch.zeros(4, dtype=torch.int64, device="cuda"))


def test_static_scratch_matches_workspace_version_twice(dass):
    lib = dass.load()
    cases = [(3, 40_000, 11, 640, 360, 16), (2, 15_000, 12, 320, 200, 8)]   # second call is smaller
    for n_cams, n, seed, w, h, tile in cases:
        cams = synth.arc_cameras(n_cams, 4.0, w, h)
        splats = _records(n_cams, n, seed, w, h)
        tiles_total, _ = dass.tile_layout(cams, tile)
        cap = 2_000_000
        ref_pairs, ref_ranges, ref_cnt = _outputs(cap, tiles_total)
        ws = torch.empty(dass.dass_bin_sort_workspace(n_cams * n, cap, tiles_total), dtype=torch.uint8,
                         device="cuda")
        dass.dass_bin_sort(splats, n, cams, tile, ref_pairs, ref_ranges, ref_cnt, ws)
        pairs, ranges, cnt = _outputs(cap, tiles_total)
        arr = dass.cameras(cams)
        st = lib.dass_bin_sort_static(C.c_void_p(splats.data_ptr()), n, arr, n_cams, tile,
                                      C.c_void_p(pairs.data_ptr()), cap, C.c_void_p(ranges.data_ptr()),
                                      C.c_void_p(cnt.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, lib.dass_last_error()
        torch.cuda.synchronize()
        m = int(ref_cnt[0])
        assert m > 100_000 and int(ref_cnt[1]) == 0
        assert torch.equal(cnt[:3], ref_cnt[:3])
        assert torch.equal(pairs[:m], ref_pairs[:m])
        assert torch.equal(ranges, ref_ranges)


def test_static_scratch_rejects_oversized_request(dass):
    lib = dass.load()
    cams = synth.arc_cameras(2, 4.0, 64, 48)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    arr = dass.cameras(cams)
    # 2 x 4M records need far more than the static array
    st = lib.dass_bin_sort_static(p, 4_000_000, arr, 2, 16, p, 1_000_000, p, C.c_void_p(cnt.data_ptr()), None)
    assert st == dass.ERR_OOM
    assert b"DASS_BIN_SORT_STATIC_BYTES" in lib.dass_last_error()
    torch.cuda.synchronize()
    assert int(cnt.abs().sum()) == 0
