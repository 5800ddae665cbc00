"""Incremental binning (dass_bin_sort_split + dass_bin_sort_merge): a stage of Sec. 3.2-3.4 trains
only some rows, so the other rows' pairs are binned and sorted once and every iteration merges the
moving rows' pairs into them. Checked against the full binning dass_bin_sort of the same records:
pair lists, tile ranges and counters equal element by element, at tiles 8/16/32, with exact depth
ties between static and moving records, moving sets that are empty, partial and complete, moved
records that change tiles, and a pair buffer too small for the merged list."""
import numpy as np
import pytest
import torch

from paper_2411_14847_gb300 import synth

from test_gpu_render import _synthetic_records

pytestmark = pytest.mark.gpu

I32, I64, U8 = torch.int32, torch.int64, torch.uint8


def _full(cams, n, tile, rec, cap):
    from paper_2411_14847_gb300 import raster
    fr = raster.Frame(cams, n, tile=tile, batch=128, pair_capacity=cap)
    fr.splats.copy_(torch.from_numpy(rec))
    m = fr.bin_sort()
    return fr, m


def _split(D, fr, n, cams, tile, moving, cap):
    s = dict(rec=torch.full((cap,), -1, dtype=I32, device="cuda"),
             depth=torch.zeros(cap, dtype=I32, device="cuda"),
             start=torch.zeros(fr.tiles_total + 1, dtype=I32, device="cuda"),
             counters=torch.zeros(4, dtype=I64, device="cuda"),
             moving_rec=torch.zeros(len(cams) * n, dtype=I32, device="cuda"),
             n_moving_rec=torch.zeros(1, dtype=I64, device="cuda"),
             rows=torch.zeros(n, dtype=I32, device="cuda"),
             n_rows=torch.zeros(1, dtype=I64, device="cuda"))
    ws = torch.empty(D.dass_bin_sort_split_workspace(n, len(cams), cap), dtype=U8, device="cuda")
    D.dass_bin_sort_split(fr.splats, n, cams, tile, moving, s["rec"], s["depth"], s["start"], s["counters"],
                          s["moving_rec"], s["n_moving_rec"], s["rows"], s["n_rows"], ws)
    return s


def _merge(D, fr, n, cams, tile, s, moving_cap, cap):
    pair_rec = torch.full((cap,), -1, dtype=I32, device="cuda")
    ranges = torch.full((fr.tiles_total, 2), -7, dtype=I32, device="cuda")
    counters = torch.full((4,), -5, dtype=I64, device="cuda")
    ws = torch.empty(D.dass_bin_sort_merge_workspace(moving_cap, cap, fr.tiles_total), dtype=U8, device="cuda")
    D.dass_bin_sort_merge(fr.splats, n, cams, tile, s["moving_rec"], s["n_moving_rec"], moving_cap, s["rec"],
                          s["depth"], s["start"], s["counters"], pair_rec, ranges, counters, ws)
    return pair_rec, ranges, counters


def _moved(rec, n, n_cams, rows, seed):
    """The records of `rows` in every camera moved on screen (other tiles), resized and given depths
    from the same small set as the static records (exact ties across the two lists)."""
    rng = np.random.default_rng(seed)
    out = rec.copy()
    for c in range(n_cams):
        r = c * n + rows
        out[r, 0] += rng.uniform(-25, 25, r.size).astype(np.float32)
        out[r, 1] += rng.uniform(-25, 25, r.size).astype(np.float32)
        out[r, 5] = rng.uniform(0.02, 1.0, r.size).astype(np.float32)
        out[r, 9] = rng.integers(1, 40, r.size).astype(np.float32) * 0.25
    return out


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("frac", [0.0, 0.15, 1.0])
def test_merge_equals_full_binning(dass, tile, frac):
    from paper_2411_14847_gb300 import dass as D
    cams = synth.arc_cameras(3, 4.0, 100, 70)
    n = 1500
    rec, _ = _synthetic_records(len(cams), n, 5, 100, 70)
    rng = np.random.default_rng(6)
    rows = np.sort(rng.choice(n, int(frac * n), replace=False)).astype(np.int64)
    mask = np.zeros(n, np.uint8)
    mask[rows] = 1
    cap = 8 * len(cams) * n
    fr0, m0 = _full(cams, n, tile, rec, cap)
    s = _split(D, fr0, n, cams, tile, torch.as_tensor(mask).cuda(), cap)
    torch.cuda.synchronize()
    assert int(s["n_rows"].item()) == rows.size and int(s["n_moving_rec"].item()) == rows.size * len(cams)
    assert np.array_equal(s["rows"][:rows.size].cpu().numpy(), rows)
    want_list = np.concatenate([c * n + rows for c in range(len(cams))]) if rows.size else np.zeros(0)
    assert np.array_equal(s["moving_rec"][:want_list.size].cpu().numpy(), want_list)
    # the static lists: the full binning's lists without the moving records, with their depth keys
    ms = int(s["counters"][2].item())
    assert int(s["counters"][1].item()) == 0
    moving_rec = set(want_list.tolist())
    keep = np.array([r not in moving_rec for r in fr0.pair_rec[:m0].cpu().numpy().tolist()], dtype=bool)
    assert ms == int(keep.sum())
    assert np.array_equal(s["rec"][:ms].cpu().numpy(), fr0.pair_rec[:m0].cpu().numpy()[keep])
    assert np.array_equal(s["depth"][:ms].cpu().numpy().view(np.float32), rec[s["rec"][:ms].cpu().numpy(), 9])
    for case, recs in (("unmoved", rec), ("moved", _moved(rec, n, len(cams), rows, 7))):
        fr, m = _full(cams, n, tile, recs, cap)
        pr, rg, ct = _merge(D, fr, n, cams, tile, s, max(1, rows.size * len(cams)), cap)
        torch.cuda.synchronize()
        assert int(fr.counters[1].item()) == 0 and m > 0
        assert ct[:3].tolist() == fr.counters[:3].tolist(), case
        assert torch.equal(pr[:m], fr.pair_rec[:m]), case
        assert torch.equal(rg, fr.tile_ranges), case


def test_merge_overflow_flag_and_clamped_ranges(dass):
    """A pair buffer smaller than the merged list: counters[0] the full count, counters[1] = 1,
    counters[2] = the capacity; every range inside the capacity and every stored record valid."""
    from paper_2411_14847_gb300 import dass as D
    cams = synth.arc_cameras(2, 4.0, 100, 70)
    n = 1200
    rec, _ = _synthetic_records(len(cams), n, 8, 100, 70)
    rows = np.arange(0, n, 5)
    mask = np.zeros(n, np.uint8)
    mask[rows] = 1
    big = 8 * len(cams) * n
    fr, m = _full(cams, n, 16, rec, big)
    s = _split(D, fr, n, cams, 16, torch.as_tensor(mask).cuda(), big)
    torch.cuda.synchronize()
    ms = int(s["counters"][2].item())
    cap = (ms + m) // 2 if ms < m else m // 2
    assert 0 < cap < m
    # a static part built for the small buffer too, so that both parts and the output share it
    s_small = _split(D, fr, n, cams, 16, torch.as_tensor(mask).cuda(), cap)
    pr, rg, ct = _merge(D, fr, n, cams, 16, s_small, rows.size * len(cams), cap)
    torch.cuda.synchronize()
    assert int(ct[0].item()) == m and int(ct[1].item()) == 1 and int(ct[2].item()) == cap
    r = rg.cpu().numpy().astype(np.int64)
    assert (r >= 0).all() and (r <= cap).all() and (r[:, 0] <= r[:, 1]).all()
    stored = pr[:cap].cpu().numpy()
    assert (stored >= 0).all() and (stored < len(cams) * n).all()
