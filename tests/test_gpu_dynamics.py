"""Identity-feature rendering and the per-Gaussian dynamics query (Sec. 3.3) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import composite as comp
from oracle import dynamics as odyn
from oracle import grad as og
from paper_2411_14847_gb300 import synth

from test_gpu_render import _small_multicam

pytestmark = pytest.mark.gpu


def _render_gpu_features(scene, cams, deg, feats, tile=16):
    from paper_2411_14847_gb300 import dass as D, raster
    fr = raster.Frame(cams, scene.n, tile=tile, batch=128)
    fr.project(raster.to_device(scene.arrays()))
    fr.bin_sort()
    f = torch.as_tensor(feats, dtype=torch.float32, device="cuda").contiguous()
    out = torch.empty((fr.pixels, feats.shape[1]), device="cuda")
    D.dass_render_features(fr.splats, fr.pair_rec, fr.tile_ranges, cams, tile, f, scene.n, out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("nf,tile", [(16, 16), (8, 32), (4, 8)])
def test_feature_render_parity(dass, nf, tile):
    deg = 1
    scene, cams = _small_multicam(seed=51, n=1500, deg=deg, n_cams=2, w=64, h=48)
    feats = np.random.default_rng(0).normal(size=(scene.n, nf)).astype(np.float32)
    out = _render_gpu_features(scene, cams, deg, feats, tile=tile).cpu().numpy()
    projs = og.project_all(scene.arrays(), cams, deg)
    off = 0
    for proj, cam in zip(projs, cams):
        ref = odyn.render_features(proj, feats.astype(np.float64), cam.width, cam.height).numpy()
        got = out[off:off + cam.width * cam.height].reshape(cam.height, cam.width, nf)
        off += cam.width * cam.height
        px, py = comp.pixel_grid(cam.width, cam.height)
        flags = comp.composite_pixels(proj, px, py, want_flags=True)["flagged"].numpy().reshape(cam.height, cam.width)
        err = np.abs(got - ref).max(axis=2)
        assert np.all(err[~flags] < 1e-4), err[~flags].max()
        assert (~flags).mean() > 0.95


def test_dynamic_query_end_to_end(dass):
    """Gaussians of 8 object classes in vertical slabs; the dynamic area covers part of one slab's
    image. Per-pixel IDs, the dynamic object set and the per-Gaussian dynamics mask against the
    oracle pipeline run on its own rendered features."""
    from paper_2411_14847_gb300 import dass as D
    deg = 1
    scene, cams = _small_multicam(seed=52, n=4000, deg=deg, n_cams=2, w=96, h=72)
    means = np.asarray(scene.arrays()["means"])
    K = 8
    cls = np.clip(((means[:, 0] + 1.7) / 3.4 * K).astype(int), 0, K - 1)
    rng = np.random.default_rng(1)
    feats = (2.0 * np.eye(K)[cls] + rng.normal(0, 0.1, (scene.n, K))).astype(np.float32)
    W = np.eye(K, dtype=np.float32)
    b = np.zeros(K, dtype=np.float32)
    out = _render_gpu_features(scene, cams, deg, feats)
    Wt, bt = torch.as_tensor(W, device="cuda"), torch.as_tensor(b, device="cuda")
    ids = torch.empty(out.shape[0], dtype=torch.int32, device="cuda")
    D.dass_object_ids(out, Wt, bt, ids)
    # oracle: features rendered by the oracle, classified there
    projs = og.project_all(scene.arrays(), cams, deg)
    ref_feat = np.concatenate([odyn.render_features(p, feats.astype(np.float64), c.width, c.height).numpy()
                               .reshape(-1, K) for p, c in zip(projs, cams)])
    ref_ids = odyn.object_ids(ref_feat, W, b)
    logits = ref_feat @ W.T.astype(np.float64) + b
    top2 = np.sort(logits, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-3
    got_ids = ids.cpu().numpy()
    assert np.array_equal(got_ids[clear], ref_ids[clear])
    # dynamic area: the pixels of slab 3 in the left half of every image
    area = np.zeros(out.shape[0], dtype=np.uint8)
    off = 0
    for c in cams:
        a = (ref_ids[off:off + c.width * c.height].reshape(c.height, c.width) == 3)
        a[:, c.width // 2:] = False
        area[off:off + c.width * c.height] = a.reshape(-1)
        off += c.width * c.height
    area_t = torch.as_tensor(area, device="cuda")
    obj = torch.empty(K, dtype=torch.uint8, device="cuda")
    hist = torch.empty(K, dtype=torch.int32, device="cuda")
    D.dass_dynamic_objects(ids, area_t, K, 20, obj, hist)
    ref_obj = odyn.dynamic_objects(ref_ids, area, K, 20)
    assert np.array_equal(obj.cpu().numpy().astype(bool), ref_obj)
    assert ref_obj[3] and ref_obj.sum() >= 1
    dmask = torch.empty(scene.n, dtype=torch.uint8, device="cuda")
    D.dass_dynamic_gaussians(torch.as_tensor(feats, device="cuda"), Wt, bt, obj, dmask)
    ref_dyn = odyn.dynamic_gaussians(feats.astype(np.float64), W, b, ref_obj)
    assert np.array_equal(dmask.cpu().numpy().astype(bool), ref_dyn)
    assert np.array_equal(ref_dyn, ref_obj[cls])
    # the shift stage's dyn_idx from the mask (stable compaction)
    rows = torch.empty(scene.n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(D.dass_mask_rows_workspace(scene.n), dtype=torch.uint8, device="cuda")
    D.dass_mask_rows(dmask, rows, cnt, ws)
    k = int(cnt.item())
    assert np.array_equal(rows[:k].cpu().numpy(), np.nonzero(ref_dyn)[0])


def test_mask_rows_edge_cases(dass):
    from paper_2411_14847_gb300 import dass as D
    rng = np.random.default_rng(3)
    for n, p in ((1, 1.0), (5000, 0.0), (70000, 0.3), (12345, 1.0)):
        m = (rng.uniform(size=n) < p).astype(np.uint8)
        mt = torch.as_tensor(m, device="cuda")
        rows = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws = torch.empty(D.dass_mask_rows_workspace(n), dtype=torch.uint8, device="cuda")
        D.dass_mask_rows(mt, rows, cnt, ws)
        k = int(cnt.item())
        assert k == int(m.sum())
        assert np.array_equal(rows[:k].cpu().numpy(), np.nonzero(m)[0])
