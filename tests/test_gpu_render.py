"""GPU parity of the rasteriser (preprocess, bin/sort, forward, backward) against the FP64 oracle.

Tolerances: rendered colours max-abs <= 1e-4 on [0,1]; gradients relative L2 <= 1e-3 per
parameter tensor; sort order within each tile bit-exact, and each tile's set of Gaussians equal
to the oracle's except for footprint decisions within 1e-4 relative of their threshold. Pixels where a skip (alpha vs 1/255)
or stop (T(1-alpha) vs 1e-4) decision lies within 1e-3 relative of its threshold may take
either branch: there the GPU must match one of the oracle's alternatives.
"""
import math

import numpy as np
import pytest
import torch

from oracle import binning, composite as comp
from oracle import grad as og
from oracle import loss as oloss
from paper_2411_14847_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _small_multicam(seed=7, n=3000, deg=3, n_cams=3, w=96, h=72):
    scene = synth.random_scene(n, deg, seed, box=synth.ARC_BOX, log_scale_mean=-3.2)
    cams = synth.arc_cameras(n_cams, 4.0, w, h)
    return scene, cams


def _frame(dass, cams, n, tile=16, batch=128):
    from paper_2411_14847_gb300 import raster
    return raster.Frame(cams, n, tile=tile, batch=batch)


def _check_image(gpu_img, proj, cam, flagged_img=None, tol=1e-4):
    """Compare a [3,H,W] GPU image with the oracle; returns (#mismatch, #flagged-resolved)."""
    ref = comp.render_image(proj, cam.width, cam.height, want_flags=True)
    gi = gpu_img.detach().cpu().double()
    err = (gi - ref["image"]).abs().amax(0)
    bad = torch.nonzero(err > tol)
    unresolved = 0
    resolved = 0
    order = comp.depth_order(proj)
    for y, x in bad.tolist():
        alts = comp.pixel_alternatives(proj, float(x), float(y), order=order)
        ok = alts is not None and any(max(abs(a[0][c] - float(gi[c, y, x])) for c in range(3)) <= tol for a in alts)
        if ok and bool(ref["flagged"][y, x]):
            resolved += 1
        else:
            unresolved += 1
    return unresolved, resolved, ref, float(err.max())


def test_preprocess_parity(dass):
    scene, cams = _small_multicam()
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n)
    fr.project(g)
    torch.cuda.synchronize()
    sp = fr.splats.cpu().numpy().reshape(len(cams), scene.n, 12)
    projs = og.project_all(scene.arrays(), cams, 3)
    for c, p in enumerate(projs):
        rad = sp[c, :, 10].view(np.int32)
        vis = rad > 0
        assert vis.sum() > 100
        valid = p["valid"].numpy()
        assert np.all(valid[vis])
        np.testing.assert_allclose(sp[c, vis, 0:2], p["mean2d"].numpy()[vis], rtol=0, atol=2e-3)
        np.testing.assert_allclose(sp[c, vis, 9], p["depth"].numpy()[vis], rtol=1e-6)
        np.testing.assert_allclose(sp[c, vis, 5], p["opacity"].numpy()[vis], rtol=1e-5)
        np.testing.assert_allclose(sp[c, vis, 6:9], p["rgb"].numpy()[vis], atol=1e-5)
        assert rel_l2(sp[c, vis, 2:5], p["conic"].numpy()[vis]) < 1e-5


def _synthetic_records(n_cams, n, seed, width, height):
    """Screen-space records drawn directly (not produced by the CUDA preprocess), depth ties included."""
    rng = np.random.default_rng(seed)
    R = n_cams * n
    rec = np.zeros((R, 12), np.float32)
    rec[:, 0] = rng.uniform(-20, width + 20, R)
    rec[:, 1] = rng.uniform(-20, height + 20, R)
    sx, sy = rng.uniform(0.5, 8.0, R), rng.uniform(0.5, 8.0, R)
    th = rng.uniform(0, np.pi, R)
    c, s = np.cos(th), np.sin(th)
    cxx = c * c * sx * sx + s * s * sy * sy
    cyy = s * s * sx * sx + c * c * sy * sy
    cxy = c * s * (sx * sx - sy * sy)
    det = cxx * cyy - cxy * cxy
    rec[:, 2], rec[:, 3], rec[:, 4] = cyy / det, -cxy / det, cxx / det
    rec[:, 5] = rng.uniform(0.02, 1.0, R)
    rec[:, 9] = rng.integers(1, 40, R).astype(np.float32) * 0.25       # many exact depth ties
    rad = np.where(rng.uniform(size=R) < 0.1, 0, 30).astype(np.int32)
    rec[:, 10] = rad.view(np.float32)
    return rec, rad


def test_bin_sort_matches_oracle_binning(dass):
    cams = synth.arc_cameras(3, 4.0, 100, 70)
    n = 1500
    rec, rad = _synthetic_records(len(cams), n, 3, 100, 70)
    cam_of = np.repeat(np.arange(len(cams)), n)
    conic = rec[:, 2:5].astype(np.float64)
    for tile in (8, 16, 32):
        from paper_2411_14847_gb300 import raster
        fr = raster.Frame(cams, n, tile=tile, batch=128)
        fr.splats.copy_(torch.from_numpy(rec))
        m = fr.bin_sort()
        torch.cuda.synchronize()
        sure, maybe, total = binning.bin_records(rec[:, 0], rec[:, 1], conic, rec[:, 5], rad, cam_of, cams, tile)
        pr = fr.pair_rec[:m].cpu().numpy().astype(np.int64)
        rg = fr.tile_ranges.cpu().numpy().astype(np.int64)
        assert rg.shape[0] == total and int(sum(rg[:, 1] - rg[:, 0])) == m
        for t in range(total):
            lst = pr[rg[t, 0]:rg[t, 1]].tolist()
            keys = [binning.order_key(rec[r, 9], r) for r in lst]
            assert keys == sorted(keys) and len(set(lst)) == len(lst), t
            got = set(lst)
            s_t, m_t = sure.get(t, set()), maybe.get(t, set())
            assert s_t <= got <= (s_t | m_t), (tile, t, s_t - got, got - s_t - m_t)


def test_bin_sort_long_tile_lists(dass):
    """Tiles with long lists (about 6,000 and 20,000 pairs, far more than one compositing batch or one
    sort block): order and tile sets as in the oracle's binning."""
    from paper_2411_14847_gb300 import raster
    cams = synth.arc_cameras(2, 4.0, 64, 48)
    n = 24000
    rng = np.random.default_rng(11)
    rec = np.zeros((2 * n, 12), np.float32)
    rec[:, 0] = rng.uniform(20.0, 27.0, 2 * n)
    rec[:, 1] = rng.uniform(18.0, 25.0, 2 * n)
    sig = rng.uniform(0.5, 1.5, 2 * n)
    rec[:, 2], rec[:, 4] = 1.0 / sig ** 2, 1.0 / sig ** 2
    rec[:, 5] = rng.uniform(0.05, 1.0, 2 * n)
    rec[:, 9] = rng.integers(1, 200, 2 * n).astype(np.float32) * 0.125      # depth ties
    rad = np.full(2 * n, 6, np.int32)
    rad[n + 7000:] = 0                                                        # camera 1: 7,000 visible
    rec[:, 10] = rad.view(np.float32)
    fr = raster.Frame(cams, n, tile=8, batch=64)
    fr.splats.copy_(torch.from_numpy(rec))
    m = fr.bin_sort()
    torch.cuda.synchronize()
    cam_of = np.repeat(np.arange(2), n)
    sure, maybe, total = binning.bin_records(rec[:, 0], rec[:, 1], rec[:, 2:5].astype(np.float64), rec[:, 5], rad,
                                             cam_of, cams, 8)
    pr = fr.pair_rec[:m].cpu().numpy().astype(np.int64)
    rg = fr.tile_ranges.cpu().numpy().astype(np.int64)
    lens = rg[:, 1] - rg[:, 0]
    assert lens[:48].max() > 16384 and 4096 < lens[48:].max() <= 16384, (lens[:48].max(), lens[48:].max())
    for t in range(total):
        lst = pr[rg[t, 0]:rg[t, 1]].tolist()
        keys = [binning.order_key(rec[r, 9], r) for r in lst]
        assert keys == sorted(keys) and len(set(lst)) == len(lst), t
        got = set(lst)
        s_t, m_t = sure.get(t, set()), maybe.get(t, set())
        assert s_t <= got <= (s_t | m_t), (t, len(s_t - got), len(got - s_t - m_t))


def test_bin_sort_overflow_flag_and_regrow(dass):
    scene, cams = _small_multicam(n=2000)
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    fr = raster.Frame(cams, scene.n, pair_capacity=64)
    fr.project(g)
    from paper_2411_14847_gb300 import dass as D
    D.dass_bin_sort(fr.splats, fr.n, fr.cams, fr.tile, fr.pair_rec, fr.tile_ranges, fr.counters, fr.workspace)
    m, over = fr.counters[:2].tolist()
    assert over == 1 and m > 64
    m2 = fr.bin_sort()
    assert m2 == m and int(fr.counters[1]) == 0


def test_forward_parity_config_a(dass):
    scene, cams = synth.config_a()
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n)
    img = fr.render(g)[0]
    torch.cuda.synchronize()
    proj = og.project_all(scene.arrays(), cams, 0)[0]
    bad, resolved, ref, maxerr = _check_image(img, proj, cams[0])
    assert bad == 0, (bad, resolved, maxerr)
    # T_final and last contributor on pixels away from threshold ties
    tf = fr.T_final.cpu().double().view(128, 128)
    fl = ref["flagged"]
    assert float((tf - ref["T_final"]).abs()[~fl].max()) < 1e-5
    nl = fr.n_last.cpu().numpy().reshape(128, 128)
    pr = fr.pair_rec.cpu().numpy()
    gpu_last = np.where(nl >= 0, pr[np.clip(nl, 0, None)] % scene.n, -1)
    ok = ~fl.numpy()
    np.testing.assert_array_equal(gpu_last[ok], ref["n_last"].numpy()[ok])


@pytest.mark.parametrize("tile,batch", [(16, 128), (8, 64), (32, 256)])
def test_forward_parity_multicam_sh3(dass, tile, batch):
    scene, cams = _small_multicam()
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n, tile=tile, batch=batch)
    imgs = fr.render(g)
    torch.cuda.synchronize()
    projs = og.project_all(scene.arrays(), cams, 3)
    for img, p, cam in zip(imgs, projs, cams):
        bad, resolved, _, maxerr = _check_image(img, p, cam)
        assert bad == 0, (bad, resolved, maxerr)


def test_forward_parity_max_cameras(dass):
    """The largest camera table one call accepts (64 views, packed into the kernel parameters):
    every view against the oracle, and a 65th view is refused on the host."""
    from paper_2411_14847_gb300 import dass as D, raster
    scene, cams = _small_multicam(seed=13, n=400, deg=1, n_cams=64, w=24, h=18)
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n, tile=16, batch=64)
    imgs = fr.render(g)
    torch.cuda.synchronize()
    projs = og.project_all(scene.arrays(), cams, 1)
    for img, p, cam in zip(imgs, projs, cams):
        bad, resolved, _, maxerr = _check_image(img, p, cam)
        assert bad == 0, (bad, resolved, maxerr)
    with pytest.raises(D.DassError):
        D.tile_layout(list(cams) + [cams[0]], 16)


def test_images_bit_identical_across_tiles_and_batches(dass):
    scene, cams = _small_multicam(seed=11)
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    ref = None
    for tile in (8, 16, 32):
        for batch in (32, 64, 128, 256):
            fr = _frame(dass, cams, scene.n, tile=tile, batch=batch)
            fr.render(g)
            out = torch.cat([fr.image, fr.T_final])
            if ref is None:
                ref = out.clone()
            else:
                assert torch.equal(out, ref), (tile, batch)


def test_empty_scene_and_all_culled(dass):
    cams = synth.arc_cameras(2, 4.0, 40, 30)
    from paper_2411_14847_gb300 import raster
    scene = synth.random_scene(50, 0, 5)
    scene.means[:, 2] = -10.0          # every Gaussian behind the cameras
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n)
    imgs = fr.render(g, bg=(0.25, 0.5, 0.75))
    torch.cuda.synchronize()
    assert int(fr.counters[0]) == 0
    for im in imgs:
        assert torch.allclose(im[0], torch.full_like(im[0], 0.25)) and torch.allclose(im[2], torch.full_like(im[2], 0.75))
    assert bool((fr.T_final == 1).all()) and bool((fr.n_last == -1).all())


def _grad_case(dass, scene, cams, deg, lam, tile=16, batch=128):
    from paper_2411_14847_gb300 import dass as D, raster
    target_scene = synth.perturbed(scene, 2001)
    targets = og.render(target_scene.arrays(), cams, deg)
    targets = [t["image"] for t in targets]
    params = {k: v.clone().requires_grad_(True) for k, v in raster.to_device(scene.arrays()).items()}
    fr = _frame(dass, cams, scene.n, tile=tile, batch=batch)
    img = raster.render_autograd(params, fr)
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, D.dass_loss_workspace(cams)), dtype=torch.uint8, device="cuda")
    D.dass_loss(img.detach(), tgt, cams, lam, dimg, loss, ws)
    img.backward(dimg)
    torch.cuda.synchronize()
    ref = og.loss_grads(scene.arrays(), cams, deg, targets, lam)
    return params, ref, float(loss)


def test_gradient_parity_config_a(dass):
    scene, cams = synth.config_a()
    params, ref, loss = _grad_case(dass, scene, cams, 0, 0.0)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    for k in og.PARAMS:
        assert rel_l2(params[k].grad.cpu().numpy(), ref[k].numpy()) < 1e-3, k


def test_gradient_parity_multicam_sh3_dssim(dass):
    scene, cams = _small_multicam(n=1500, w=64, h=48)
    params, ref, loss = _grad_case(dass, scene, cams, 3, 0.2)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    for k in og.PARAMS:
        assert rel_l2(params[k].grad.cpu().numpy(), ref[k].numpy()) < 1e-3, k


def _opaque_mix_scene(seed, n, deg=3):
    """A scene where one Gaussian in six has opacity above 0.99 (logit 5 to 7), so the 0.99 alpha clamp
    acts at many pixels and the compositing rounds mix entries that may clamp with entries that cannot."""
    scene, cams = _small_multicam(seed=seed, n=n, deg=deg, w=64, h=48)
    rng = np.random.default_rng(seed + 100)
    hot = rng.random(scene.n) < 1.0 / 6.0
    scene.opacity_logit = np.where(hot, rng.uniform(5.0, 7.0, scene.n), scene.opacity_logit).astype(np.float32)
    return scene, cams


@pytest.mark.parametrize("tile,batch", [(32, 32), (16, 64), (8, 256)])
def test_alpha_clamp_rounds_parity(dass, tile, batch):
    """Rounds with and without a possible clamp (App. A.1: alpha = min(0.99, o G)) against the oracle:
    images, and the gradients of every parameter (the clamp has zero derivative)."""
    scene, cams = _opaque_mix_scene(17, 1500)
    params, ref, loss = _grad_case(dass, scene, cams, 3, 0.2, tile=tile, batch=batch)
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    for k in og.PARAMS:
        assert rel_l2(params[k].grad.cpu().numpy(), ref[k].numpy()) < 1e-3, k
    from paper_2411_14847_gb300 import raster
    fr = _frame(dass, cams, scene.n, tile=tile, batch=batch)
    imgs = fr.render(raster.to_device(scene.arrays()))
    torch.cuda.synchronize()
    projs = og.project_all(scene.arrays(), cams, 3)
    n_clamped = 0
    for img, p, cam in zip(imgs, projs, cams):
        bad, resolved, _, maxerr = _check_image(img, p, cam)
        assert bad == 0, (bad, resolved, maxerr)
        n_clamped += int((p["opacity"] >= 0.99).sum())
    assert n_clamped > 100


def test_alpha_clamp_images_bit_identical_across_tiles_and_batches(dass):
    """The clamp-free and general round forms give the same bits, whatever mix of entries a round holds."""
    scene, cams = _opaque_mix_scene(19, 2500)
    from paper_2411_14847_gb300 import raster
    g = raster.to_device(scene.arrays())
    ref = None
    for tile in (8, 16, 32):
        for batch in (32, 64, 128, 256):
            fr = _frame(dass, cams, scene.n, tile=tile, batch=batch)
            fr.render(g)
            out = torch.cat([fr.image, fr.T_final])
            if ref is None:
                ref = out.clone()
            else:
                assert torch.equal(out, ref), (tile, batch)


def test_tile_order_longest_first_and_results_unchanged(dass):
    """dass_tile_order: a permutation of the tiles by descending list length (to within its 8
    buckets per power of two, empty lists last); compositing in that order gives the same images,
    T_final and n_last bit for bit, and the same gradients up to the order of the atomic sums."""
    from paper_2411_14847_gb300 import dass as D, raster
    scene, cams = _small_multicam(seed=23, n=4000)
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n, tile=16, batch=64)
    fr.render(g)
    dimg = torch.randn_like(fr.image) * 1e-3
    fr.render_bwd(dimg)
    torch.cuda.synchronize()
    ref = [fr.image.clone(), fr.T_final.clone(), fr.n_last.clone(), fr.splat_grads.clone()]
    # the order property on synthetic ranges (empty, short and 2^20-long lists, 50k tiles)
    rng = np.random.default_rng(5)
    ln = np.where(rng.random(50_000) < 0.1, 0, np.exp(rng.uniform(0, 12, 50_000)).astype(np.int64))
    ln[:3] = (0, 1, 1 << 20)
    start = np.concatenate([[0], np.cumsum(ln)[:-1]])
    syn = torch.as_tensor(np.stack([start, start + ln], 1).astype(np.int32), device="cuda")
    o_syn = torch.full((ln.size,), -1, dtype=torch.int32, device="cuda")
    D.dass_tile_order(syn, o_syn)
    for rgs, o in ((syn, o_syn), (fr.tile_ranges, None)):
        if o is None:
            o = torch.full((fr.tiles_total,), -1, dtype=torch.int32, device="cuda")
            D.dass_tile_order(fr.tile_ranges, o)
            order = o
        torch.cuda.synchronize()
        oh = o.cpu().numpy()
        np.testing.assert_array_equal(np.sort(oh), np.arange(oh.size))
        r = rgs.cpu().numpy().astype(np.int64)
        lo = (r[:, 1] - r[:, 0])[oh]
        later_max = np.maximum.accumulate(lo[::-1])[::-1]      # longest list at or after each position
        pos = lo > 0
        assert np.all(later_max[pos] <= lo[pos] * 1.125)
        assert np.all(later_max[~pos] == 0)                     # empty lists last
    D.dass_render_fwd(fr.splats, fr.pair_rec, fr.tile_ranges, cams, 16, 64, fr.image, fr.T_final, fr.n_last,
                      order=order)
    D.dass_render_bwd(fr.splats, fr.pair_rec, fr.tile_ranges, cams, 16, 64, fr.T_final, fr.n_last, dimg,
                      fr.splat_grads, order=order)
    torch.cuda.synchronize()
    assert torch.equal(fr.image, ref[0]) and torch.equal(fr.T_final, ref[1]) and torch.equal(fr.n_last, ref[2])
    assert rel_l2(fr.splat_grads.cpu().numpy(), ref[3].cpu().numpy()) < 1e-5


def test_loss_parity(dass):
    from paper_2411_14847_gb300 import dass as D
    cams = synth.arc_cameras(2, 4.0, 53, 37)
    rng = np.random.default_rng(0)
    imgs = [rng.uniform(0, 1, (3, 37, 53)) for _ in cams]
    tgts = [rng.uniform(0, 1, (3, 37, 53)) for _ in cams]
    x = torch.tensor(np.concatenate([i.reshape(-1) for i in imgs]), dtype=torch.float32, device="cuda")
    y = torch.tensor(np.concatenate([i.reshape(-1) for i in tgts]), dtype=torch.float32, device="cuda")
    for lam in (0.0, 0.2, 1.0):
        ref_loss, ref_g = oloss.loss_and_image_grad([torch.tensor(i).float().double() for i in imgs],
                                                    [torch.tensor(t).float().double() for t in tgts], lam)
        dx = torch.empty_like(x)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = torch.empty(D.dass_loss_workspace(cams), dtype=torch.uint8, device="cuda")
        D.dass_loss(x, y, cams, lam, dx, loss, ws)
        torch.cuda.synchronize()
        assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
        assert rel_l2(dx.cpu().numpy(), np.concatenate([g.reshape(-1).numpy() for g in ref_g])) < 1e-4


@pytest.mark.parametrize("w,h", [(53, 37), (130, 75)])
def test_loss_cached_target_stats_parity(dass, w, h):
    """Target window statistics against the oracle's filter, and the loss that reads them against
    the oracle and against the uncached loss (same planes, ragged 32 x 32 output tiles)."""
    from paper_2411_14847_gb300 import dass as D
    cams = synth.arc_cameras(3, 4.0, w, h)
    rng = np.random.default_rng(1)
    imgs = [rng.uniform(0, 1, (3, h, w)) for _ in cams]
    tgts = [rng.uniform(0, 1, (3, h, w)) for _ in cams]
    x = torch.tensor(np.concatenate([i.reshape(-1) for i in imgs]), dtype=torch.float32, device="cuda")
    y = torch.tensor(np.concatenate([i.reshape(-1) for i in tgts]), dtype=torch.float32, device="cuda")
    stats = torch.empty(2 * y.numel(), device="cuda")
    D.dass_loss_target_stats(y, cams, stats)
    torch.cuda.synchronize()
    mom = [oloss.window_moments(torch.tensor(t).float().double()) for t in tgts]
    want_m = np.concatenate([m[0].reshape(-1).numpy() for m in mom])
    want_q = np.concatenate([m[1].reshape(-1).numpy() for m in mom])
    got = stats.cpu().numpy().reshape(-1, 2)
    assert np.abs(got[:, 0] - want_m).max() < 2e-6
    assert np.abs(got[:, 1] - want_q).max() < 2e-6
    ws = torch.empty(D.dass_loss_workspace(cams), dtype=torch.uint8, device="cuda")
    for lam in (0.2, 1.0):
        ref_loss, ref_g = oloss.loss_and_image_grad([torch.tensor(i).float().double() for i in imgs],
                                                    [torch.tensor(t).float().double() for t in tgts], lam)
        dx, dx0 = torch.empty_like(x), torch.empty_like(x)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        loss0 = torch.zeros(1, dtype=torch.float64, device="cuda")
        D.dass_loss_cached(x, y, stats, cams, lam, dx, loss, ws)
        D.dass_loss(x, y, cams, lam, dx0, loss0, ws)
        torch.cuda.synchronize()
        want_g = np.concatenate([g.reshape(-1).numpy() for g in ref_g])
        assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
        assert rel_l2(dx.cpu().numpy(), want_g) < 1e-4
        assert float(loss) == pytest.approx(float(loss0), rel=1e-6)
        assert rel_l2(dx.cpu().numpy(), dx0.cpu().numpy()) < 1e-5


def test_backward_mean_only_for_unmasked_gaussians(dass):
    """With a per-Gaussian mask, unmasked Gaussians receive only dL/dmean2D (same values as the
    full backward); masked ones receive the full splat gradient."""
    from paper_2411_14847_gb300 import dass as D, raster
    scene, cams = _small_multicam(n=2500)
    g = raster.to_device(scene.arrays())
    fr = _frame(dass, cams, scene.n, tile=16, batch=128)
    fr.render(g)
    dimg = torch.randn_like(fr.image) * 1e-3
    fr.render_bwd(dimg)
    full = fr.splat_grads.clone()
    mask = (torch.rand(scene.n, device="cuda") < 0.2).to(torch.uint8)
    D.dass_render_bwd(fr.splats, fr.pair_rec, fr.tile_ranges, cams, 16, 128, fr.T_final, fr.n_last, dimg,
                      fr.splat_grads, full_grad=mask, rec_stride=scene.n)
    torch.cuda.synchronize()
    part = fr.splat_grads.view(len(cams), scene.n, 12)
    ref = full.view(len(cams), scene.n, 12)
    m = mask.bool()
    assert rel_l2(part[:, m].cpu().numpy(), ref[:, m].cpu().numpy()) < 1e-5
    assert rel_l2(part[:, ~m, 0:2].cpu().numpy(), ref[:, ~m, 0:2].cpu().numpy()) < 1e-5
    assert float(part[:, ~m, 2:].abs().max()) == 0.0
    assert float(ref[:, ~m, 2:9].abs().max()) > 0.0


def test_autograd_gradients_with_shift_offsets(dass):
    """The autograd Function through the dynamics-aware shift (Sec. 3.3): gradients of all six
    inputs -- means, log-scales, quaternions, opacity logits, SH and the dynamic rows' offsets --
    against the oracle's analytic (autodiff) gradients, which are pinned by finite differences."""
    from paper_2411_14847_gb300 import dass as D, raster
    scene, cams = _small_multicam(n=1500, w=64, h=48, deg=1)
    deg = 1
    rng = np.random.default_rng(12)
    dyn = np.sort(rng.choice(scene.n, 150, replace=False)).astype(np.int32)
    off = np.zeros((150, 7))
    off[:, :3] = rng.normal(0, 0.02, (150, 3))
    off[:, 3:] = np.array([1.0, 0, 0, 0]) + rng.normal(0, 0.05, (150, 4))
    targets = [t["image"] for t in og.render(synth.perturbed(scene, 2001).arrays(), cams, deg)]
    ref = og.loss_grads(scene.arrays(), cams, deg, targets, 0.2, dyn_idx=dyn, offsets=off)
    params = {k: v.clone().requires_grad_(True) for k, v in raster.to_device(scene.arrays()).items()}
    off_t = torch.tensor(off, dtype=torch.float32, device="cuda", requires_grad=True)
    dyn_t = torch.as_tensor(dyn, device="cuda")
    fr = _frame(dass, cams, scene.n)
    img = raster.render_autograd(params, fr, dyn_idx=dyn_t, offsets=off_t)
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, D.dass_loss_workspace(cams)), dtype=torch.uint8, device="cuda")
    D.dass_loss(img.detach(), tgt, cams, 0.2, dimg, loss, ws)
    img.backward(dimg)
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(ref["loss"], rel=1e-4)
    for k in og.PARAMS:
        assert rel_l2(params[k].grad.cpu().numpy(), ref[k].numpy()) < 1e-3, k
    assert rel_l2(off_t.grad.cpu().numpy(), ref["offsets"].numpy()) < 1e-3
