"""Continuous-batching render server: results alone vs in a mixed batch, continuous admission,
admission by device memory, scene swaps while requests are in flight."""
import time

import numpy as np
import pytest
import torch

from paper_2411_14847_gb300 import synth

pytestmark = pytest.mark.gpu


def _scenes():
    from paper_2411_14847_gb300 import raster
    out = {}
    for sid, (n, seed) in enumerate([(5000, 31), (12000, 32), (20000, 33)]):
        sc = synth.random_scene(n, 1, seed, box=synth.ARC_BOX, log_scale_mean=-3.3)
        out[sid] = (sc, raster.to_device(sc.arrays()))
    return out


def _requests(k, seed):
    rng = np.random.default_rng(seed)
    sizes = [(64, 48), (96, 72), (128, 96), (80, 80)]
    cams = synth.sphere_cameras(k, seed, 3.0, 5.0, sizes)
    return [(int(rng.integers(0, 3)), c) for c in cams]


def test_alone_equals_mixed_and_direct_render(dass):
    from paper_2411_14847_gb300 import raster
    from paper_2411_14847_gb300.serve import RenderServer
    scenes = _scenes()
    reqs = _requests(12, 4)
    with RenderServer(max_batch=1, n_streams=1) as alone:
        for sid, (_, g) in scenes.items():
            alone.set_scene(sid, g)
        ref = [alone.submit(s, c).result(timeout=60).clone() for s, c in reqs]
        assert max(alone.stats.batch_sizes) == 1
    with RenderServer(max_batch=8, n_streams=2) as mixed:
        for sid, (_, g) in scenes.items():
            mixed.set_scene(sid, g)
        futs = [mixed.submit(s, c) for s, c in reqs]
        got = [f.result(timeout=60) for f in futs]
        assert max(mixed.stats.batch_sizes) > 1
    for a, b in zip(ref, got):
        assert torch.allclose(a, b, atol=1e-4, rtol=0)
        assert torch.equal(a, b)        # per-pixel work does not depend on the batch
    # the serving path renders what the training-path renderer renders for the same view
    sid, cam = reqs[0]
    fr = raster.Frame([cam], scenes[sid][0].n, tile=16, batch=128)
    img = fr.render(scenes[sid][1])[0]
    assert torch.allclose(img, ref[0], atol=1e-4, rtol=0)
    assert float(ref[0].abs().sum()) > 0


def test_continuous_admission(dass):
    from paper_2411_14847_gb300.serve import RenderServer
    scenes = _scenes()
    with RenderServer(max_batch=4, n_streams=2) as srv:
        for sid, (_, g) in scenes.items():
            srv.set_scene(sid, g)
        first = [srv.submit(s, c) for s, c in _requests(8, 5)]
        while not srv.log:                       # wait until the first batch is on the GPU
            time.sleep(0.001)
        later = [srv.submit(s, c) for s, c in _requests(8, 6)]
        for f in first + later:
            assert f.result(timeout=60).shape[0] == 3
        bids_first = {b for b, rids, _, _ in srv.log if any(r < 8 for r in rids)}
        bids_later = {b for b, rids, _, _ in srv.log if any(r >= 8 for r in rids)}
        assert len(srv.log) >= 3 and bids_later - bids_first


def test_admission_by_memory_budget_and_rejection(dass):
    from paper_2411_14847_gb300.serve import RenderServer
    scenes = _scenes()
    reqs = _requests(6, 7)
    with RenderServer(max_batch=8, n_streams=1) as probe:
        for sid, (_, g) in scenes.items():
            probe.set_scene(sid, g)
        single = [probe.estimate_bytes(s, c) for s, c in reqs]
    budget = int(max(single) * 1.01)
    with RenderServer(max_batch=8, n_streams=2, hbm_budget=budget) as srv:
        for sid, (_, g) in scenes.items():
            srv.set_scene(sid, g)
        futs = [srv.submit(s, c) for s, c in reqs]
        for f in futs:
            assert f.result(timeout=60).shape[0] == 3
        assert all(est <= budget for _, _, _, est in srv.log)     # never more in flight than the budget
        huge = synth.pinhole(synth.look_at((0, 0, -4.0)), 4096, 4096)
        bad = srv.submit(2, huge)
        with pytest.raises(MemoryError):
            bad.result(timeout=60)
        assert srv.stats.rejected == 1


def test_scene_swap_keeps_inflight_version(dass):
    from paper_2411_14847_gb300 import raster
    from paper_2411_14847_gb300.serve import RenderServer
    scenes = _scenes()
    cam = synth.pinhole(synth.look_at((0.3, -0.2, -4.0)), 96, 72)
    sc0, g0 = scenes[0]
    g1 = raster.to_device(synth.perturbed(sc0, 9, mean_std=0.05, dc_std=0.5).arrays())
    with RenderServer(max_batch=4, n_streams=2) as srv:
        srv.set_scene(0, g0)
        a = srv.submit(0, cam)
        img_a = a.result(timeout=60).clone()
        srv.set_scene(0, g1)
        b = srv.submit(0, cam)
        img_b = b.result(timeout=60).clone()
        srv.set_scene(0, g0)
        c = srv.submit(0, cam)
        img_c = c.result(timeout=60).clone()
    assert torch.equal(img_a, img_c) and not torch.equal(img_a, img_b)
