"""The whole timestep behind the C ABI (dass_timestep, Sec. 3.1: G_{t-1} and the views of t give
G_t) against the same sequence composed from the individual entry points and stage drivers, its
transactional pair-overflow behaviour, and its host-buffer form."""
import numpy as np
import pytest
import torch

from oracle import grad as og
from paper_2411_14847_gb300 import synth

from test_gpu_render import _small_multicam, rel_l2

pytestmark = pytest.mark.gpu

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _case(seed=71, n=1600, n_var=240, deg=1):
    """A scene whose last n_var rows are var rows (the layout of G_{t-1} after a timestep)."""
    scene, cams = _small_multicam(seed=seed, n=n, deg=deg, n_cams=2, w=80, h=60)
    arrays = {k: np.asarray(v) for k, v in scene.arrays().items()}
    is_var = np.zeros(n, dtype=np.uint8)
    is_var[n - n_var:] = 1
    tgt_imgs = [r["image"] for r in og.render(synth.perturbed(scene, 3001).arrays(), cams, deg)]
    tgt = torch.cat([t.reshape(-1) for t in tgt_imgs]).float().cuda()
    dyn = torch.as_tensor(np.random.default_rng(seed).choice(n - n_var, 120, replace=False).astype(np.int32)).cuda()
    idx, off = synth.dynamic_split(120, 1.0, seed + 1, dmu_std=1e-3, dq_std=1e-3)
    off = torch.as_tensor(off).float().cuda()
    z = torch.as_tensor(synth.standard_normal((n + 400, 3), seed + 2)).float().cuda()
    return arrays, is_var, cams, deg, tgt, dyn, off, z


def _composed(arrays, is_var, cams, deg, tgt, dyn, off, z, t, s1, s2, s3, k_max, hp):
    """The timestep from the stage drivers and entry points, in the order dass_timestep runs them."""
    from paper_2411_14847_gb300 import dass as D, raster
    from paper_2411_14847_gb300.timestep import DensifyStage, InheritStage, ShiftStage
    g = raster.to_device(arrays)
    n = g["means"].shape[0]
    isv = torch.as_tensor(is_var).cuda()
    erase = t % 20 == 0
    m = None
    if s1 > 0 and not erase and int(isv.sum()):
        st1 = InheritStage(g, isv, cams, tgt, tile=16, batch=128, lambda_inher=hp["lambda_inher"])
        m = st1.run(s1)[:n].contiguous()
    out = {k: torch.zeros((n + k_max,) + tuple(v.shape[1:]), device="cuda") for k, v in g.items()}
    isv_b = torch.zeros(n + k_max, dtype=torch.uint8, device="cuda")
    remap = torch.empty(n, dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(max(1, D.dass_inherit_workspace(n)), dtype=torch.uint8, device="cuda")
    D.dass_inherit(g, isv, m if m is not None else torch.ones(n, device="cuda"), erase, out, isv_b, remap, n_out, ws)
    n1 = int(n_out.item())
    b = {k: v[:n1] for k, v in out.items()}
    st2 = ShiftStage(b, cams, tgt, dyn, off.clone(), tile=16, batch=128, lambda_dssim=0.2)
    st2.run(s2)
    rm, rq = b["means"].clone(), b["quats"].clone()
    D.dass_shift(dyn, st2.offsets, b["means"], b["quats"], rm, rq)
    b["means"].copy_(rm)
    b["quats"].copy_(rq)
    s_err = torch.zeros(n1, dtype=torch.uint8, device="cuda")
    ews = torch.empty(D.dass_error_pass_workspace(cams), dtype=torch.uint8, device="cuda")
    D.dass_error_pass(st2.frame.image, tgt, cams, 0.95, b["means"], isv_b[:n1], s_err, ews)
    sel = torch.empty(max(1, k_max), dtype=torch.int32, device="cuda")
    nsel = torch.zeros(1, dtype=torch.int32, device="cuda")
    sws = torch.empty(D.dass_densify_select_workspace(n1), dtype=torch.uint8, device="cuda")
    D.dass_densify_select(st2.stat_accum, st2.stat_count, s_err, isv_b[:n1], hp["tau_pos"], hp["tau_err"], k_max,
                          sel, nsel, sws)
    n_total = torch.zeros(1, dtype=torch.int64, device="cuda")
    D.dass_spawn(out, n1, isv_b, sel, nsel, k_max, z[:n1].contiguous(), n_total)
    n2 = int(n_total.item())
    c = {k: v[:n2] for k, v in out.items()}
    n_base = int((isv_b[:n2] == 0).sum())
    st3 = DensifyStage(c, n_base, cams, tgt, tile=16, batch=128, lambda_dssim=0.2)
    st3.run(s3)
    pm = torch.empty(n2, device="cuda")
    D.dass_prune_logits(c["opacity_logit"], 0.005, pm)
    fin = {k: torch.empty_like(v) for k, v in c.items()}
    isv_f = torch.empty(n2, dtype=torch.uint8, device="cuda")
    remap2 = torch.empty(n2, dtype=torch.int32, device="cuda")
    ws2 = torch.empty(max(1, D.dass_inherit_workspace(n2)), dtype=torch.uint8, device="cuda")
    D.dass_inherit(c, isv_b[:n2], pm, False, fin, isv_f, remap2, n_out, ws2)
    n3 = int(n_out.item())
    return dict(n1=n1, n2=n2, n3=n3, scene={k: v[:n3] for k, v in fin.items()}, is_var=isv_f[:n3],
                offsets=st2.offsets, loss_shift=st2.loss, loss_densify=st3.loss,
                m=m, spawned=int(nsel.item()))


@pytest.mark.parametrize("t", [3, 20])
def test_timestep_equals_composed_stages(dass, t):
    """dass_timestep (inheritance stage s1 = 3, shift s2 = 6, spawn of at most 40, densification
    stage s3 = 3, pruning) equals the composition of InheritStage, dass_inherit, ShiftStage,
    dass_shift, dass_error_pass, dass_densify_select, dass_spawn, DensifyStage, dass_prune_logits and
    dass_inherit, up to the order of floating-point atomics: row counts exactly, losses to 1e-4,
    learned offsets to 1e-2 relative L2, base rows that no stage trains bit-identical. At t = 20 every
    var row is erased first (App. B.2)."""
    from paper_2411_14847_gb300.timestep import Timestep
    arrays, is_var, cams, deg, tgt, dyn, off, z = _case()
    n = arrays["means"].shape[0]
    k_max = 40
    ts = Timestep(cams, n + 400, deg, tile=16, batch=128, n_shift=6, k_max=k_max, n_inherit=3, n_densify=3,
                  lambda_inher=1e-4, tau_pos=2e-5, tau_err=1e-5)
    ts.load(arrays, is_var=is_var)
    off_ts = off.clone()
    res = ts.run(t, tgt, dyn, off_ts, z=z)
    st = res["stats"]
    ref = _composed(arrays, is_var, cams, deg, tgt, dyn, off, z, t, 3, 6, 3, k_max,
                    dict(lambda_inher=1e-4, tau_pos=2e-5, tau_err=1e-5))
    assert st["erased"] == (1 if t == 20 else 0) and st["inherit_ran"] == (0 if t == 20 else 1)
    assert st["n_inherited"] == ref["n1"]
    if t == 20:
        assert ref["n1"] == int((is_var == 0).sum())
    assert st["n_spawned"] == ref["spawned"] and ref["spawned"] > 0
    assert ts.n == ref["n3"] == st["n_out"]
    assert st["loss_shift"] == pytest.approx(ref["loss_shift"], rel=1e-4)
    assert st["loss_densify"] == pytest.approx(ref["loss_densify"], rel=1e-4)
    assert rel_l2(off_ts.cpu().numpy(), ref["offsets"].cpu().numpy()) < 1e-2
    assert torch.equal(ts.is_var[:ts.n], ref["is_var"])
    # base rows: only the dynamic rows' means and rotations move; everything else is copied bit-exact
    nb = int((ref["is_var"] == 0).sum())
    static = np.setdiff1d(np.arange(nb), dyn.cpu().numpy())
    for k in PARAMS:
        got, want = ts.view()[k][:nb].cpu().numpy(), ref["scene"][k][:nb].cpu().numpy()
        assert np.array_equal(got[static], want[static]), k
        assert rel_l2(got, want) < 1e-3, k
    for k in PARAMS:                       # var rows: trained by the densification stage
        assert rel_l2(ts.view()[k][nb:].cpu().numpy(), ref["scene"][k][nb:].cpu().numpy()) < 1e-2, k


def test_timestep_overflow_leaves_the_scene_and_regrows(dass):
    """A pair buffer far too small makes a stage overflow: dass_timestep returns DASS_ERR_CAPACITY
    with the pair count it needed and G_{t-1} untouched; Timestep regrows from that count and the
    rerun succeeds."""
    from paper_2411_14847_gb300 import dass as D
    from paper_2411_14847_gb300.timestep import Timestep
    arrays, is_var, cams, deg, tgt, dyn, off, z = _case(seed=72)
    n = arrays["means"].shape[0]
    ts = Timestep(cams, n + 400, deg, tile=16, batch=128, n_shift=3, k_max=40)
    ts.load(arrays, is_var=is_var)
    before = {k: v[:n].clone() for k, v in ts.bufs.items()}
    ts.pair_capacity = 2048
    with pytest.raises(D.DassError) as e:
        ts.run(1, tgt, dyn, off.clone(), z=z, max_regrow=0)
    assert e.value.status == D.ERR_CAPACITY
    assert ts.n == n and ts.pair_capacity > 2048
    for k in PARAMS:
        assert torch.equal(ts.bufs[k][:n], before[k]), k
    res = ts.run(1, tgt, dyn, off.clone(), z=z)
    assert res["n"] == ts.n and res["stats"]["pairs_max"] <= ts.pair_capacity


def test_timestep_host_buffers(dass):
    """The host-buffer form: images uploaded from pinned host memory by the call itself, G_t written
    into pinned host buffers before it returns; equal to the device-buffer form."""
    from paper_2411_14847_gb300.timestep import Timestep
    arrays, is_var, cams, deg, tgt, dyn, off, z = _case(seed=73)
    n = arrays["means"].shape[0]
    res = {}
    for mode in ("device", "host"):
        ts = Timestep(cams, n + 400, deg, tile=16, batch=128, n_shift=4, k_max=40)
        ts.load(arrays, is_var=is_var)
        if mode == "device":
            r = ts.run(5, tgt, dyn, off.clone(), z=z)
            res[mode] = (r, {k: v.cpu() for k, v in ts.view().items()})
        else:
            host_tgt = tgt.cpu().pin_memory()
            dev_tgt = torch.zeros_like(tgt)
            host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in ts.bufs.items()}
            host_out["is_var"] = torch.empty(ts.is_var.shape, dtype=torch.uint8).pin_memory()
            r = ts.run(5, dev_tgt, dyn, off.clone(), z=z, targets_host=host_tgt, host_out=host_out)
            assert torch.equal(dev_tgt, tgt)
            res[mode] = (r, {k: host_out[k][:ts.n].clone() for k in PARAMS})
            assert torch.equal(host_out["is_var"][:ts.n], ts.is_var[:ts.n].cpu())
            for k in PARAMS:
                assert torch.equal(res[mode][1][k], ts.view()[k].cpu()), k
    (rd, gd), (rh, gh) = res["device"], res["host"]
    assert rd["n"] == rh["n"] and rd["spawned"] == rh["spawned"]
    assert rh["loss"] == pytest.approx(rd["loss"], rel=1e-5)
    for k in PARAMS:
        assert rel_l2(gh[k].numpy(), gd[k].numpy()) < 1e-4, k


def test_timestep_prefetches_the_next_images(dass):
    """Two timesteps where the first call also uploads the second's images (from pinned host memory
    into a second device buffer, overlapped with its stages) and the second call trains on that
    buffer: the uploaded images are exact, and G_t after both steps equals the device-buffer form.
    A descriptor with only one of the two prefetch fields is refused."""
    from paper_2411_14847_gb300 import dass as D
    from paper_2411_14847_gb300.timestep import Timestep
    arrays, is_var, cams, deg, tgt, dyn, off, z = _case(seed=74)
    tgt2 = (tgt.flip(0) * 0.5 + 0.25).contiguous()
    n = arrays["means"].shape[0]
    res = {}
    for mode in ("device", "prefetch"):
        ts = Timestep(cams, n + 400, deg, tile=16, batch=128, n_shift=4, k_max=40)
        ts.load(arrays, is_var=is_var)
        if mode == "device":
            r1 = ts.run(5, tgt, dyn, off.clone(), z=z)
            r2 = ts.run(6, tgt2, dyn, off.clone(), z=z)
        else:
            host_a, host_b = tgt.cpu().pin_memory(), tgt2.cpu().pin_memory()
            dev_a, dev_b = torch.zeros_like(tgt), torch.zeros_like(tgt)
            r1 = ts.run(5, dev_a, dyn, off.clone(), z=z, targets_host=host_a, next_targets_host=host_b,
                        next_targets=dev_b)
            assert torch.equal(dev_a, tgt) and torch.equal(dev_b, tgt2)
            r2 = ts.run(6, dev_b, dyn, off.clone(), z=z)
            p2_n = ts.n
            with pytest.raises(ValueError):
                ts.run(7, dev_b, dyn, off.clone(), z=z, next_targets=dev_a)
            # a descriptor valid but for its prefetch fields: one of the two, or the targets' own buffer
            off0, off1 = off.clone(), off.clone()
            d = ts._desc_template(int(dyn.numel()))
            ts._n_host.value = ts.n
            d.targets, d.t = dev_b.data_ptr(), 7
            d.dyn_idx, d.offsets_init, d.offsets, d.z = dyn.data_ptr(), off0.data_ptr(), off1.data_ptr(), z.data_ptr()
            d.workspace, d.workspace_bytes = ts.workspace.data_ptr(), ts.workspace.numel()
            for nh, nd in ((None, dev_a), (host_a, None), (host_a, dev_b)):
                d.next_targets_host = nh.data_ptr() if nh is not None else None
                d.next_targets = nd.data_ptr() if nd is not None else None
                with pytest.raises(D.DassError) as e:
                    D.dass_timestep(d, stream=ts.stream)
                assert e.value.status == D.ERR_INVALID_ARG
            assert ts.n == p2_n
        res[mode] = (r1, r2, {k: v.cpu() for k, v in ts.view().items()})
    (d1, d2, gd), (p1, p2, gp) = res["device"], res["prefetch"]
    assert (d1["n"], d2["n"], d1["spawned"], d2["spawned"]) == (p1["n"], p2["n"], p1["spawned"], p2["spawned"])
    assert p2["loss"] == pytest.approx(d2["loss"], rel=1e-5)
    for k in PARAMS:
        assert rel_l2(gp[k].numpy(), gd[k].numpy()) < 1e-4, k
