"""Hash-encoding deformation field kernels (dass_field_fwd / dass_field_bwd) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import field as fld

from test_gpu_render import rel_l2

pytestmark = pytest.mark.gpu

CASES = [(4, 16, 16), (2, 16, 14), (2, 8, 10), (4, 8, 12)]   # (features, levels, log2 T)


def _setup(feats, levels, log2t, n=3000, seed=0):
    rng = np.random.default_rng(seed)
    T = 1 << log2t
    prm = {"table": rng.uniform(-0.05, 0.05, (levels, T, feats)),
           "w1": rng.normal(0, 0.2, (64, levels * feats)), "b1": rng.normal(0, 0.1, 64),
           "w2": rng.normal(0, 0.1, (7, 64)), "b2": rng.normal(0, 0.01, 7)}
    lo, hi = np.array([-1.7, -1.3, -1.0]), np.array([1.7, 1.3, 1.0])
    means = rng.uniform(lo - 0.1, hi + 0.1, (n, 3))          # some outside the box (clamped)
    res = fld.level_resolutions(levels)
    return prm, lo, hi, means, res, rng


def _field(prm, res, log2t, lo, hi):
    from paper_2411_14847_gb300 import dass as D
    dp = {k: torch.as_tensor(v, dtype=torch.float32, device="cuda").contiguous() for k, v in prm.items()}
    return D.field_struct(dp, res, log2t, lo, hi), dp


@pytest.mark.parametrize("feats,levels,log2t", CASES)
def test_field_forward_parity(dass, feats, levels, log2t):
    from paper_2411_14847_gb300 import dass as D
    prm, lo, hi, means, res, rng = _setup(feats, levels, log2t)
    f, dp = _field(prm, res, log2t, lo, hi)
    m = torch.as_tensor(means, dtype=torch.float32, device="cuda")
    rows = torch.as_tensor(np.sort(rng.choice(means.shape[0], 1000, replace=False)), dtype=torch.int32,
                           device="cuda")
    out = torch.empty((1000, 7), device="cuda")
    D.dass_field_fwd(f, m, out, rows=rows)
    torch.cuda.synchronize()
    ref = fld.field_offsets(means.astype(np.float32)[rows.cpu().numpy()],
                            {k: torch.as_tensor(v.astype(np.float32)).double() for k, v in prm.items()},
                            res, lo, hi, fp32_positions=True).numpy()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=2e-6)


@pytest.mark.parametrize("feats,levels,log2t", CASES)
def test_field_backward_parity(dass, feats, levels, log2t):
    from paper_2411_14847_gb300 import dass as D
    prm, lo, hi, means, res, rng = _setup(feats, levels, log2t, n=2000, seed=1)
    f, dp = _field(prm, res, log2t, lo, hi)
    d_off = rng.normal(size=(means.shape[0], 7))
    m = torch.as_tensor(means, dtype=torch.float32, device="cuda")
    grads = {k: torch.zeros_like(v) for k, v in dp.items()}
    D.dass_field_bwd(f, m, torch.as_tensor(d_off, dtype=torch.float32, device="cuda"), grads)
    torch.cuda.synchronize()
    ref, _ = fld.field_grads(means.astype(np.float32).astype(np.float64),
                             {k: v.astype(np.float32).astype(np.float64) for k, v in prm.items()}, res, lo, hi,
                             d_off.astype(np.float32).astype(np.float64), fp32_positions=True)
    for k in ("table", "w1", "b1", "w2", "b2"):
        assert rel_l2(grads[k].cpu().numpy(), ref[k].numpy()) < 1e-4, k


def test_field_shift_stage_gradient_chain(dass):
    """One iteration of the field-driven shift stage: the gradients of both fields' parameters
    equal the oracle chain loss(render(shift(field offsets))) -> d offsets (oracle autodiff
    through the renderer and the shift) -> field parameters (oracle autodiff through the field)."""
    from oracle import grad as og
    from paper_2411_14847_gb300 import raster, synth
    from paper_2411_14847_gb300.timestep import FieldShiftStage
    from test_gpu_render import _small_multicam
    deg = 1
    scene, cams = _small_multicam(seed=41, n=1000, deg=deg, n_cams=2, w=64, h=48)
    rng = np.random.default_rng(5)
    dyn = np.sort(rng.choice(scene.n, 100, replace=False)).astype(np.int32)
    targets = [t["image"] for t in og.render(synth.perturbed(scene, 2001).arrays(), cams, deg)]
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    lo, hi = np.array([-2.0, -2.0, -2.0]), np.array([2.0, 2.0, 2.0])
    st = FieldShiftStage(raster.to_device(scene.arrays()), cams, tgt, torch.as_tensor(dyn, device="cuda"),
                         tile=16, batch=128, lambda_dssim=0.2, levels=8, bbox=(lo, hi), lr=0.0)
    # non-trivial fields: random output layers (the identity initialisation has zero w2 gradients
    # flowing back only through w2)
    for gi, grp in enumerate(st.groups):
        grp["params"]["w2"].normal_(0.0, 0.05, generator=torch.Generator(device="cuda").manual_seed(gi))
        grp["params"]["table"].uniform_(-0.05, 0.05, generator=torch.Generator(device="cuda").manual_seed(9 + gi))
    prm_host = [{k: v.detach().cpu().double() for k, v in grp["params"].items()} for grp in st.groups]
    st.run(1)
    torch.cuda.synchronize()
    means = np.asarray(scene.arrays()["means"], dtype=np.float32).astype(np.float64)
    offsets = np.zeros((scene.n, 7))
    for grp, prm in zip(st.groups, prm_host):
        rows = grp["rows"].cpu().numpy()
        offsets[rows] = fld.field_offsets(means[rows], prm, grp["res"], lo, hi, fp32_positions=True).numpy()
    ref = og.loss_grads(scene.arrays(), cams, deg, targets, 0.2, dyn_idx=np.arange(scene.n), offsets=offsets)
    assert st.loss == pytest.approx(ref["loss"], rel=1e-4)
    d_off = ref["offsets"].numpy()
    for grp, prm in zip(st.groups, prm_host):
        rows = grp["rows"].cpu().numpy()
        want, _ = fld.field_grads(means[rows], {k: v.numpy() for k, v in prm.items()}, grp["res"], lo, hi,
                                  d_off[rows], fp32_positions=True)
        for k in ("table", "w1", "b1", "w2", "b2"):
            assert rel_l2(grp["grads"][k].cpu().numpy(), want[k].numpy()) < 1e-3, (grp["n"], k)


def test_field_shift_stage_learns_a_translation(dass):
    """Targets rendered from the scene translated by +0.03 in x: the two fields learn offsets that
    move the Gaussians that way and the loss drops."""
    from oracle import grad as og
    from paper_2411_14847_gb300 import raster
    from paper_2411_14847_gb300.timestep import FieldShiftStage
    from test_gpu_render import _small_multicam
    deg = 1
    scene, cams = _small_multicam(seed=42, n=3000, deg=deg, n_cams=3, w=96, h=72)
    arrays = scene.arrays()
    moved = dict(arrays, means=np.asarray(arrays["means"]) + np.array([0.03, 0.0, 0.0]))
    targets = og.render(moved, cams, deg)
    tgt = torch.cat([t["image"].reshape(-1) for t in targets]).float().cuda()
    rng = np.random.default_rng(6)
    dyn = torch.as_tensor(np.sort(rng.choice(scene.n, 300, replace=False)).astype(np.int32), device="cuda")
    st = FieldShiftStage(raster.to_device(arrays), cams, tgt, dyn, tile=16, batch=128, lambda_dssim=0.2,
                         levels=16, lr=3e-3)
    st.run(1)
    loss0 = st.loss
    st.run(60)
    assert st.loss < 0.8 * loss0
    for grp in st.groups:
        dx = grp["offsets"][:grp["n"], 0].mean().item()
        assert dx > 0.005, (grp["n"], dx)
