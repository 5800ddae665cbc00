"""Densification-stage training of the var Gaussians (Sec. 3.4, s3 iterations, every parameter of
the var rows, base rows fixed) and the low-opacity pruning that follows it, against the oracle."""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle.stages import prune_low_opacity
from paper_2411_14847_gb300 import synth

from test_gpu_render import _small_multicam, rel_l2

pytestmark = pytest.mark.gpu


def _case(seed=31, n=1500, n_var=300, deg=1):
    scene, cams = _small_multicam(seed=seed, n=n, deg=deg, n_cams=2, w=80, h=60)
    arrays = {k: np.asarray(v) for k, v in scene.arrays().items()}
    targets = [r["image"] for r in og.render(synth.perturbed(scene, 2001).arrays(), cams, deg)]
    return arrays, cams, deg, n - n_var, targets


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_densify_stage_gradients_of_var_rows(dass, lam):
    """One iteration's compact var-row gradients equal the oracle's full-parameter gradients of
    those rows (the base rows only receive what the statistics need)."""
    from paper_2411_14847_gb300 import raster
    from paper_2411_14847_gb300.timestep import DensifyStage
    arrays, cams, deg, n_base, targets = _case()
    ref = og.loss_grads(arrays, cams, deg, targets, lam)
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    st = DensifyStage(raster.to_device(arrays), n_base, cams, tgt, tile=16, batch=128, lambda_dssim=lam,
                      lr=dict(means=0.0, log_scales=0.0, quats=0.0, opacity_logit=0.0, sh_dc=0.0, sh_rest=0.0))
    st.run(1)
    torch.cuda.synchronize()
    assert st.loss == pytest.approx(ref["loss"], rel=1e-4)
    for k, gk in (("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"),
                  ("opacity_logit", "opacity_logit"), ("sh", "sh")):
        got = st.grads[gk].cpu().numpy().reshape(-1)
        want = ref[k].numpy()[n_base:].reshape(-1)
        assert rel_l2(got, want) < 1e-3, k


@pytest.mark.parametrize("deg", [1, 3])
def test_densify_stage_trains_only_var_rows(dass, deg):
    """The stage lowers the loss, moves var rows and leaves every base row bit-identical (SH degree
    3 takes the per-band learning rates through row-selected updates)."""
    from paper_2411_14847_gb300 import raster
    from paper_2411_14847_gb300.timestep import DensifyStage
    arrays, cams, deg, n_base, targets = _case(seed=32, deg=deg)
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    g = raster.to_device(arrays)
    before = {k: v.clone() for k, v in g.items()}
    st = DensifyStage(g, n_base, cams, tgt, tile=16, batch=128, lambda_dssim=0.2)
    st.run(1)
    loss0 = st.loss
    st.run(30)
    assert st.loss < loss0
    for k in g:
        assert torch.equal(g[k][:n_base], before[k][:n_base]), k
        assert not torch.equal(g[k][n_base:], before[k][n_base:]), k


def test_prune_matches_oracle(dass):
    from paper_2411_14847_gb300 import dass as D, raster
    arrays, cams, deg, n_base, targets = _case(seed=33)
    rng = np.random.default_rng(3)
    arrays["opacity_logit"] = arrays["opacity_logit"].copy()
    arrays["opacity_logit"][n_base:] = rng.uniform(-8.0, 1.0, arrays["opacity_logit"].shape[0] - n_base)
    n = arrays["means"].shape[0]
    is_var = np.zeros(n, dtype=bool)
    is_var[n_base:] = True
    ref, ref_var = prune_low_opacity(arrays, is_var, 0.005)
    g = raster.to_device(arrays)
    m = torch.empty(n, device="cuda")
    D.dass_prune_logits(g["opacity_logit"], 0.005, m)
    out = {k: torch.empty_like(v) for k, v in g.items()}
    isv_out = torch.empty(n, dtype=torch.uint8, device="cuda")
    remap = torch.empty(n, dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(max(1, D.dass_inherit_workspace(n)), dtype=torch.uint8, device="cuda")
    D.dass_inherit(g, torch.as_tensor(is_var.astype(np.uint8), device="cuda"), m, False, out, isv_out, remap, n_out, ws)
    k = int(n_out.item())
    assert k == ref["means"].shape[0]
    for name in g:
        assert np.array_equal(out[name][:k].cpu().numpy(), np.asarray(ref[name], dtype=np.float32)), name
    assert np.array_equal(isv_out[:k].cpu().numpy().astype(bool), ref_var)


def test_timestep_with_densify_stage_and_pruning(dass):
    """A full timestep with s3 > 0: var rows after the spawn are trained, pruning keeps every base
    row, and the var rows stay the contiguous tail."""
    from paper_2411_14847_gb300.timestep import Timestep
    arrays, cams, deg, n_base, targets = _case(seed=34, n_var=200)
    n = arrays["means"].shape[0]
    is_var = np.zeros(n, dtype=np.uint8)
    is_var[n_base:] = 1
    tgt = torch.cat([t.reshape(-1) for t in targets]).float().cuda()
    ts = Timestep(cams, n + 300, deg, tile=16, batch=128, n_shift=4, k_max=100, n_densify=10, tau_pos=1e-5)
    ts.load(arrays, is_var=is_var)
    dyn = torch.arange(0, 50, dtype=torch.int32, device="cuda")
    off = torch.zeros((50, 7), device="cuda")
    off[:, 3] = 1.0
    res = ts.run(1, tgt, dyn, off)
    assert res["densify_loss"] is not None
    isv = ts.is_var[:ts.n].cpu().numpy()
    nb = int((isv == 0).sum())
    assert nb == n_base
    assert np.all(isv[:nb] == 0) and np.all(isv[nb:] == 1)
    assert res["n"] == ts.n and res["pruned"] >= 0
