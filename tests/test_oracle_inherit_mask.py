"""Pins of the learned selective-inheritance mask in the oracle (Sec. 3.2 Eq. 1-2, App. B.2 STE).

* The hard mask of Eq. 1 (zero opacity and scale) renders exactly what the scene without the
  masked Gaussians renders.
* d_keep, the derivative of the fidelity loss w.r.t. the mask multiplier of Eq. 1, matches
  central finite differences of the loss under a relaxed (continuous) multiplier.
* The straight-through gradient of a rendered var Gaussian is sigmoid'(m) (d_keep + lambda);
  a masked var Gaussian contributes nothing to the render, so its gradient is the mask-loss
  term lambda sigmoid'(m) alone; base rows get none.
"""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle.loss import loss_and_image_grad
from paper_2411_14847_gb300 import synth

from test_oracle_fd import _scene, _smooth


def _setup(seed_range=range(60), n=6):
    deg = 1
    for seed in seed_range:
        arrays, cam = _scene(seed, n=n, deg=deg)
        if _smooth(arrays, cam, deg):
            return arrays, cam, deg
    pytest.fail("no smooth scene found")


def test_hard_mask_equals_subset_render():
    arrays, cam, deg = _setup()
    is_var = np.array([0, 1, 0, 1, 1, 0], dtype=bool)
    m = np.array([0.0, -0.7, 0.0, 1.3, -0.2, 0.0])
    keep = og.ste_keep(torch.as_tensor(m), is_var).detach().numpy()
    assert np.array_equal(keep, [1, 0, 1, 1, 0, 1])
    full = og.render(arrays, [cam], deg, keep=keep)[0]["image"]
    rows = np.nonzero(keep > 0)[0]
    sub = {k: np.asarray(v)[rows] for k, v in arrays.items()}
    ref = og.render(sub, [cam], deg)[0]["image"]
    assert torch.equal(full, ref)


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_keep_gradient_finite_differences(lam):
    arrays, cam, deg = _setup()
    is_var = np.array([1, 1, 0, 1, 0, 1], dtype=bool)
    m = np.array([0.4, 1.1, 0.0, 0.3, 0.0, 2.0])       # every var row rendered (m > 0)
    target = [np.random.default_rng(5).uniform(0, 1, (3, cam.height, cam.width))]
    res = og.inherit_mask_grads(arrays, [cam], deg, target, lam, m, is_var, lam_inher=0.0)

    def fid(k):
        img = og.render(arrays, [cam], deg, keep=k)[0]["image"]
        return float(loss_and_image_grad([img], [torch.as_tensor(target[0])], lam)[0])

    h = 1e-6
    for i in range(len(m)):
        kp = np.ones(len(m))
        km = np.ones(len(m))
        kp[i] += h
        km[i] -= h
        fd = (fid(kp) - fid(km)) / (2 * h)
        assert abs(float(res["d_keep"][i]) - fd) <= 1e-6 + 1e-5 * abs(fd), (i, float(res["d_keep"][i]), fd)


def test_ste_gradient_and_masked_rows():
    arrays, cam, deg = _setup()
    is_var = np.array([1, 1, 0, 1, 0, 1], dtype=bool)
    m = np.array([0.4, -0.9, 0.0, 0.3, 0.0, -2.0])
    lam_inher = 0.05
    target = [np.random.default_rng(6).uniform(0, 1, (3, cam.height, cam.width))]
    res = og.inherit_mask_grads(arrays, [cam], deg, target, 0.2, m, is_var, lam_inher)
    sg = 1.0 / (1.0 + np.exp(-m))
    dsg = sg * (1.0 - sg)
    d_keep = res["d_keep"].numpy()
    dm = res["dm"].numpy()
    for i in range(len(m)):
        if not is_var[i]:
            assert dm[i] == 0.0
        elif m[i] <= 0:
            assert d_keep[i] == 0.0                      # not rendered: no fidelity gradient
            assert dm[i] == pytest.approx(lam_inher * dsg[i], rel=1e-12)
        else:
            assert dm[i] == pytest.approx(dsg[i] * (d_keep[i] + lam_inher), rel=1e-10, abs=1e-15)
    # the loss includes the mask loss over the var rows only
    assert res["loss"] == pytest.approx(res["fidelity"] + lam_inher * sg[is_var].sum(), rel=1e-12)
