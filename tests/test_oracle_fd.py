"""Central finite differences pin the oracle's reverse-mode gradients (FP64).

Inputs are redrawn until every Gaussian-pixel pair sits away from the discontinuities of
the definition (alpha = 1/255, alpha = 0.99, T(1 - alpha) = 1e-4), so that the loss is
smooth in a neighbourhood of the evaluation point.
"""
import numpy as np
import pytest
import torch

from oracle import composite as comp
from oracle import grad as og
from paper_2411_14847_gb300 import synth


def _scene(seed, n=6, size=12, deg=1):
    rng = np.random.default_rng(seed)
    vm = synth.look_at((0.6, -0.3, -4.0))
    cam = synth.pinhole(vm, size, size, 50.0)
    arrays = dict(means=rng.uniform(-0.5, 0.5, (n, 3)), log_scales=rng.normal(-1.6, 0.25, (n, 3)),
                  quats=rng.normal(size=(n, 4)), opacity_logit=rng.normal(0.0, 0.8, n),
                  sh=rng.normal(0, 0.5, (n, (deg + 1) ** 2, 3)))
    return arrays, cam


def _smooth(arrays, cam, deg, dyn=None, off=None, margin=2e-2):
    proj = og.project_all(arrays, [cam], deg, dyn, off)[0]
    order = comp.depth_order(proj)
    px, py = comp.pixel_grid(cam.width, cam.height)
    a = comp.alpha_matrix(proj["mean2d"][order], proj["conic"][order], proj["opacity"][order], px, py)
    if bool(((a * 255 - 1).abs() < margin).any()) or bool(((a - 0.99).abs() < 1e-3).any()):
        return False
    keep = a >= 1 / 255
    t = torch.cumprod(torch.where(keep, 1 - a, torch.ones_like(a)), 1)
    return not bool(((t * 1e4 - 1).abs() < margin).any())


def _fd(fun, x, idx, h):
    xp = x.copy()
    xm = x.copy()
    xp.flat[idx] += h
    xm.flat[idx] -= h
    return (fun(xp) - fun(xm)) / (2 * h)


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_fd_all_parameters(lam):
    deg = 1
    for seed in range(50):
        arrays, cam = _scene(seed, deg=deg)
        if _smooth(arrays, cam, deg):
            break
    else:
        pytest.fail("no smooth scene found")
    target = [np.random.default_rng(99).uniform(0, 1, (3, cam.height, cam.width))]
    res = og.loss_grads(arrays, [cam], deg, target, lam)

    for name in og.PARAMS:
        base = np.asarray(arrays[name], dtype=np.float64)

        def f(x, name=name):
            a2 = dict(arrays)
            a2[name] = x
            from oracle.loss import fidelity_loss
            img = og.render(a2, [cam], deg)[0]["image"]
            return float(fidelity_loss([img], [torch.tensor(target[0])], lam))

        g = res[name].numpy().reshape(-1)
        for idx in range(0, base.size, max(1, base.size // 12)):
            h = 1e-6 * max(1.0, abs(base.flat[idx]))
            fd = _fd(f, base, idx, h)
            assert abs(fd - g[idx]) <= 1e-6 * max(1e-3, abs(g[idx])) + 1e-9, (name, idx, fd, g[idx])


def test_fd_shift_offsets():
    deg = 1
    dyn = np.array([0, 2, 3])
    rng = np.random.default_rng(5)
    off = np.zeros((3, 7))
    off[:, :3] = rng.normal(0, 0.02, (3, 3))
    off[:, 3:] = np.array([1.0, 0, 0, 0]) + rng.normal(0, 0.1, (3, 4))
    for seed in range(50):
        arrays, cam = _scene(100 + seed, deg=deg)
        if _smooth(arrays, cam, deg, dyn, off):
            break
    target = [np.random.default_rng(98).uniform(0, 1, (3, cam.height, cam.width))]
    res = og.loss_grads(arrays, [cam], deg, target, 0.2, dyn_idx=dyn, offsets=off)

    def f(x):
        from oracle.loss import fidelity_loss
        img = og.render(arrays, [cam], deg, dyn, x)[0]["image"]
        return float(fidelity_loss([img], [torch.tensor(target[0])], 0.2))

    g = res["offsets"].numpy().reshape(-1)
    for idx in range(off.size):
        fd = _fd(f, off, idx, 1e-6)
        assert abs(fd - g[idx]) <= 1e-6 * max(1e-3, abs(g[idx])) + 1e-9, (idx, fd, g[idx])
    # rotation offsets only enter through norm(sigma): the gradient is orthogonal to sigma
    sg = off[:, 3:]
    np.testing.assert_allclose((res["offsets"].numpy()[:, 3:] * sg).sum(1), 0.0, atol=1e-10)


def test_fd_dmean2d_matches_pixel_gradient():
    # dL/d mean2D reported per camera equals d/du of the loss with everything else fixed.
    deg = 0
    for seed in range(50):
        arrays, cam = _scene(200 + seed, deg=deg)
        if _smooth(arrays, cam, deg):
            break
    target = [np.zeros((3, cam.height, cam.width))]
    res = og.loss_grads(arrays, [cam], deg, target, 0.0)
    proj = og.project_all(arrays, [cam], deg)[0]
    from oracle.loss import fidelity_loss
    px, py = comp.pixel_grid(cam.width, cam.height)
    for i in range(3):
        for k in range(2):
            vals = []
            for sgn in (1, -1):
                p2 = {kk: (vv.clone() if isinstance(vv, torch.Tensor) else vv) for kk, vv in proj.items()}
                p2["mean2d"][i, k] += sgn * 1e-6
                col = comp.composite_pixels(p2, px, py)["color"].T.reshape(3, cam.height, cam.width)
                vals.append(float(fidelity_loss([col], [torch.tensor(target[0])], 0.0)))
            fd = (vals[0] - vals[1]) / 2e-6
            assert fd == pytest.approx(float(res["dmean2d"][0][i, k]), rel=1e-5, abs=1e-10)
