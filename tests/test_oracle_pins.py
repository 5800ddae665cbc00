"""Pins of the FP64 oracle against closed forms, library routines, brute force and invariants.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign,
a transposed operand, a reversed depth order) fails at least one of them.
"""
import math

import numpy as np
import pytest
import torch

from oracle import binning, composite as comp, gaussians as G, loss as L, stages as S
from oracle import grad as og
from paper_2411_14847_gb300 import synth

DT = torch.float64


def _cam(width=32, height=24, fx=40.0, fy=44.0, vm=None):
    if vm is None:
        vm = np.eye(4)
        vm[2, 3] = 4.0
    return synth.Camera(vm, fx, fy, (width - 1) / 2.0, (height - 1) / 2.0, width, height)


def _proj_of(means, log_s, quats, logit, sh, deg, cam):
    s, qn, o = G.activate(torch.tensor(log_s, dtype=DT), torch.tensor(quats, dtype=DT),
                          torch.tensor(logit, dtype=DT))
    return G.project(torch.tensor(means, dtype=DT), s, qn, o, torch.tensor(sh, dtype=DT), deg, cam)


# ------------------------------------------------------------- projection / EWA

def test_isotropic_on_axis_closed_form():
    # Isotropic Gaussian at the origin seen from z = -4: Sigma2D = (f^2 s^2 / Z^2 + 0.3) I, mean = (cx, cy).
    cam = _cam(fx=50.0, fy=50.0)
    s = 0.05
    p = _proj_of(np.zeros((1, 3)), np.full((1, 3), math.log(s)), np.array([[1.0, 0, 0, 0]]), np.zeros(1),
                 np.zeros((1, 1, 3)), 0, cam)
    expect = 50.0 ** 2 * s * s / 16.0 + 0.3
    a, b, c = p["cov2d"][0].tolist()
    assert a == pytest.approx(expect, rel=1e-12) and c == pytest.approx(expect, rel=1e-12)
    assert abs(b) < 1e-15
    assert p["mean2d"][0].tolist() == pytest.approx([cam.cx, cam.cy], abs=1e-12)
    assert p["conic"][0].tolist() == pytest.approx([1 / expect, 0.0, 1 / expect], rel=1e-12)
    assert float(p["depth"][0]) == pytest.approx(4.0)


def test_isotropic_off_axis_jacobian_closed_form():
    # Sigma = s^2 I, so Sigma2D = s^2 J J^T + 0.3 I with the EWA Jacobian at (X, Y, Z).
    cam = _cam(fx=40.0, fy=44.0)
    X, Y, Zw = 0.7, -0.4, 1.0
    s = 0.1
    p = _proj_of(np.array([[X, Y, Zw]]), np.full((1, 3), math.log(s)), np.array([[0.3, 0.1, -0.5, 0.8]]),
                 np.zeros(1), np.zeros((1, 1, 3)), 0, cam)
    Z = Zw + 4.0
    fx, fy = 40.0, 44.0
    a = s * s * (fx * fx / Z ** 2 + fx * fx * X * X / Z ** 4) + 0.3
    b = s * s * (fx * fy * X * Y / Z ** 4)
    c = s * s * (fy * fy / Z ** 2 + fy * fy * Y * Y / Z ** 4) + 0.3
    assert p["cov2d"][0].tolist() == pytest.approx([a, b, c], rel=1e-10)
    assert p["mean2d"][0].tolist() == pytest.approx([fx * X / Z + cam.cx, fy * Y / Z + cam.cy], rel=1e-12)


def test_near_plane_cull():
    cam = _cam()
    p = _proj_of(np.array([[0, 0, -3.85], [0, 0, -3.75]]), np.full((2, 3), -3.0), np.tile([1.0, 0, 0, 0], (2, 1)),
                 np.zeros(2), np.zeros((2, 1, 3)), 0, cam)
    assert p["valid"].tolist() == [False, True]   # Z = 0.15 culled, Z = 0.25 kept


# ------------------------------------------------------------- quaternions

def test_quaternion_identities():
    rng = np.random.default_rng(0)
    q1 = torch.tensor(rng.normal(size=(5, 4)), dtype=DT)
    q1 = q1 / q1.norm(dim=-1, keepdim=True)
    q2 = torch.tensor(rng.normal(size=(5, 4)), dtype=DT)
    q2 = q2 / q2.norm(dim=-1, keepdim=True)
    R1, R2 = G.quat_to_rotmat(q1), G.quat_to_rotmat(q2)
    # Hamilton product composes rotations in order: R(q1 x q2) = R(q1) R(q2)
    assert torch.allclose(G.quat_to_rotmat(G.quat_mul(q1, q2)), R1 @ R2, atol=1e-12)
    assert torch.allclose(R1 @ R1.transpose(-1, -2), torch.eye(3, dtype=DT).expand(5, 3, 3), atol=1e-12)
    conj = q1 * torch.tensor([1.0, -1, -1, -1], dtype=DT)
    assert torch.allclose(G.quat_mul(q1, conj), torch.tensor([1.0, 0, 0, 0], dtype=DT).expand(5, 4), atol=1e-12)
    # 90 degrees about +z maps +x to +y
    qz = torch.tensor([[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]], dtype=DT)
    assert torch.allclose(G.quat_to_rotmat(qz)[0] @ torch.tensor([1.0, 0, 0], dtype=DT),
                          torch.tensor([0.0, 1, 0], dtype=DT), atol=1e-12)


def test_covariance_closed_form():
    # Rotation of 90 degrees about z swaps the x/y scales.
    q = torch.tensor([[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]], dtype=DT)
    s = torch.tensor([[0.3, 0.1, 0.2]], dtype=DT)
    sig = G.covariance3d(s, q)[0]
    assert torch.allclose(sig, torch.diag(torch.tensor([0.01, 0.09, 0.04], dtype=DT)), atol=1e-12)


# ------------------------------------------------------------- spherical harmonics

def _real_sh_scipy(l, m, dirs):
    from scipy.special import sph_harm_y
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    yc = sph_harm_y(l, abs(m), theta, phi)
    sign = (-1) ** abs(m)                       # undo the Condon-Shortley phase
    return math.sqrt(2) * sign * (np.real(yc) if m > 0 else np.imag(yc))


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    basis = G.sh_basis(torch.tensor(d, dtype=DT), 3).numpy()
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(basis[:, k], _real_sh_scipy(l, m, d), rtol=1e-10, atol=1e-12)
            k += 1


def test_sh_basis_orthonormal_and_low_order_forms():
    # Quadrature on a Gauss-Legendre x uniform-phi grid integrates degree <= 6 products exactly.
    zs, wz = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * 2 * math.pi / 24
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    W = np.outer(wz, np.full(24, 2 * math.pi / 24)).reshape(-1)
    r = np.sqrt(1 - Z ** 2)
    d = np.stack([r * np.cos(P), r * np.sin(P), Z], -1).reshape(-1, 3)
    B = G.sh_basis(torch.tensor(d, dtype=DT), 3).numpy()
    gram = (B * W[:, None]).T @ B
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)
    # degree 0/1 closed forms: Y00 = 1/(2 sqrt(pi)), Y_{1,1} = sqrt(3/(4 pi)) x
    assert B[0, 0] == pytest.approx(0.5 / math.sqrt(math.pi))
    np.testing.assert_allclose(B[:, 3], math.sqrt(3 / (4 * math.pi)) * d[:, 0], atol=1e-12)


def test_sh_degree0_colour():
    rgb = np.array([0.2, 0.5, 0.9])
    dc = (rgb - 0.5) * 2 * math.sqrt(math.pi)
    out = G.sh_to_rgb(torch.tensor(dc[None, None, :], dtype=DT), torch.tensor([[0.0, 0, 1]], dtype=DT), 0)
    np.testing.assert_allclose(out[0].numpy(), rgb, atol=1e-12)
    clamped = G.sh_to_rgb(torch.tensor([[[-5.0, 0, 0]]], dtype=DT), torch.tensor([[0.0, 0, 1]], dtype=DT), 0)
    assert float(clamped[0, 0]) == 0.0


# ------------------------------------------------------------- compositing

def _manual_proj(mean2d, conic, opacity, rgb, depth):
    n = len(depth)
    return dict(mean2d=torch.tensor(mean2d, dtype=DT), conic=torch.tensor(conic, dtype=DT),
                opacity=torch.tensor(opacity, dtype=DT), rgb=torch.tensor(rgb, dtype=DT),
                depth=torch.tensor(depth, dtype=DT), valid=torch.ones(n, dtype=torch.bool))


def test_single_gaussian_footprint_closed_form():
    conic = [0.2, 0.05, 0.1]
    proj = _manual_proj([[5.3, 4.1]], [conic], [0.8], [[0.9, 0.4, 0.1]], [2.0])
    px, py = comp.pixel_grid(12, 10)
    r = comp.composite_pixels(proj, px, py)
    dx, dy = px.numpy() - 5.3, py.numpy() - 4.1
    a = np.minimum(0.99, 0.8 * np.exp(-0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) - conic[1] * dx * dy))
    a = np.where(a >= 1 / 255, a, 0.0)
    np.testing.assert_allclose(r["color"].numpy(), a[:, None] * np.array([0.9, 0.4, 0.1])[None], atol=1e-14)
    np.testing.assert_allclose(r["T_final"].numpy(), 1 - a, atol=1e-14)


def test_two_gaussians_nearer_first():
    # Both centred on pixel (2, 2); the nearer one (depth 1) is blended first.
    proj = _manual_proj([[2.0, 2.0], [2.0, 2.0]], [[1, 0, 1], [1, 0, 1]], [0.3, 0.6],
                        [[1.0, 0, 0], [0, 1.0, 0]], [5.0, 1.0])
    r = comp.composite_pixels(proj, torch.tensor([2.0], dtype=DT), torch.tensor([2.0], dtype=DT))
    a_near, a_far = 0.6, 0.3
    expect = [a_far * (1 - a_near), a_near, 0.0]         # c1 a1 + c2 a2 (1 - a1), near = green
    np.testing.assert_allclose(r["color"][0].numpy(), expect, atol=1e-15)
    assert float(r["T_final"][0]) == pytest.approx((1 - a_near) * (1 - a_far))
    assert int(r["n_last"][0]) == 0                       # index of the far (last added) Gaussian


def test_stop_rule_excludes_the_stopping_gaussian():
    # alphas 0.99, 0.99: after the first T = 0.01; T(1 - 0.99) = 1e-4 is not < 1e-4 -> added;
    # the third (0.5) would give 5e-5 < 1e-4 -> excluded and the pixel stops.
    proj = _manual_proj([[0.0, 0.0]] * 3, [[1, 0, 1]] * 3, [1.0, 1.0, 1.0],
                        [[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]], [1.0, 2.0, 3.0])
    proj["opacity"] = torch.tensor([1.0, 1.0, 0.5], dtype=DT)
    r = comp.composite_pixels(proj, torch.tensor([0.0], dtype=DT), torch.tensor([0.0], dtype=DT))
    T2 = 0.01 * 0.01
    if T2 < 1e-4:          # float64 rounding of 0.01*0.01 decides whether the 2nd stops too
        expect = [0.99, 0.0, 0.0]
        t_fin = 0.01
    else:
        expect = [0.99, 0.0099, 0.0]
        t_fin = T2
    np.testing.assert_allclose(r["color"][0].numpy(), expect, atol=1e-15)
    assert float(r["T_final"][0]) == pytest.approx(t_fin)
    # a third Gaussian that would bring T below 1e-4 is never added
    assert float(r["color"][0, 2]) == 0.0


def test_skip_below_one_over_255():
    proj = _manual_proj([[0.0, 0.0], [0.0, 0.0]], [[1, 0, 1]] * 2, [0.0039, 0.5], [[1.0, 0, 0], [0, 1.0, 0]],
                        [1.0, 2.0])
    r = comp.composite_pixels(proj, torch.tensor([0.0], dtype=DT), torch.tensor([0.0], dtype=DT))
    np.testing.assert_allclose(r["color"][0].numpy(), [0.0, 0.5, 0.0], atol=1e-15)
    assert int(r["n_contrib"][0]) == 1


def _tiny_scene(seed, n=8, size=8):
    rng = np.random.default_rng(seed)
    cam = _cam(size, size, fx=size * 1.2, fy=size * 1.2)
    means = rng.uniform(-0.8, 0.8, (n, 3))
    return dict(means=means, log_scales=rng.normal(-1.8, 0.3, (n, 3)), quats=rng.normal(size=(n, 4)),
                opacity_logit=rng.normal(0.5, 1.0, n), sh=rng.normal(0, 0.6, (n, 4, 3))), cam


def test_brute_force_scalar_loop_matches_vectorised():
    for seed in range(4):
        arrays, cam = _tiny_scene(seed)
        proj = og.project_all(arrays, [cam], 1)[0]
        px, py = comp.pixel_grid(cam.width, cam.height)
        r = comp.composite_pixels(proj, px, py)
        for p in range(px.shape[0]):
            col, T, last = comp.composite_reference_loop(proj, float(px[p]), float(py[p]))
            np.testing.assert_allclose(r["color"][p].numpy(), col, atol=1e-13)
            assert float(r["T_final"][p]) == pytest.approx(T, abs=1e-14)
            assert int(r["n_last"][p]) == last


def test_brute_force_permutation_invariance():
    # The image depends on the depth order only: relabelling the Gaussians changes nothing.
    arrays, cam = _tiny_scene(7)
    perm = np.random.default_rng(3).permutation(8)
    a2 = {k: v[perm] for k, v in arrays.items()}
    i1 = og.render(arrays, [cam], 1)[0]["image"]
    i2 = og.render(a2, [cam], 1)[0]["image"]
    assert torch.allclose(i1, i2, atol=1e-14)


def test_compositing_invariants():
    sc, cams = synth.config_a()
    sub = {k: v[:400] for k, v in sc.arrays().items()}
    proj = og.project_all(sub, cams, 0)[0]
    order = comp.depth_order(proj)
    px, py = comp.pixel_grid(128, 128)
    sel = torch.arange(0, px.shape[0], 37)
    r = comp.composite_pixels(proj, px[sel], py[sel], order=order)
    # sum of weights + T_final = 1 with a constant white colour
    white = dict(proj, rgb=torch.ones_like(proj["rgb"]))
    rw = comp.composite_pixels(white, px[sel], py[sel], order=order)
    np.testing.assert_allclose((rw["color"][:, 0] + rw["T_final"]).numpy(), 1.0, atol=1e-12)
    assert bool((r["T_final"] > 0).all()) and bool((r["T_final"] <= 1).all())
    assert float(r["color"].min()) >= 0.0
    assert float(r["color"].max()) <= float(proj["rgb"].max()) + 1e-12


def test_sh0_constant_colour_image_equals_rgb_times_coverage():
    sc, cams = synth.config_a()
    sub = {k: v[:300].copy() for k, v in sc.arrays().items()}
    sub["sh"][:] = np.float32((0.7 - 0.5) * 2 * math.sqrt(math.pi))
    r = og.render(sub, cams, 0)[0]
    np.testing.assert_allclose(r["image"].numpy(), np.broadcast_to(0.7 * (1 - r["T_final"].numpy())[None], (3, 128, 128)),
                               atol=1e-6)


def test_alternatives_cover_the_plain_result():
    arrays, cam = _tiny_scene(11)
    proj = og.project_all(arrays, [cam], 1)[0]
    col, T, _ = comp.composite_reference_loop(proj, 3.0, 4.0)
    alts = comp.pixel_alternatives(proj, 3.0, 4.0)
    assert any(np.allclose(a[0], col, atol=1e-13) for a in alts)


# ------------------------------------------------------------- footprint / binning

def test_footprint_radius_contains_alpha_footprint():
    sc, cams = synth.config_a()
    proj = og.project_all(sc.arrays(), cams, 0)[0]
    r = G.footprint_radius(proj["cov2d"], proj["opacity"])
    px, py = comp.pixel_grid(128, 128)
    idx = torch.nonzero(proj["valid"]).flatten()[:200]
    a = comp.alpha_matrix(proj["mean2d"][idx], proj["conic"][idx], proj["opacity"][idx], px, py)
    dist = torch.maximum((px[:, None] - proj["mean2d"][idx, 0][None]).abs(),
                         (py[:, None] - proj["mean2d"][idx, 1][None]).abs())
    inside = dist <= r[idx][None]
    assert bool(((a >= 1 / 255) <= inside).all())


def test_binning_hand_example_and_ties():
    cams = [_cam(64, 64), _cam(64, 64)]          # 4 x 4 tiles of 16 px per camera
    u = np.array([20.0, 28.0, 20.0, 40.0])
    v = np.array([5.0, 28.0, 8.0, 40.0])
    sig = np.array([2.0, 1.5, 1.0, 1.5])          # isotropic footprints: conic = I / sigma^2
    conic = np.stack([1 / sig ** 2, np.zeros(4), 1 / sig ** 2], 1)
    opac = np.ones(4)                             # k2 = 2 ln 255 + 0.01 = 11.102
    rad = np.array([7, 5, 4, 0])                  # record 3 is invisible
    cam_of = np.array([0, 0, 0, 1])
    sure, maybe, total = binning.bin_records(u, v, conic, opac, rad, cam_of, cams, 16)
    assert total == 32 and not maybe
    # record 1 at (28, 28): the corner tile (2, 2) is out (nearest pixel centre (32, 32) has
    # q = 32 / 2.25 = 14.2 > k2) although the square of radius 5 would overlap it
    assert sure == {0: {0}, 1: {0, 2}, 5: {1}, 6: {1}, 9: {1}}
    assert sorted(sure[1], key=lambda r: binning.order_key([3.0, 2.0, 3.0, 1.0][r], r)) == [0, 2]
    assert binning.rect_min_quadratic(1.0, 0.0, 1.0, 3.0, 5.0, -1.0, 1.0) == 9.0
    assert binning.rect_min_quadratic(2.0, 1.0, 1.0, 1.0, 2.0, -10.0, 10.0) == pytest.approx(1.0)  # y = -x


# ------------------------------------------------------------- loss

def test_ssim_self_is_one_and_direct_loop():
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.uniform(size=(3, 9, 13)), dtype=DT)
    y = torch.tensor(rng.uniform(size=(3, 9, 13)), dtype=DT)
    assert torch.allclose(L.ssim_map(x, x), torch.ones_like(x), atol=1e-12)
    assert torch.allclose(L.ssim_map(x, y), L.ssim_direct(x, y), atol=1e-12)


def test_ssim_constant_shift_closed_form():
    x = torch.full((3, 30, 30), 0.4, dtype=DT)
    y = torch.full((3, 30, 30), 0.7, dtype=DT)
    m = L.ssim_map(x, y)
    assert float(m[1, 15, 15]) == pytest.approx(L.constant_shift_ssim(0.4, 0.7), rel=1e-12)


def test_ssim_matches_scipy_filter():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(6)
    img = rng.uniform(size=(3, 20, 17))
    g = L.gaussian_window().numpy()
    w2 = np.outer(g, g)
    ref = np.stack([correlate(img[c], w2, mode="constant", cval=0.0) for c in range(3)])
    np.testing.assert_allclose(L._filter(torch.tensor(img, dtype=DT)).numpy(), ref, atol=1e-13)
    assert g.sum() == pytest.approx(1.0) and np.argmax(g) == 5


def test_window_moments_match_scipy_and_constant_images():
    """The target's window statistics (w * y, w * y^2) that the cached-statistics loss reads: SciPy's
    zero-padded correlation of y and of y^2 with the 11 x 11 window, and (c, c^2) for a constant image
    c at pixels whose window lies inside the image (the window sums to one)."""
    from scipy.ndimage import correlate
    rng = np.random.default_rng(16)
    img = rng.uniform(size=(3, 19, 23))
    g = L.gaussian_window().numpy()
    w2 = np.outer(g, g)
    m1, m2 = L.window_moments(torch.tensor(img, dtype=DT))
    for c in range(3):
        np.testing.assert_allclose(m1[c].numpy(), correlate(img[c], w2, mode="constant", cval=0.0), atol=1e-13)
        np.testing.assert_allclose(m2[c].numpy(), correlate(img[c] ** 2, w2, mode="constant", cval=0.0),
                                   atol=1e-13)
    c1, c2 = L.window_moments(torch.full((3, 16, 16), 0.7, dtype=DT))
    np.testing.assert_allclose(c1[:, 5:11, 5:11].numpy(), 0.7, rtol=1e-13)
    np.testing.assert_allclose(c2[:, 5:11, 5:11].numpy(), 0.49, rtol=1e-13)
    assert float(c1[0, 0, 0]) == pytest.approx(0.7 * float(g[5:].sum()) ** 2, rel=1e-13)   # corner: a quarter window


def test_fidelity_loss_l1_closed_form():
    x = torch.full((3, 4, 4), 0.25, dtype=DT)
    y = torch.full((3, 4, 4), 0.75, dtype=DT)
    assert float(L.fidelity_loss([x], [y], 0.0)) == pytest.approx(0.5)
    loss, g = L.loss_and_image_grad([x], [y], 0.0)
    assert torch.allclose(g[0], torch.full_like(x, -1.0 / 48))


# ------------------------------------------------------------- Adam

def test_adam_first_step_closed_form_and_untouched_rows():
    rng = np.random.default_rng(2)
    p = rng.normal(size=(6, 7))
    g = rng.normal(size=(6, 7))
    z = np.zeros_like(p)
    rows = np.array([1, 4])
    p1, m1, v1 = S.adam(p, g, z, z, 1, lr=1e-3, rows=rows)
    np.testing.assert_allclose(p1[rows], p[rows] - 1e-3 * np.sign(g[rows]), atol=1e-12)
    other = np.setdiff1d(np.arange(6), rows)
    assert np.array_equal(p1[other], p[other]) and not m1[other].any() and not v1[other].any()
    np.testing.assert_allclose(m1[rows], 0.1 * g[rows])
    np.testing.assert_allclose(v1[rows], 0.001 * g[rows] ** 2)


def test_adam_constant_gradient_second_step():
    # With a constant gradient the bias-corrected ratio stays sign(g): two steps move 2 lr.
    p, m, v = S.adam(np.ones(3), np.array([2.0, -3.0, 0.5]), np.zeros(3), np.zeros(3), 1, lr=0.1)
    p, m, v = S.adam(p, np.array([2.0, -3.0, 0.5]), m, v, 2, lr=0.1)
    np.testing.assert_allclose(p, [0.8, 1.2, 0.8], atol=1e-12)


# ------------------------------------------------------------- shift / inheritance

def test_shift_identity_and_rotation():
    rng = np.random.default_rng(4)
    means = rng.normal(size=(10, 3))
    quats = rng.normal(size=(10, 4))
    idx = np.array([2, 5, 7])
    off = np.zeros((3, 7))
    off[:, 3] = 2.0                                   # unnormalised identity rotation offset
    m2, q2 = S.shift(means, quats, idx, off)
    np.testing.assert_allclose(m2.numpy(), means)
    qn = quats / np.linalg.norm(quats, axis=1, keepdims=True)
    np.testing.assert_allclose(q2[idx].numpy(), qn[idx], atol=1e-15)
    other = np.setdiff1d(np.arange(10), idx)
    np.testing.assert_array_equal(q2[other].numpy(), quats[other])
    # sigma = conj(norm(q)) undoes the rotation: q' = identity
    off2 = np.zeros((3, 7))
    off2[:, 0] = [0.1, 0.2, 0.3]
    off2[:, 3:] = qn[idx] * np.array([1, -1, -1, -1]) * 3.0
    m3, q3 = S.shift(means, quats, idx, off2)
    np.testing.assert_allclose(q3[idx].numpy(), np.tile([1.0, 0, 0, 0], (3, 1)), atol=1e-14)
    np.testing.assert_allclose(m3[idx].numpy(), means[idx] + off2[:, :3], atol=1e-15)
    m4, q4 = S.shift(means, quats, np.zeros(0, np.int64), np.zeros((0, 7)))
    np.testing.assert_array_equal(m4.numpy(), means)


def test_inheritance_copy():
    arrays = dict(means=np.arange(18.0).reshape(6, 3), opacity_logit=np.arange(6.0))
    is_var = np.array([0, 0, 0, 1, 1, 1], bool)
    m = np.array([0.0, 0.0, 0.0, 1.0, 0.0, -2.0])
    out, nv, remap = S.inherit(arrays, is_var, m, t=3)
    assert out["opacity_logit"].tolist() == [0, 1, 2, 3]          # m = 0 quantises to 0
    assert nv.tolist() == [False, False, False, True] and remap.tolist() == [0, 1, 2, 3, -1, -1]
    out, nv, _ = S.inherit(arrays, is_var, np.ones(6), t=5)
    assert np.array_equal(out["means"], arrays["means"])
    out, nv, _ = S.inherit(arrays, is_var, np.ones(6), t=20)       # erased every 20 timesteps
    assert out["opacity_logit"].tolist() == [0, 1, 2] and not nv.any()


# ------------------------------------------------------------- error guidance

def test_percentile_matches_numpy_lower():
    e = np.random.default_rng(9).uniform(size=(37, 29)).astype(np.float32)
    assert S.percentile_lower(e, 0.95) == np.percentile(e, 95, method="lower")
    assert S.error_bitmap(e, S.percentile_lower(e)).sum() == e.size - 1 - int(math.floor(0.95 * (e.size - 1)))


def test_error_map_f32():
    a = np.zeros((3, 2, 2), np.float32)
    b = np.zeros((3, 2, 2), np.float32)
    b[:, 0, 1] = [0.3, -0.3, 0.6]
    np.testing.assert_array_equal(S.error_map_f32(a, b), np.array([[0, 0.4], [0, 0]], np.float32))


def test_alg1_centre_and_consistency_with_projection():
    cam = synth.config_a()[1][0]
    xc, yc, w = S.alg1_pixels(np.array([[0.0, 0.0, 0.0]]), cam)
    assert xc[0] == pytest.approx(63.5) and yc[0] == pytest.approx(63.5) and w[0] == pytest.approx(4.0)
    pts = np.random.default_rng(0).uniform(-1, 1, (50, 3))
    xc, yc, _ = S.alg1_pixels(pts, cam)
    proj = og.project_all(dict(means=pts, log_scales=np.zeros((50, 3)), quats=np.tile([1.0, 0, 0, 0], (50, 1)),
                               opacity_logit=np.zeros(50), sh=np.zeros((50, 1, 3))), [cam], 0)[0]
    np.testing.assert_allclose(xc, proj["mean2d"][:, 0].numpy(), atol=1e-9)
    np.testing.assert_allclose(yc, proj["mean2d"][:, 1].numpy(), atol=1e-9)


def test_error_subset_hand_example():
    cam = _cam(8, 6, fx=8.0, fy=8.0)
    D = np.zeros((6, 8), bool)
    D[2, 5] = True
    # a point projecting to (5, 2): X/Z = (5 - 3.5)/8, Y/Z = (2 - 2.5)/8 at Z = 4
    pt = np.array([[1.5 / 8 * 4, -0.5 / 8 * 4, 0.0], [0.0, 0.0, -10.0]])
    s, amb = S.error_subset(pt, [cam], [D])
    assert s.tolist() == [True, False] and not amb.any()


def test_densify_select_eq4():
    g = np.array([5.0, 1.0, 3.0, 3.0, 0.5, 9.0], np.float32)
    s_err = np.array([0, 1, 0, 1, 1, 0], bool)
    base = np.array([1, 1, 1, 1, 1, 0], bool)
    # tau_pos = 2.5: {0, 2, 3}; S_err n g > 0.8: {1, 3}; var row 5 excluded
    sel = S.densify_select(g, s_err, base, 2.5, 0.8, 10)
    assert sel.tolist() == [0, 1, 2, 3]
    assert S.densify_select(g, s_err, base, 2.5, 0.8, 2).tolist() == [0, 2]


def test_spawn_rule():
    arrays = dict(means=np.array([[1.0, 2, 3], [0, 0, 0]]), log_scales=np.log(np.array([[0.1, 0.2, 0.3]] * 2)),
                  quats=np.array([[2.0, 0, 0, 0], [1.0, 0, 0, 0]]), opacity_logit=np.array([0.3, 0.4]),
                  sh=np.zeros((2, 1, 3)))
    z = np.array([[1.0, -1.0, 2.0], [0, 0, 0]])
    out = S.spawn(arrays, [0], z)
    np.testing.assert_allclose(out["means"][0], [1.1, 1.8, 3.6])
    np.testing.assert_allclose(out["log_scales"][0], np.log(np.array([0.1, 0.2, 0.3]) / 1.6))


def test_mean_grad_and_ndc_norm():
    assert S.mean_grad_f32([3.0, 1.0], [2, 0]).tolist() == [1.5, 0.0]
    assert float(S.ndc_grad_norm(torch.tensor([[3.0 / 50, 4.0 / 20]]), 100, 40)[0]) == pytest.approx(5.0)


def test_prune_low_opacity_closed_form():
    """Sec. 3.4 pruning: base rows always kept; var rows kept iff opacity > threshold; layout
    base-then-var with each group's order preserved."""
    from oracle.stages import prune_low_opacity
    logit = np.array([-9.0, 2.0, -6.0, -4.0, 0.0, -5.5])     # opacities ~1.2e-4, .88, 2.5e-3, .018, .5, 4.1e-3
    is_var = np.array([0, 1, 1, 0, 1, 1], dtype=bool)
    arrays = {"opacity_logit": logit, "means": np.arange(18.0).reshape(6, 3)}
    out, new_var = prune_low_opacity(arrays, is_var, 0.005)
    assert out["opacity_logit"].tolist() == [-9.0, -4.0, 2.0, 0.0]
    assert out["means"][:, 0].tolist() == [0.0, 9.0, 3.0, 12.0]
    assert new_var.tolist() == [False, False, True, True]


# ------------------------------------------------------------- densification-statistics visibility

def _stats_proj(u, v, sigma, opacity, valid=True):
    """Projection dict of isotropic splats: cov2d = sigma^2 I, so lambda_max = sigma^2 exactly."""
    n = len(u)
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    return dict(mean2d=torch.tensor(np.stack([u, v], 1), dtype=DT),
                cov2d=torch.tensor(np.stack([s2, np.zeros(n), s2], 1), dtype=DT),
                opacity=torch.tensor(opacity, dtype=DT),
                valid=torch.tensor(np.broadcast_to(valid, (n,)).copy(), dtype=torch.bool))


def test_stats_visible_edges_near_plane_and_opacity():
    """Visibility rule of the positional-gradient statistics (Sec. 3.4, reading: radius > 0 and
    the square of half-side r around mean2D overlapping the pixel-centre box [0, W-1] x [0, H-1]).
    sigma = 2 px and opacity 1 give r = ceil(2 sqrt(2 ln 255 + 0.01)) = ceil(6.664) = 7, so a
    splat is visible exactly while its centre lies within 7 px outside an edge: each edge is
    probed at r (visible) and r + 1 (not), plus half-pixel offsets."""
    cam = _cam(32, 24)
    W, H = 32, 24
    r = 7
    assert math.ceil(2.0 * math.sqrt(2.0 * math.log(255.0) + 0.01)) == r
    cx, cy = 15.0, 11.0
    cases = [  # (u, v, visible)
        (-r, cy, True), (-r - 1, cy, False), (-r + 0.5, cy, True), (-r - 0.5, cy, False),
        (W - 1 + r, cy, True), (W - 1 + r + 1, cy, False), (W - 1 + r - 0.5, cy, True), (W - 1 + r + 0.5, cy, False),
        (cx, -r, True), (cx, -r - 1, False), (cx, -r - 0.5, False),
        (cx, H - 1 + r, True), (cx, H - 1 + r + 1, False), (cx, H - 1 + r + 0.5, False),
        (-r, -r, True), (W - 1 + r, H - 1 + r, True), (-r - 1, H - 1 + r, False),   # corners
    ]
    u = np.array([c[0] for c in cases], dtype=np.float64)
    v = np.array([c[1] for c in cases], dtype=np.float64)
    vis = og.stats_visible(_stats_proj(u, v, np.full(len(cases), 2.0), np.ones(len(cases))), cam)
    assert vis.tolist() == [c[2] for c in cases]
    # behind the near plane (valid = False): never visible, even at the image centre
    assert og.stats_visible(_stats_proj([cx], [cy], [2.0], [1.0], valid=False), cam).tolist() == [False]
    # 255 o <= 1 has no footprint (r = 0); just above 1/255 the radius is 1 and a centred splat counts
    o = np.array([1.0 / 255.0, 0.0039, 0.004])
    vis = og.stats_visible(_stats_proj(np.full(3, cx), np.full(3, cy), np.full(3, 2.0), o), cam)
    assert vis.tolist() == [False, False, True]
    # the radius, not the centre, decides: a centre 1 px outside with r = 1 is visible, 2 px is not
    r1 = _stats_proj(np.array([-1.0, -2.0]), np.full(2, cy), np.full(2, 2.0), np.full(2, 0.004))
    assert G.footprint_radius(r1["cov2d"], r1["opacity"]).tolist() == [1.0, 1.0]
    assert og.stats_visible(r1, cam).tolist() == [True, False]


# ------------------------------------------------------------- near-threshold alternatives

def test_alternatives_single_result_away_from_thresholds():
    """Three splats at the pixel with alphas far from 1/255 and T(1 - alpha) far from 1e-4:
    exactly one alternative, equal to the hand-composited colour."""
    proj = _manual_proj([[0.0, 0.0]] * 3, [[1, 0, 1]] * 3, [0.5, 0.3, 0.2],
                        [[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]], [1.0, 2.0, 3.0])
    alts = comp.pixel_alternatives(proj, 0.0, 0.0)
    assert len(alts) == 1
    col, T = alts[0]
    expect = [0.5, 0.3 * 0.5, 0.2 * 0.5 * 0.7]
    np.testing.assert_allclose(col, expect, atol=1e-15)
    assert T == pytest.approx(0.5 * 0.7 * 0.8, abs=1e-15)


def test_alternatives_exactly_two_at_an_alpha_tie():
    """A splat whose alpha is exactly 1/255 at the pixel may be skipped or blended: exactly two
    alternatives, with and without its contribution; 1% above the threshold there is one."""
    a_tie = 1.0 / 255.0
    proj = _manual_proj([[0.0, 0.0]] * 2, [[1, 0, 1]] * 2, [0.5, a_tie], [[1.0, 0, 0], [0, 1.0, 0]], [1.0, 2.0])
    alts = comp.pixel_alternatives(proj, 0.0, 0.0)
    assert len(alts) == 2
    cols = sorted(tuple(a[0]) for a in alts)
    np.testing.assert_allclose(cols[0], [0.5, 0.0, 0.0], atol=1e-15)             # skipped
    np.testing.assert_allclose(cols[1], [0.5, a_tie * 0.5, 0.0], atol=1e-15)      # blended
    assert sorted(a[1] for a in alts) == pytest.approx([0.5 * (1 - a_tie), 0.5])
    proj["opacity"] = torch.tensor([0.5, 1.01 * a_tie], dtype=DT)
    assert len(comp.pixel_alternatives(proj, 0.0, 0.0)) == 1


def test_alternatives_exactly_two_at_a_stop_tie():
    """T (1 - alpha) within 0.1% of 1e-4 may stop or blend: exactly two alternatives."""
    # alpha 0.99 then alpha 0.99 * (1 - 1e-6): T before the second is 0.01, T(1 - alpha) ~ 1e-4
    a2 = 0.99 * (1.0 - 1e-6)
    proj = _manual_proj([[0.0, 0.0]] * 2, [[1, 0, 1]] * 2, [1.0, a2], [[1.0, 0, 0], [0, 1.0, 0]], [1.0, 2.0])
    alts = comp.pixel_alternatives(proj, 0.0, 0.0)
    assert len(alts) == 2
    cols = sorted(tuple(a[0]) for a in alts)
    np.testing.assert_allclose(cols[0], [0.99, 0.0, 0.0], atol=1e-15)              # stopped
    np.testing.assert_allclose(cols[1], [0.99, a2 * 0.01, 0.0], atol=1e-12)        # blended
