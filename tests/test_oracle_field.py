"""Pins of the oracle's hash-encoding deformation field (Sec. 3.3, App. B.2; I-NGP encoding + MLP)."""
import numpy as np
import pytest
import torch

from oracle import field as fld


def _params(rng, levels, feats, log2t, hidden=64, scale=1e-1):
    T = 1 << log2t
    return {"table": rng.uniform(-scale, scale, (levels, T, feats)),
            "w1": rng.normal(0, 0.3, (hidden, levels * feats)), "b1": rng.normal(0, 0.1, hidden),
            "w2": rng.normal(0, 0.3, (7, hidden)), "b2": rng.normal(0, 0.1, 7)}


def _t(p):
    return {k: torch.as_tensor(v) for k, v in p.items()}


def test_level_resolutions_closed_forms():
    """Level sizes grow geometrically from n_min to n_max: with n_max / n_min = 2^(levels - 1) every
    level doubles exactly; one level is n_min alone, two are the ends; the 16-level 16..2048 grid is
    strictly increasing from 16 to 2048 with a nearly constant ratio (128^(1/15) ~ 1.38)."""
    assert fld.level_resolutions(8, 16, 2048) == [16 << l for l in range(8)]
    assert fld.level_resolutions(5, 8, 128) == [8, 16, 32, 64, 128]
    assert fld.level_resolutions(1, 16, 2048) == [16]
    assert fld.level_resolutions(2, 16, 2048) == [16, 2048]
    res = fld.level_resolutions(16, 16, 2048)
    assert res[0] == 16 and res[-1] == 2048 and all(a < b for a, b in zip(res, res[1:]))
    ratios = [b / a for a, b in zip(res, res[1:])]
    assert all(1.33 < r < 1.43 for r in ratios)


def test_dense_level_reproduces_linear_functions():
    """On a densely indexed level, a table holding a linear function of the vertex coordinates is
    interpolated to that same function of x * N (trilinear interpolation is exact on linear
    functions): pins the dense layout, the trilinear weights and the box normalisation."""
    n, log2t = 5, 10                                     # (5+1)^3 = 216 <= 1024: dense
    v = n + 1
    i, j, k = np.meshgrid(np.arange(v), np.arange(v), np.arange(v), indexing="ij")
    idx = (i + v * (j + v * k)).reshape(-1)
    lin = np.stack([0.5 * i - 2.0 * j + 3.0 * k + 1.0, -i + 0.25 * k], axis=-1).reshape(-1, 2)
    table = np.zeros((1, 1 << log2t, 2))
    table[0, idx] = lin
    rng = np.random.default_rng(0)
    lo, hi = np.array([-1.0, -2.0, 0.5]), np.array([1.0, 2.0, 3.0])
    p = rng.uniform(lo, hi, (50, 3))
    enc = fld.encode(p, torch.as_tensor(table), [n], lo, hi).numpy()
    s = (p - lo) / (hi - lo) * n
    want = np.stack([0.5 * s[:, 0] - 2.0 * s[:, 1] + 3.0 * s[:, 2] + 1.0, -s[:, 0] + 0.25 * s[:, 2]], axis=1)
    np.testing.assert_allclose(enc, want, rtol=0, atol=1e-12)


def test_hashed_level_uses_the_spatial_hash():
    """On a hashed level the entry of vertex (a, 0, 0) is row a mod T (first prime 1, the other
    coordinates 0); positions outside the box clamp to its faces."""
    n, log2t = 300, 8                                    # 301^3 >> 256: hashed
    T = 1 << log2t
    table = np.arange(T, dtype=np.float64).reshape(1, T, 1).repeat(2, axis=2)
    lo, hi = np.zeros(3), np.ones(3)
    a = np.array([0, 7, 255, 256, 299])
    p = np.stack([a / n, np.zeros_like(a, dtype=float), np.zeros_like(a, dtype=float)], axis=1)
    enc = fld.encode(p, torch.as_tensor(table), [n], lo, hi).numpy()
    np.testing.assert_allclose(enc[:, 0], (a % T).astype(float), rtol=0, atol=1e-9)
    # clamping: a point beyond the box equals the face point
    e2 = fld.encode(np.array([[2.0, -1.0, 0.0]]), torch.as_tensor(table), [n], lo, hi).numpy()
    e3 = fld.encode(np.array([[1.0, 0.0, 0.0]]), torch.as_tensor(table), [n], lo, hi).numpy()
    np.testing.assert_array_equal(e2, e3)


def test_mlp_closed_forms():
    rng = np.random.default_rng(1)
    prm = _params(rng, 2, 2, 6)
    prm["table"][:] = 0.0                               # encoding 0: out = w2 relu(b1) + b2
    p = rng.uniform(-1, 1, (4, 3))
    off = fld.field_offsets(p, _t(prm), [4, 8], -np.ones(3), np.ones(3)).numpy()
    want = prm["w2"] @ np.maximum(prm["b1"], 0.0) + prm["b2"] + np.array([0, 0, 0, 1.0, 0, 0, 0])
    np.testing.assert_allclose(off, np.broadcast_to(want, off.shape), rtol=1e-12)
    prm["w2"][:] = 0.0                                  # zero output layer: identity rotation + b2
    off = fld.field_offsets(p, _t(prm), [4, 8], -np.ones(3), np.ones(3)).numpy()
    np.testing.assert_allclose(off, np.broadcast_to(prm["b2"] + np.array([0, 0, 0, 1.0, 0, 0, 0]), off.shape))


def test_field_gradients_finite_differences():
    rng = np.random.default_rng(2)
    levels, feats, log2t = 3, 2, 6
    res = [3, 5, 9]                                     # 4^3 = 64 <= T: dense; 6^3, 10^3 > 64: hashed
    prm = _params(rng, levels, feats, log2t, scale=0.5)
    lo, hi = -np.ones(3), np.ones(3)
    p = rng.uniform(-0.9, 0.9, (6, 3))
    d = rng.normal(size=(6, 7))
    grads, _ = fld.field_grads(p, prm, res, lo, hi, d)

    def f(prm2):
        return float((fld.field_offsets(p, _t(prm2), res, lo, hi).numpy() * d).sum())

    h = 1e-6
    for name in ("table", "w1", "b1", "w2", "b2"):
        g = grads[name].numpy()
        flat = np.flatnonzero(np.abs(g) > 1e-8)
        picks = flat[:: max(1, flat.size // 6)][:6] if flat.size else [0]
        for idx in picks:
            pp = {k: v.copy() for k, v in prm.items()}
            pm = {k: v.copy() for k, v in prm.items()}
            pp[name].flat[idx] += h
            pm[name].flat[idx] -= h
            fd = (f(pp) - f(pm)) / (2 * h)
            assert g.flat[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, idx)
