"""Pins of the oracle's identity-feature rendering and dynamics query (Sec. 3.3)."""
import numpy as np
import torch

from oracle import composite as comp
from oracle import dynamics as dyn
from oracle import grad as og
from paper_2411_14847_gb300 import synth

from test_oracle_fd import _scene


def test_feature_render_against_scalar_loop():
    """One-hot features render each Gaussian's blend weight; weighting the colours with them gives
    the colour of the independent scalar compositing loop, and all-one features give 1 - T."""
    arrays, cam = _scene(3, n=6, size=10, deg=0)
    proj = og.project_all(arrays, [cam], 0)[0]
    n = proj["mean2d"].shape[0]
    w = dyn.render_features(proj, np.eye(n), cam.width, cam.height).numpy()
    ones = dyn.render_features(proj, np.ones((n, 4)), cam.width, cam.height).numpy()
    rgb = proj["rgb"].numpy()
    for y in range(cam.height):
        for x in range(cam.width):
            col, T, _ = comp.composite_reference_loop(proj, x, y)
            np.testing.assert_allclose(w[y, x] @ rgb, np.asarray(col), rtol=0, atol=1e-12)
            np.testing.assert_allclose(ones[y, x], 1.0 - T, rtol=0, atol=1e-12)


def test_object_ids_and_dynamic_query_hand_case():
    W = np.eye(3)
    b = np.zeros(3)
    x = np.array([[0.9, 0.1, 0.0], [0.2, 0.2, 0.1], [0.0, 0.3, 0.7], [0.1, 0.6, 0.2]])
    ids = dyn.object_ids(x, W, b)
    assert ids.tolist() == [0, 0, 2, 1]                     # the tie in row 1 goes to class 0
    area = np.array([0, 1, 1, 1])
    assert dyn.dynamic_objects(ids, area, 3, 1).tolist() == [True, True, True]
    assert dyn.dynamic_objects(ids, np.array([1, 1, 0, 0]), 3, 2).tolist() == [True, False, False]
    g = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    assert dyn.dynamic_gaussians(g, W, b, np.array([False, True, False])).tolist() == [False, True, False]
