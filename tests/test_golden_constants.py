"""The constants and worked values the paper prints (tests/golden/paper_constants.txt, each line
cited) against the host-side defaults of the library and the oracle's Alg. 1."""
import inspect
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        body = line.split("#", 1)[0].split()
        if body:
            rows.setdefault(body[0], []).append([float(v) for v in body[1:]])
    return rows


def test_schedule_and_inheritance_period():
    from paper_2411_14847_gb300 import timestep
    g = _golden()
    assert tuple(timestep.PAPER_SCHEDULE) == tuple(int(v) for v in g["schedule_s1_s2_s3"][0])
    erase = inspect.signature(timestep.Timestep.__init__).parameters["erase_every"].default
    assert erase == int(g["erase_every"][0][0])


def test_deformation_field_sizes():
    from paper_2411_14847_gb300 import timestep
    g = _golden()
    p = inspect.signature(timestep.FieldShiftStage.__init__).parameters
    feats, log2t = p["dyn_spec"].default
    assert (log2t, feats) == tuple(int(v) for v in g["hash_dyn_log2T_F"][0])
    feats, log2t = p["st_spec"].default
    assert (log2t, feats) == tuple(int(v) for v in g["hash_st_log2T_F"][0])


def test_identity_encoding_width_is_supported():
    from paper_2411_14847_gb300 import dass
    assert int(_golden()["identity_dims"][0][0]) in dass.FEATURE_WIDTHS


def test_alg1_worked_values():
    """The oracle's Alg. 1 pixel formula at hand-evaluated points: a camera looking down +z whose
    full projection maps x to x_norm exactly (fx = W/2 at unit depth, centred principal point)."""
    from oracle import stages
    from paper_2411_14847_gb300 import synth
    for W, xn, want in _golden()["alg1"]:
        W = int(W)
        cam = synth.pinhole(np.eye(4), W, W)
        cam.fx = cam.fy = W / 2.0
        cam.cx = cam.cy = (W - 1) / 2.0
        xc, _, ph = stages.alg1_pixels(np.array([[xn, 0.0, 1.0]]), cam)
        assert ph[0] > 0
        assert math.floor(xc[0] + 0.5) == int(want), (W, xn, xc[0])
