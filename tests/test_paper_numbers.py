"""Numbers the paper prints (tests/golden/paper_numbers.json, each cited)."""
import json
import os

from paper_2508_16471_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_pb_rotation_increment():
    g = GOLD["pb_rotation_increment_deg"]
    p = g["inputs"]["pitch_nm"] / g["inputs"]["lambda_nm"]
    v = inputs.pb_rotation_increment_deg(pitch=p, theta_t_deg=g["inputs"]["theta_t_deg"])
    assert abs(v - g["value"]) <= g["tol"]


def test_fraunhofer_distance():
    g = GOLD["fraunhofer"]
    rf = 2.0 * g["D_lambda"] ** 2  # in wavelengths
    assert rf == g["R_F_lambda"]
    assert abs(rf * g["lambda_nm"] * 1e-6 - g["R_F_mm"]) < 0.005


def test_unknowns_are_three_per_cell():
    g = GOLD["metasurface_mesh"]
    assert g["unknowns"] == 3 * g["cells"]


def test_metasurface_geometry_uses_design_rule():
    grid, eps, ang = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
    import math
    step = math.radians(inputs.pb_rotation_increment_deg())
    assert abs((ang[1, 0] - ang[0, 0]) - step) < 1e-15
    assert abs(ang[0, 1] - ang[0, 0]) < 1e-15
    assert set(float(v) for v in set(eps.ravel().tolist())) == {1.0, 5.8}
