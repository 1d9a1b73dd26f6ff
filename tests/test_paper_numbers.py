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


def test_paper_scale_metasurface_geometry():
    """The paper-scale box (Sec. III-B): 40 x 12 x 2 wavelengths at 62 cells per
    wavelength, fins of 486 x 219 x 830 nm at 1550 nm on the 667 nm pitch, the
    PB rotation step between columns, the height-first grid frame, and
    unit-cell cuts that never split a fin."""
    import math

    import numpy as np
    from scipy import ndimage
    g, eps, info = inputs.metasurface_paper()
    assert info["n_paper"] == (2480, 744, 124) and g.n == (124, 744, 2480)
    assert abs(g.h - 1.0 / 62.0) < 1e-15
    p = 667.0 / 1550.0
    assert info["fins"] == (int(40.0 // p), int(12.0 // p)) == (92, 27)
    ang = info["angles"]
    assert np.allclose(np.diff(ang[:, 0]), math.radians(inputs.pb_rotation_increment_deg()), atol=1e-14)
    assert set(np.unique(eps).tolist()) == {1.0, 3.44 ** 2}
    lab, nf = ndimage.label(eps > 1.0)
    assert nf == 92 * 27
    # one fin holds about l d h / cells^3 voxels (centre rule; rounding of the outline)
    per = np.bincount(lab.ravel())[1:]
    vol = 486 * 219 * 830 / 1550.0 ** 3 / g.h ** 3
    assert abs(per.mean() / vol - 1.0) < 0.05
    assert info["z_cells"] == 34  # 830 nm = 33.2 cells at h = lambda/62
    # vectors map between frames by the x <-> z swap, its own inverse
    v = np.array([0.1, 0.2, 0.3])
    assert np.array_equal(inputs.to_grid_frame(v), v[::-1])
    assert np.array_equal(inputs.to_grid_frame(inputs.to_grid_frame(v)), v)
    # the unit-cell cuts (grid frame) leave every fin inside one block
    cuts = info["cell_cuts"]
    assert cuts[0] == [] and len(cuts[1]) == 26 and len(cuts[2]) == 91
    for s in ndimage.find_objects(lab):
        for a in (1, 2):
            c = np.asarray(cuts[a])
            assert np.searchsorted(c, s[a].start, side="right") == np.searchsorted(c, s[a].stop - 1, side="right")


def test_even_cuts():
    assert inputs.even_cuts(744, 7) == [106, 213, 319, 425, 531, 638]
    assert inputs.even_cuts(10, 1) == []
    c = inputs.even_cuts(2480, 7)
    sizes = [b - a for a, b in zip([0] + c, c + [2480])]
    assert len(c) == 6 and min(sizes) >= 354 and max(sizes) <= 355
