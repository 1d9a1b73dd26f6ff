"""Host logic of the block-Jacobi preconditioner (vie_block_layout; no GPU):
the blocks of the cut tiling, each cropped to the box of its body voxels, the
common box and the per-block voxel maps, against a direct NumPy restatement."""
import numpy as np
import pytest

from paper_2508_16471_gb300 import inputs


def _expected(n, mask, cuts):
    ijk = np.argwhere(mask)  # C order == increasing linear index
    tile = np.zeros(len(ijk), dtype=np.int64)
    for a in range(3):
        tile = tile * (len(cuts[a]) + 1) + np.searchsorted(np.asarray(cuts[a], int), ijk[:, a], side="right")
    ids = np.unique(tile)
    lo = {t: ijk[tile == t].min(0) for t in ids}
    hi = {t: ijk[tile == t].max(0) for t in ids}
    box = np.max([hi[t] - lo[t] + 1 for t in ids], axis=0)
    m = -np.ones((len(ids),) + tuple(box), dtype=np.int64)
    for s, t in enumerate(ids):
        for v in np.flatnonzero(tile == t):
            p = ijk[v] - lo[t]
            m[s, p[0], p[1], p[2]] = v
    return tuple(int(b) for b in box), len(ids), m


@pytest.mark.parametrize("case", ["random", "fins", "uncut"])
def test_block_layout_matches_numpy(vielib, case):
    if case == "fins":
        g, eps, _ = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
        cuts = ([32], [32], [])
    elif case == "uncut":
        g, eps = inputs.random_body(5, n_min=20, n_max=20)
        cuts = ([], [], [])
    else:
        g, eps = inputs.random_body(3, n_min=30, n_max=30)
        cuts = ([10, 20], [16], [5, 27])
    mask = eps > 1.0
    vox = np.flatnonzero(mask)
    box, T, m = vielib.block_layout(g.n, vox, cuts)
    box_e, T_e, m_e = _expected(g.n, mask, cuts)
    assert box == box_e and T == T_e
    assert np.array_equal(m, m_e)
    # every body voxel appears exactly once
    got = m[m >= 0]
    assert np.array_equal(np.sort(got), np.arange(len(vox)))


def test_block_layout_rejects_bad_input(vielib):
    n = (8, 8, 8)
    vox = np.array([3, 9, 100])
    with pytest.raises(vielib.VieError):
        vielib.block_layout(n, vox, ([0], [], []))       # cut at the boundary
    with pytest.raises(vielib.VieError):
        vielib.block_layout(n, vox, ([5, 3], [], []))    # not increasing
    with pytest.raises(vielib.VieError):
        vielib.block_layout(n, np.array([9, 3]), ([], [], []))   # voxels not increasing
    with pytest.raises(vielib.VieError):
        vielib.block_layout(n, np.array([3, 600]), ([], [], []))  # outside the grid
