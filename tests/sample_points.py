"""Voxel picks for the sampled checks at sizes where the oracle cannot
evaluate every output: the places where an FFT operator goes wrong first
(the body's extreme voxels along each axis, the body voxels nearest the grid's
eight corners, where zero padding and cropping act, and surface voxels, where
the contrast jumps), topped up with random body voxels."""
import numpy as np


def pick_voxels(mask, count=32, seed=0):
    """Return (T, 3) distinct voxel indices inside ``mask`` (a boolean grid),
    T = ``count`` (or all body voxels if there are fewer)."""
    mask = np.asarray(mask, bool)
    n = np.array(mask.shape)
    body = np.argwhere(mask)
    if len(body) <= count:
        return body
    chosen = []

    def add(i):
        i = int(i)
        if i not in chosen:
            chosen.append(i)

    for a in range(3):  # extremes along each axis
        add(np.argmin(body[:, a]))
        add(np.argmax(body[:, a]))
    for corner in np.stack(np.meshgrid([0, 1], [0, 1], [0, 1], indexing="ij"), -1).reshape(-1, 3):
        c = corner * (n - 1)
        add(np.argmin(np.sum((body - c) ** 2, axis=1)))
    # surface: a 6-neighbour outside the body or outside the grid
    pad = np.pad(mask, 1, constant_values=False)
    inner = np.ones_like(mask)
    for a in range(3):
        for s in (-1, 1):
            inner &= np.roll(pad, s, axis=a)[1:-1, 1:-1, 1:-1]
    surf = np.flatnonzero(~inner[tuple(body.T)])
    rng = np.random.default_rng(seed)
    for i in rng.permutation(surf)[:max(0, count // 3)]:
        add(i)
    for i in rng.permutation(len(body)):
        if len(chosen) >= count:
            break
        add(i)
    return body[np.array(chosen[:count])]
