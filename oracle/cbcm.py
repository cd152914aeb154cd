"""Plain CPU oracle of the block-structured cube layout (test infrastructure
only; Sec 2.2, the grid generation of the cube-based Cartesian mesh).

The domain is first divided into equal cubes of `cube` cells at spacing H.
Cubes near the terrain are split into eight, level after level, up to the
finest level; cube sizes are then adjusted so that neighbouring cubes, across
faces, edges and corners, differ by at most one level (2:1); cubes lying
completely inside the terrain are dropped.

Reading of the refinement test (the paper only says that cubes close to the
terrain surface are split; the reading is fitted to its cube counts): a cube
of level l below the finest level is split when (i) its bottom lies below the
highest terrain point and (ii) the horizontal distance between its footprint
and the finest-level corners where the terrain is raised above its lowest
value is at most one cube width.  Lateral boundaries are periodic.

Brute force over the finest cube grid: an array holds, for every position of
a finest-level cube, the level of the leaf cube that covers it.  Splitting a
cube raises the level of all its positions by one.  The 2:1 balance is the
plain definition iterated to its fixed point: wherever two touching positions
differ by more than one level, the cube of the coarser one is split; the
least balanced refinement containing the terrain refinement is unique, so the
order of the splits does not matter.  Only tests import this module.
"""
from __future__ import annotations

import itertools

import numpy as np


def _near_terrain(c0, c1, size, hmax, raised, Lx, Ly):
    """Refinement test of a cube with horizontal footprint [c0, c1] (metres,
    x and y) whose bottom is at c0[2]: bottom below the highest terrain and a
    raised corner within one cube width of the footprint (periodic)."""
    if not c0[2] < hmax or len(raised) == 0:
        return False
    best = np.inf
    for px, py in raised:
        dx = min(max(0.0, c0[0] - x, x - c1[0]) for x in (px - Lx, px, px + Lx))
        dy = min(max(0.0, c0[1] - y, y - c1[1]) for y in (py - Ly, py, py + Ly))
        best = min(best, (dx * dx + dy * dy) ** 0.5)
        if best <= size:
            return True
    return False


def cube_layout(nx0: int, ny0: int, nz0: int, cube: int, H: float, nlev: int, h_finest: np.ndarray):
    """Leaf cubes (level, ci, cj, ck), ci.. in cube units of their level,
    sorted by (level, ck, cj, ci). h_finest: corner heights of the finest
    level, shape (ny0 2^(nlev-1), nx0 2^(nlev-1)), periodic."""
    assert nx0 % cube == 0 and ny0 % cube == 0 and nz0 % cube == 0 and nlev >= 1
    L = nlev - 1
    hf = np.asarray(h_finest, dtype=np.float64)
    assert hf.shape == (ny0 << L, nx0 << L)
    df = H / (1 << L)
    Lx, Ly = nx0 * H, ny0 * H
    hmin, hmax = float(hf.min()), float(hf.max())
    raised = [(I * df, J * df) for J, I in zip(*np.nonzero(hf > hmin))]
    nf = ((nz0 // cube) << L, (ny0 // cube) << L, (nx0 // cube) << L)  # finest cube grid (k, j, i)
    lev = np.zeros(nf, dtype=np.int64)

    def width(l):  # finest positions along one edge of a level-l cube
        return 1 << (L - l)

    # terrain refinement, level by level, of every level-l leaf
    for l in range(L):
        f = width(l)
        s = cube * H / (1 << l)
        for ck, cj, ci in itertools.product(range(nf[0] // f), range(nf[1] // f), range(nf[2] // f)):
            blk = lev[ck * f:(ck + 1) * f, cj * f:(cj + 1) * f, ci * f:(ci + 1) * f]
            if (blk == l).all() and _near_terrain((ci * s, cj * s, ck * s), ((ci + 1) * s, (cj + 1) * s), s, hmax,
                                                  raised, Lx, Ly):
                blk[...] = l + 1

    # 2:1 balance across faces, edges and corners (periodic in x and y)
    while True:
        coarse = np.zeros(nf, dtype=bool)
        for dk, dj, di in itertools.product((-1, 0, 1), repeat=3):
            if dk == dj == di == 0:
                continue
            nb = np.roll(np.roll(lev, -dj, axis=1), -di, axis=2)
            if dk:
                nb = np.roll(nb, -dk, axis=0)
                edge = nf[0] - 1 if dk == 1 else 0  # no neighbour across the floor or the top
                nb[edge] = -1
            coarse |= nb > lev + 1
        if not coarse.any():
            break
        for k, j, i in zip(*np.nonzero(coarse)):
            b = lev[k, j, i]
            if b >= L:
                continue
            f = width(b)
            ck, cj, ci = k // f, j // f, i // f
            lev[ck * f:(ck + 1) * f, cj * f:(cj + 1) * f, ci * f:(ci + 1) * f] = b + 1

    # leaves (every level-l cube whose positions all carry level l), minus the
    # cubes completely inside the terrain
    out = []
    for l in range(nlev):
        f = width(l)
        s = cube * H / (1 << l)
        w = cube << (L - l)  # cube width in finest cells
        for ck, cj, ci in itertools.product(range(nf[0] // f), range(nf[1] // f), range(nf[2] // f)):
            blk = lev[ck * f:(ck + 1) * f, cj * f:(cj + 1) * f, ci * f:(ci + 1) * f]
            if not (blk == l).all():
                assert not (blk == l).any(), "a leaf must be a whole cube"
                continue
            I = np.arange(ci * w, (ci + 1) * w + 1) % hf.shape[1]
            J = np.arange(cj * w, (cj + 1) * w + 1) % hf.shape[0]
            if hf[np.ix_(J, I)].min() >= (ck + 1) * s:
                continue
            out.append((l, ci, cj, ck))
    return out
