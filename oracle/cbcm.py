"""Plain CPU oracle of the block-structured cube layout (test infrastructure
only; Sec 2.2, the grid generation of the cube-based Cartesian mesh).

The domain is first divided into equal cubes of `cube` cells at spacing H.
Cubes near the terrain are split into eight, level after level, up to the
finest level; cube sizes are then adjusted so that neighbouring cubes, across
faces, edges and corners, differ by at most one level (2:1); cubes lying
completely inside the terrain are dropped.

Reading of the refinement test (the paper only says that cubes close to the
terrain surface are split; the reading is fitted to its cube counts): a cube
of level l below the finest level is split when (i) its bottom lies below the highest terrain point and (ii) the
horizontal distance between its footprint and the columns where the terrain
is raised above its lowest value is at most one cube width. Lateral
boundaries are periodic. Only tests import this module.
"""
from __future__ import annotations

import math

import numpy as np


def cube_layout(nx0: int, ny0: int, nz0: int, cube: int, H: float, nlev: int, h_finest: np.ndarray):
    """Leaf cubes (level, ci, cj, ck), ci.. in cube units of their level,
    sorted by (level, ck, cj, ci). h_finest: corner heights of the finest
    level, shape (ny0 2^(nlev-1), nx0 2^(nlev-1)), periodic."""
    assert nx0 % cube == 0 and ny0 % cube == 0 and nz0 % cube == 0 and nlev >= 1
    L = nlev - 1
    hf = np.asarray(h_finest, dtype=np.float64)
    assert hf.shape == (ny0 << L, nx0 << L)
    Lx, Ly = nx0 * H, ny0 * H
    df = H / (1 << L)  # finest spacing
    hmin, hmax = float(hf.min()), float(hf.max())
    jr, ir = np.nonzero(hf > hmin)
    rx, ry = ir * df, jr * df  # raised corner points
    ncx = [(nx0 // cube) << l for l in range(nlev)]
    ncy = [(ny0 // cube) << l for l in range(nlev)]
    ncz = [(nz0 // cube) << l for l in range(nlev)]
    size = [cube * H / (1 << l) for l in range(nlev)]
    refined = [set() for _ in range(nlev)]

    def exists(l, c):
        return l == 0 or (c[0] // 2, c[1] // 2, c[2] // 2) in refined[l - 1]

    def axis_gap(p, a0, a1, period):
        # distance from coordinates p to the interval [a0, a1] on a circle
        best = None
        for sh in (-period, 0.0, period):
            q = p + sh
            g = np.maximum(0.0, np.maximum(a0 - q, q - a1))
            best = g if best is None else np.minimum(best, g)
        return best

    def near_terrain(l, c):
        s = size[l]
        if not (c[2] * s < hmax) or rx.size == 0:
            return False
        gx = axis_gap(rx, c[0] * s, (c[0] + 1) * s, Lx)
        gy = axis_gap(ry, c[1] * s, (c[1] + 1) * s, Ly)
        return bool(np.min(np.sqrt(gx * gx + gy * gy)) <= s)

    # refinement by the terrain test, level by level
    for l in range(L):
        for ck in range(ncz[l]):
            for cj in range(ncy[l]):
                for ci in range(ncx[l]):
                    c = (ci, cj, ck)
                    if exists(l, c) and near_terrain(l, c):
                        refined[l].add(c)

    def leaf_level(l, c):
        """Level of the leaf covering the region of cube c of level l."""
        # the centre of the region in finest cube units
        f = 1 << (L - l)
        p = ((2 * c[0] + 1) * f, (2 * c[1] + 1) * f, (2 * c[2] + 1) * f)  # twice the finest index
        for m in range(nlev):
            g = 1 << (L - m + 1)
            cm = (p[0] // g, p[1] // g, p[2] // g)
            if cm not in refined[m]:
                return m, cm
        raise AssertionError("refined at the finest level")

    # 2:1 balance across faces, edges and corners (periodic in x and y)
    changed = True
    while changed:
        changed = False
        for l in range(L, 1, -1):
            for c in sorted(refined[l - 1]):
                for a in range(2):
                    for b in range(2):
                        for e in range(2):
                            leaf = (2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e)
                            if leaf in refined[l]:
                                continue
                            for dk in (-1, 0, 1):
                                for dj in (-1, 0, 1):
                                    for di in (-1, 0, 1):
                                        if di == dj == dk == 0:
                                            continue
                                        nk = leaf[2] + dk
                                        if nk < 0 or nk >= ncz[l]:
                                            continue
                                        nb = ((leaf[0] + di) % ncx[l], (leaf[1] + dj) % ncy[l], nk)
                                        m, cm = leaf_level(l, nb)
                                        if m < l - 1:
                                            refined[m].add(cm)
                                            changed = True
    # leaves, minus the cubes completely inside the terrain
    out = []
    for l in range(nlev):
        s, f = size[l], cube << (L - l)  # cube width in finest cells
        for ck in range(ncz[l]):
            for cj in range(ncy[l]):
                for ci in range(ncx[l]):
                    c = (ci, cj, ck)
                    if not exists(l, c) or c in refined[l]:
                        continue
                    I = np.arange(ci * f, (ci + 1) * f + 1) % hf.shape[1]
                    J = np.arange(cj * f, (cj + 1) * f + 1) % hf.shape[0]
                    if hf[np.ix_(J, I)].min() >= (ck + 1) * s:
                        continue
                    out.append((l, ci, cj, ck))
    return out
