"""Pins of the cube-layout oracle (Sec 2.2 grid generation): the cube counts
the paper reports for its refined hemisphere grids, the 2:1 balance across
faces, edges and corners, the removal of cubes inside the terrain, and
brute-force coverage of the domain."""
import itertools

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

from oracle import cbcm


def paper_hemisphere(nlev):
    """The paper's refined-grid test: 64 x 32 x 16 km, cubes of 20^3 cells,
    H = 400 m, the 1 km hemisphere at the centre; finest spacing 400/2^(nlev-1)."""
    d = 400.0 / (1 << (nlev - 1))
    h = W.corner_heights("hemisphere", int(64000 / d), int(32000 / d), d, d, 1000.0, 1000.0)
    return cbcm.cube_layout(160, 80, 40, 20, 400.0, nlev, h)


def test_paper_cube_counts():
    """64, 148 and 232 cubes for refinement levels 0, 1 and 2, and 4096 for
    the uniform 100 m grid (the paper's counts for its four grids)."""
    assert len(paper_hemisphere(1)) == 64
    assert len(paper_hemisphere(2)) == 148
    assert len(paper_hemisphere(3)) == 232
    d = 100.0
    hflat = np.zeros((320, 640))
    assert len(cbcm.cube_layout(640, 320, 160, 20, d, 1, hflat)) == 4096


def _volume_and_balance(cubes, ncx0, ncy0, ncz0, nlev):
    L = nlev - 1
    f = {l: 1 << (L - l) for l in range(nlev)}
    grid = -np.ones((ncz0 << L, ncy0 << L, ncx0 << L), np.int8)
    for l, ci, cj, ck in cubes:
        s = f[l]
        sub = grid[ck * s:(ck + 1) * s, cj * s:(cj + 1) * s, ci * s:(ci + 1) * s]
        assert (sub == -1).all(), "cubes overlap"
        sub[...] = l
    return grid


def test_layout_tiles_the_domain_and_is_balanced():
    """Brute force on the finest cube grid: the leaves cover the domain once
    (nothing is underground here), and any two touching finest positions
    (face, edge or corner, periodic laterally) lie in cubes whose levels
    differ by at most one."""
    nlev = 3
    cubes = paper_hemisphere(nlev)
    g = _volume_and_balance(cubes, 8, 4, 2, nlev)
    assert (g >= 0).all()
    for dk, dj, di in itertools.product((-1, 0, 1), repeat=3):
        if dk == dj == di == 0:
            continue
        sh = np.roll(np.roll(g, -dj, axis=1), -di, axis=2)
        if dk == 1:
            a, b = g[:-1], sh[1:]
        elif dk == -1:
            a, b = g[1:], sh[:-1]
        else:
            a, b = g, sh
        assert np.abs(a.astype(int) - b.astype(int)).max() <= 1


def test_balance_closure_refines_a_neighbour():
    """A narrow ridge that asks for level 3 next to level-1 cubes: the
    balance pass splits the level-1 neighbours, so no level-3 cube touches a
    level-1 cube."""
    nlev = 4
    nf = 8 * 8 * (1 << (nlev - 1))
    h = np.zeros((nf // 2, nf))
    h[:, nf // 2] = 50.0  # a one-column wall along y through the middle
    cubes = cbcm.cube_layout(64, 32, 16, 8, 100.0, nlev, h)
    g = _volume_and_balance(cubes, 8, 4, 2, nlev)
    assert g.max() == 3
    for di in (-1, 1):
        assert np.abs(g.astype(int) - np.roll(g, di, axis=2).astype(int)).max() <= 1


def test_cubes_inside_the_terrain_are_dropped():
    """A plateau higher than the bottom cube layer of level 0 everywhere:
    those cubes are dropped and the rest of the domain stays covered."""
    nlev = 2
    h = np.full((2 * 32, 2 * 64), 900.0)
    h[10, 10] = 950.0  # raised somewhere, so some cubes are refined
    cubes = cbcm.cube_layout(64, 32, 32, 8, 100.0, nlev, h)
    g = _volume_and_balance(cubes, 8, 4, 4, nlev)
    # the level-0 bottom layer (0 .. 800 m) lies under the 900 m plateau
    assert (g[:2] == -1).all() and (g[2:] >= 0).all()
