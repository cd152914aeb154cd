"""Seeded synthetic workloads: terrain corner heights and run configurations.

This module only builds inputs (hill shapes sampled at grid corners, grid
sizes, flow parameters).  It holds none of the cut-cell method's arithmetic,
so both the CUDA path and the CPU oracle take their inputs from here.

The hill shapes follow the experiments of the paper: the bell-shaped hill of
Sec 3.1.1, the hemisphere of Sec 3.1.2 (a half-ellipsoid when its height
differs from its radius) and the cosine hill of the appendix.  Every hill is
centred on a grid corner at the middle of the domain; this centring gives the
18.1 deg and 71 deg resolved slopes quoted in Sec 3.1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G = 9.81
R_DRY = 287.0
CP = 1004.5
P0 = 1.0e5


def theta_surface(T_s: float = 288.0, p_s: float = 1.0e5) -> float:
    """Potential temperature of surface air at temperature T_s and pressure p_s."""
    return T_s * (P0 / p_s) ** (R_DRY / CP)


def corner_heights(kind: str, nx: int, ny: int, dx: float, dy: float, h0: float, a: float,
                   xc: float | None = None, yc: float | None = None) -> np.ndarray:
    """Terrain height at the grid corners (I*dx, J*dy), I < nx, J < ny (periodic).

    Returns an (ny, nx) float64 array, x fastest.
    """
    if xc is None:
        xc = 0.5 * nx * dx
    if yc is None:
        yc = 0.5 * ny * dy
    x = np.arange(nx, dtype=np.float64) * dx - xc
    y = np.arange(ny, dtype=np.float64) * dy - yc
    X, Y = np.meshgrid(x, y)
    r2 = X * X + Y * Y
    if kind == "bell":
        h = h0 / (1.0 + r2 / (a * a)) ** 1.5
    elif kind in ("hemisphere", "ellipsoid"):
        h = h0 * np.sqrt(np.maximum(0.0, 1.0 - r2 / (a * a)))
    elif kind == "cosine":
        r = np.sqrt(r2)
        h = np.where(r < a, 0.5 * h0 * (1.0 + np.cos(np.pi * r / a)), 0.0)
    elif kind == "flat":
        h = np.zeros_like(r2)
    else:
        raise ValueError(f"unknown terrain kind {kind!r}")
    return np.ascontiguousarray(h, dtype=np.float64)


def planar_heights(nx: int, ny: int, dx: float, dy: float, m1: float, m3: float, c: float) -> np.ndarray:
    """Corner heights of the plane h = c + m1 x + m3 y (not periodic; for geometry pins)."""
    x = np.arange(nx, dtype=np.float64) * dx
    y = np.arange(ny, dtype=np.float64) * dy
    X, Y = np.meshgrid(x, y)
    return np.ascontiguousarray(c + m1 * X + m3 * Y)


@dataclasses.dataclass
class RunConfig:
    """One single-level periodic domain (a uniform block) and its flow."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    dt: float
    steps: int
    terrain: str
    h0: float
    a: float
    U: float = 10.0
    N: float = 0.01
    theta0: float = dataclasses.field(default_factory=theta_surface)
    p_surf: float = 1.0e5
    p0: float = P0
    g: float = G
    R: float = R_DRY
    cp: float = CP
    ra_nu: float = 0.1
    c4: float = 0.005
    sponge_frac: float = 0.375
    tau_max: float = 0.01
    bc_slip: int = 1

    def heights(self) -> np.ndarray:
        return corner_heights(self.terrain, self.nx, self.ny, self.dx, self.dy, self.h0, self.a)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "RunConfig":
        return dataclasses.replace(self, **kw)


# Bell hill, one uniform 32x32x24 block of 200 m cells (top 4.8 km).
C1_BELL = RunConfig("bell-32x32x24-200m", 32, 32, 24, 200.0, 200.0, 200.0, 0.15, 100,
                    "bell", 100.0, 1000.0)
# Hemisphere of radius 1 km on a uniform 128x128x64 grid of 50 m cells.
C2_HEMI = RunConfig("hemisphere-128x128x64-50m", 128, 128, 64, 50.0, 50.0, 50.0, 0.0375, 2000,
                    "hemisphere", 1000.0, 1000.0)
# Bell hill 400 m / 2 km on 512x512x128, dx = dy = 100 m, dz = 50 m.
C3_BELL = RunConfig("bell-512x512x128-100m", 512, 512, 128, 100.0, 100.0, 50.0, 0.05, 5000,
                    "bell", 400.0, 2000.0)
# Small steep case for parity tests: hemisphere of radius 400 m on 50 m cells,
# large enough for vertical and horizontal merges and several tiles.
SMALL_HEMI = RunConfig("hemisphere-40x36x24-50m", 40, 36, 24, 50.0, 50.0, 50.0, 0.0375, 20,
                       "hemisphere", 400.0, 400.0)

PRESETS = {c.name: c for c in (C1_BELL, C2_HEMI, C3_BELL, SMALL_HEMI)}


def ensemble_configs(n: int = 64, seed: int = 1509) -> list[RunConfig]:
    """Seeded ensemble of independent single-level runs of uneven sizes.

    nx = ny drawn from {64, 96, 128, 160, 192}, nz = max(64, nx/2), isotropic
    spacing 8a/nx, hill type bell or hemisphere (half-ellipsoid), h0 in
    [100, 1000] m, a in [500, 3000] m, U in [5, 20] m/s, N in [0.005, 0.02] 1/s.
    """
    rng = np.random.default_rng(seed)
    out = []
    for e in range(n):
        nx = int(rng.choice([64, 96, 128, 160, 192]))
        nz = max(64, nx // 2)
        kind = "bell" if rng.integers(0, 2) == 0 else "ellipsoid"
        h0 = float(rng.uniform(100.0, 1000.0))
        a = float(rng.uniform(500.0, 3000.0))
        U = float(rng.uniform(5.0, 20.0))
        N = float(rng.uniform(0.005, 0.02))
        d = 8.0 * a / nx
        # the domain top must stay well above the hill
        top = nz * d
        if h0 > 0.5 * top:
            h0 = 0.5 * top
        dt = 0.15 * d / 200.0
        out.append(RunConfig(f"ens{e}-{kind}-{nx}x{nx}x{nz}", nx, nx, nz, d, d, d, dt, 500,
                             kind, h0, a, U=U, N=N))
    return out


@dataclasses.dataclass
class RefinedConfig:
    """Block-structured refinement: level 0 is `base` (the periodic domain);
    level l >= 1 is a box (nx, ny, nz, ox, oy) of cells of spacing 2^-l of the
    base spacing starting at the floor, whose cell i covers cell (i + ox) // 2
    of level l-1.  The hill (terrain, h0, a of `base`) lies in the finest
    level, centred on the domain centre; coarser levels see a flat floor."""
    name: str
    base: RunConfig
    boxes: list
    # cuts of the finest level's box into sibling blocks (its cells)
    xcuts: tuple = ()
    ycuts: tuple = ()

    @property
    def nlev(self) -> int:
        return 1 + len(self.boxes)

    def level_origin(self, l: int) -> tuple:
        """Absolute (x, y) of the low corner of level l's cell (0, 0)."""
        x = y = 0.0
        for m in range(1, l + 1):
            nx, ny, nz, ox, oy = self.boxes[m - 1]
            d = self.base.dx * 2.0 ** -m
            x += ox * d
            y += oy * d
        return x, y

    def finest_heights(self, pad: int = 0) -> np.ndarray:
        """Corner heights of the finest level for I, J = -pad .. n+pad-1
        (interior corners when pad = 0; the padded set has n + 2 pad + 1 per
        row when pad > 0, i.e. I, J = -pad .. n+pad)."""
        l = self.nlev - 1
        b = self.base
        f = 2.0 ** -l
        dx, dy = b.dx * f, b.dy * f
        if l == 0:
            return corner_heights(b.terrain, b.nx, b.ny, dx, dy, b.h0, b.a)
        nx, ny = self.boxes[l - 1][0], self.boxes[l - 1][1]
        x0, y0 = self.level_origin(l)
        xc, yc = 0.5 * b.nx * b.dx, 0.5 * b.ny * b.dy
        n_x = nx + 2 * pad + (1 if pad else 0)
        n_y = ny + 2 * pad + (1 if pad else 0)
        return corner_heights(b.terrain, n_x, n_y, dx, dy, b.h0, b.a,
                              xc=xc - (x0 - pad * dx), yc=yc - (y0 - pad * dy))

    def cells(self) -> int:
        n = self.base.cells
        for bx in self.boxes:
            n += bx[0] * bx[1] * bx[2]
        return n

    def active_cells(self) -> int:
        n = self.cells()
        for bx in self.boxes:
            n -= (bx[0] // 2) * (bx[1] // 2) * (bx[2] // 2)
        return n


# Three levels around a hemisphere of radius 600 m: 400 m / 200 m / 100 m,
# 32 x 32 x 16 cells per level (oracle-sized).
SMALL_REFINED = RefinedConfig(
    "refined-3x32x32x16-hemisphere",
    RunConfig("refined-base", 32, 32, 16, 400.0, 400.0, 400.0, 0.3, 20, "hemisphere", 600.0, 600.0),
    [(32, 32, 16, 16, 16), (32, 32, 16, 16, 16)])

# Three levels around a hemisphere of radius 500 m, 400 m / 200 m / 100 m,
# the finest 64 x 64 x 16 box cut into six sibling blocks of uneven sizes
# (x cuts 18 and 46, y cut 46; the hill, corners 28 .. 36, stays 8 corners
# clear of every cut) (oracle-sized).
SMALL_BLOCKED = RefinedConfig(
    "refined-blocks-48x48x16-hemisphere",
    RunConfig("blocked-base", 48, 48, 16, 400.0, 400.0, 400.0, 0.3, 20, "hemisphere", 500.0, 500.0),
    [(64, 64, 16, 16, 16), (64, 64, 16, 32, 32)], xcuts=(18, 46), ycuts=(46,))

# Hemisphere of radius 1 km with three levels: 200 m over the 64 x 32 x 16 km
# domain, 100 m over x in [6.4, 57.6] km, y in [1.6, 30.4] km, z < 8 km, and
# 50 m over x in [12.8, 51.2] km, y in [4.8, 27.2] km, z < 4.8 km.
C4_REFINED = RefinedConfig(
    "refined-hemisphere-200-100-50m",
    RunConfig("refined-base-320x160x80-200m", 320, 160, 80, 200.0, 200.0, 200.0, 0.15, 200,
              "hemisphere", 1000.0, 1000.0),
    [(512, 288, 80, 64, 16), (768, 448, 96, 128, 64)])

# The same three levels with the 50 m level cut into 15 sibling blocks of
# uneven sizes (x cuts 96, 250, 480, 640; y cuts 120, 300 of its 768 x 448
# cells); the hemisphere, corners 364 .. 404 in x and 204 .. 244 in y, lies in
# one block, at least 56 cells clear of every cut.
C4_BLOCKED = RefinedConfig(
    "refined-hemisphere-200-100-50m-15-blocks",
    C4_REFINED.base, C4_REFINED.boxes, xcuts=(96, 250, 480, 640), ycuts=(120, 300))
