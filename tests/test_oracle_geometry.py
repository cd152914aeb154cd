"""Pins of the oracle's cut-cell geometry (paper Sec 2.3) against closed forms,
independent computations and the values the paper prints."""
import math
import os

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
def test_gauss_legendre8_exact_to_degree_15(oracle_mod):
    # an 8-point Gauss-Legendre rule integrates every polynomial of degree <= 15 exactly
    for d in range(16):
        got = oracle_mod.gauss_legendre8(lambda s, d=d: s ** d, -1.0, 1.0)
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(got - exact) < 4e-16, (d, got, exact)
    got = oracle_mod.gauss_legendre8(lambda s: s ** 16, -1.0, 1.0)
    assert abs(got - 2.0 / 17) > 1e-6  # not exact beyond degree 15


# ---------------------------------------------------------------- line integrals
def _brute_line(z, ha, hb, length, n=200000):
    s = (np.arange(n) + 0.5) / n
    h = ha + (hb - ha) * s
    return np.maximum(z - h, 0.0).mean() * length, (h < z).mean()


@pytest.mark.parametrize("z,ha,hb", [(5.0, 0.0, 10.0), (12.0, 0.0, 10.0), (-1.0, 0.0, 10.0),
                                      (3.0, 7.0, 1.0), (4.0, 4.0, 4.0), (4.0, 2.0, 2.0)])
def test_line_integral_and_fraction(oracle_mod, z, ha, hb):
    li = oracle_mod.line_int(z, ha, hb, 3.0)
    lf = oracle_mod.line_frac(z, ha, hb)
    bi, bf = _brute_line(z, ha, hb, 3.0)
    assert abs(li - bi) < 1e-8
    assert abs(lf - bf) < 1e-5


def test_flat_terrain_at_face_level_closes_face(oracle_mod):
    # terrain exactly at a horizontal face: no fluid below it, aperture 0
    assert oracle_mod.line_frac(4.0, 4.0, 4.0) == 0.0
    assert oracle_mod.col_int(4.0, 4.0, 4.0, 4.0, 4.0, 1.0, 1.0, 1) == 0.0


# ---------------------------------------------------------------- planar terrain
def _clip_area(m1, m3, c, z, dx, dy):
    """Area of {(x,y) in [0,dx]x[0,dy] : c + m1 x + m3 y < z} by Sutherland-Hodgman
    clipping of the rectangle against the half-plane, then the shoelace formula."""
    poly = [(0.0, 0.0), (dx, 0.0), (dx, dy), (0.0, dy)]
    f = lambda p: z - (c + m1 * p[0] + m3 * p[1])  # inside where f > 0
    out = []
    for a, b in zip(poly, poly[1:] + poly[:1]):
        fa, fb = f(a), f(b)
        if fa > 0:
            out.append(a)
        if (fa > 0) != (fb > 0):
            t = fa / (fa - fb)
            out.append((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
    if len(out) < 3:
        return 0.0
    s = 0.0
    for a, b in zip(out, out[1:] + out[:1]):
        s += a[0] * b[1] - b[0] * a[1]
    return abs(s) * 0.5


def _simpson_piecewise(F, z0, z1, breaks):
    """Integral of F over [z0,z1], exact when F is a polynomial of degree <= 3
    between breakpoints (two-point Gauss rule per piece; never samples a
    breakpoint, where F may jump)."""
    pts = sorted({z0, z1, *[b for b in breaks if z0 < b < z1]})
    s = 0.0
    g = 1.0 / math.sqrt(3.0)
    for a, b in zip(pts, pts[1:]):
        m, r = 0.5 * (a + b), 0.5 * (b - a)
        s += r * (F(m - r * g) + F(m + r * g))
    return s


def _planar_cell_exact(m1, m3, c, dx, dy, z0, z1):
    hs = [c, c + m1 * dx, c + m3 * dy, c + m1 * dx + m3 * dy]
    vol = _simpson_piecewise(lambda z: _clip_area(m1, m3, c, z, dx, dy), z0, z1, hs)
    return vol


def _planar_face_exact(ha, hb, length, z0, z1):
    frac = lambda z: 0.0 if ha == hb and z <= ha else (
        1.0 if z >= max(ha, hb) else (0.0 if z <= min(ha, hb) else (z - min(ha, hb)) / abs(hb - ha)))
    return _simpson_piecewise(lambda z: frac(z) * length, z0, z1, [ha, hb])


def _planar_cases():
    rng = np.random.default_rng(2572)
    cases = [(0.3, -0.2, 37.0), (1.0, 0.0, 10.0), (0.0, 0.0, 25.0),  # slope exactly 1, flat
             (0.5, 0.5, 0.0),  # plane through the low corner
             (2.5, -0.7, 60.0), (-3.0, 1.0, 300.0)]
    for _ in range(12):
        cases.append((float(rng.uniform(-3, 3)), float(rng.uniform(-3, 3)), float(rng.uniform(-50, 250))))
    return cases


@pytest.mark.parametrize("m1,m3,c", _planar_cases())
def test_planar_terrain_volumes_and_apertures_exact(oracle_mod, m1, m3, c):
    """For planar terrain the oracle's volumes and apertures equal the closed
    form (polygon clipping integrated exactly in z) to round-off."""
    nx, ny, nz, dx, dy, dz = 4, 4, 6, 50.0, 40.0, 30.0
    h = W.planar_heights(nx + 1, ny + 1, dx, dy, m1, m3, c)
    # evaluate a single interior column directly through the column integrals
    for (i, j) in [(1, 1), (2, 1)]:
        h00, h10, h01, h11 = h[j, i], h[j, i + 1], h[j + 1, i], h[j + 1, i + 1]
        cc = h00  # plane in column-local coordinates
        for k in range(nz):
            z0, z1 = k * dz, (k + 1) * dz
            w1 = oracle_mod.col_int(z1, h00, h10, h01, h11, dx, dy, 0)
            w0 = oracle_mod.col_int(z0, h00, h10, h01, h11, dx, dy, 0)
            exact = _planar_cell_exact(m1, m3, cc, dx, dy, z0, z1)
            assert abs((w1 - w0) - exact) <= 1e-12 * dx * dy * dz, (k, w1 - w0, exact)
            # horizontal face aperture at z0
            a = oracle_mod.col_int(z0, h00, h10, h01, h11, dx, dy, 1)
            assert abs(a - _clip_area(m1, m3, cc, z0, dx, dy)) <= 1e-12 * dx * dy
            # vertical faces (x = const and y = const) through the line integral
            L = oracle_mod.line_int(z1, h00, h01, dy) - oracle_mod.line_int(z0, h00, h01, dy)
            assert abs(L - _planar_face_exact(h00, h01, dy, z0, z1)) <= 1e-12 * dy * dz


def test_planar_terrain_through_the_model(oracle_mod):
    """The same closed form through the full geometry build (periodic-safe plane
    inside one cell layer: a tilted plane that never crosses the lateral edges)."""
    # a periodic "plane" is impossible; use a plateau made of one tilted cell
    nx = ny = 8
    h = np.full((ny, nx), 10.0)
    cfg = W.RunConfig("t", nx, ny, 6, 50.0, 50.0, 40.0, 0.1, 1, "flat", 0.0, 1.0, U=0.0)
    m = oracle_mod.Model(cfg, h)
    g = m.geometry()
    # flat terrain at 10 m: bottom layer volume fraction (40-10)/40, lateral apertures 0.75
    assert np.allclose(g["vf"][0], 0.75, rtol=0, atol=1e-15)
    assert np.allclose(g["ax"][0], 0.75, rtol=0, atol=1e-15)
    assert np.allclose(g["ay"][0], 0.75, rtol=0, atol=1e-15)
    assert np.all(g["vf"][1:] == 1.0)
    assert np.all(g["az"][0] == 0.0) and np.all(g["az"][-1] == 0.0)  # floor and lid
    assert np.all(g["az"][1:-1] == 1.0)


# ---------------------------------------------------------------- bilinear terrain
def _subcolumn_volume(h00, h10, h01, h11, dx, dy, z0, z1, n):
    """The paper's sub-column approximation (narrow rectangular columns, Sec 2.3),
    midpoint heights of n x n sub-columns."""
    s = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(s, s, indexing="ij")
    hh = h00 + (h10 - h00) * X + (h01 - h00) * Y + (h00 - h01 + h11 - h10) * X * Y
    return (np.clip(z1 - np.maximum(hh, z0), 0.0, z1 - z0)).mean() * dx * dy


@pytest.mark.parametrize("hs", [(10.0, 80.0, 35.0, 5.0), (0.0, 120.0, 120.0, 0.0), (55.0, 20.0, 90.0, 140.0)])
def test_bilinear_volume_matches_subcolumn_limit(oracle_mod, hs):
    """Exact integration of the bilinear cut cell agrees with the paper's
    sub-column sum in the limit of many sub-columns (Richardson extrapolated)."""
    dx, dy, dz = 50.0, 50.0, 50.0
    for k in range(3):
        z0, z1 = k * dz, (k + 1) * dz
        v = oracle_mod.col_int(z1, *hs, dx, dy, 0) - oracle_mod.col_int(z0, *hs, dx, dy, 0)
        a = _subcolumn_volume(*hs, dx, dy, z0, z1, 1024)
        b = _subcolumn_volume(*hs, dx, dy, z0, z1, 2048)
        rich = (4.0 * b - a) / 3.0
        assert abs(v - rich) <= 2e-7 * dx * dy * dz, (k, v, rich)


def test_column_volume_sum_closed_form(oracle_mod):
    """Sum of cell volumes of a column = footprint * (top - mean height): the
    integral of a bilinear surface over its column is the mean of its corners."""
    cfg = W.SMALL_HEMI
    m = oracle_mod.Model(cfg)
    g = m.geometry()
    V0 = cfg.dx * cfg.dy * cfg.dz
    colsum = (g["vf"] * V0).sum(axis=0)
    exact = cfg.dx * cfg.dy * (cfg.nz * cfg.dz - g["hc"])
    assert np.max(np.abs(colsum - exact)) <= 1e-9 * V0


def test_vertical_face_apertures_bracket(oracle_mod):
    cfg = W.SMALL_HEMI
    g = oracle_mod.Model(cfg).geometry()
    for k in ("vf", "ax", "ay", "az"):
        assert g[k].min() >= -1e-15 and g[k].max() <= 1.0 + 1e-15


# ---------------------------------------------------------------- paper pins
def _golden_slopes():
    rows = []
    with open(os.path.join(GOLDEN, "resolved_slopes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, h0, a, dx, deg, tol, ndir = line.split()
                rows.append((kind, float(h0), float(a), float(dx), float(deg), float(tol), int(ndir)))
    return rows


def _merge_dirs(g):
    dirs = set()
    cls = g["cls"]
    for k, j, i in zip(*np.nonzero(cls == 3)):
        gx, gy = g["gx"][j, i], g["gy"][j, i]
        if abs(gx) <= 1 and abs(gy) <= 1:
            dirs.add("z")
        elif abs(gx) >= abs(gy):
            dirs.add("+x" if gx < 0 else "-x")
        else:
            dirs.add("+y" if gy < 0 else "-y")
    return dirs


@pytest.mark.parametrize("row", _golden_slopes(), ids=lambda r: r[0])
def test_paper_resolved_slope_and_merge_directions(oracle_mod, row):
    kind, h0, a, dx, deg, tol, ndir = row
    # paper domain 64 x 32 km, hill centred; 16 levels of 200 m reach 3.2 km,
    # enough above both hills for the geometry (the slope depends on h only)
    nx, ny, nz = int(64000 / dx), int(32000 / dx), 16
    cfg = W.RunConfig("paper", nx, ny, nz, dx, dx, dx, 0.1, 1, kind, h0, a, theta0=300.0)
    g = oracle_mod.Model(cfg).geometry()
    gmax = max(np.abs(g["gx"]).max(), np.abs(g["gy"]).max())
    assert abs(math.degrees(math.atan(gmax)) - deg) <= tol
    dirs = _merge_dirs(g)
    assert len(dirs) == ndir, dirs
    if ndir == 1:
        assert gmax < 1.0 and dirs == {"z"}


def test_merged_volumes_exceed_half(oracle_mod):
    """After merging every computational volume exceeds half a regular cell (Sec 2.3)."""
    for cfg in (W.SMALL_HEMI, W.C1_BELL):
        g = oracle_mod.Model(cfg).geometry()
        V0 = cfg.dx * cfg.dy * cfg.dz
        owners = (g["cls"] != 0) & (g["root"].ravel().reshape(g["cls"].shape) ==
                                    np.arange(g["cls"].size).reshape(g["cls"].shape))
        assert np.all(g["vg"][owners] >= 0.5 * V0)
        # group volume is the sum of member volumes
        tot = np.zeros(g["cls"].size)
        np.add.at(tot, g["root"].ravel()[g["root"].ravel() >= 0], (g["vf"] * V0).ravel()[g["root"].ravel() >= 0])
        assert np.allclose(tot[owners.ravel()], g["vg"].ravel()[owners.ravel()], rtol=1e-14)


def _fig6(gx, gy):
    """Fig. 6 pseudocode as a truth table (offsets di, dj, dk)."""
    if abs(gx) <= 1 and abs(gy) <= 1:
        return (0, 0, 1)
    if gx > 1 and abs(gx) >= abs(gy):
        return (-1, 0, 0)
    if gx < -1 and abs(gx) >= abs(gy):
        return (1, 0, 0)
    if gy > 1 and abs(gx) < abs(gy):
        return (0, -1, 0)
    return (0, 1, 0)


def test_merge_targets_follow_fig6(oracle_mod):
    cfg = W.SMALL_HEMI
    m = oracle_mod.Model(cfg)
    g = m.geometry()
    nz, ny, nx = g["cls"].shape
    root = g["root"]
    seen = 0
    for k, j, i in zip(*np.nonzero(g["cls"] == 3)):
        di, dj, dk = _fig6(g["gx"][j, i], g["gy"][j, i])
        t = ((k + dk), (j + dj) % ny, (i + di) % nx)
        # the absorbed cell belongs to the same group as its Fig. 6 target
        assert root[k, j, i] == root[t]
        seen += 1
    assert seen > 0


def test_fig6_tie_rules():
    # gradients of exactly +-1 merge vertically; equal magnitudes above 1 go to x
    assert _fig6(1.0, -1.0) == (0, 0, 1)
    assert _fig6(2.0, 2.0) == (-1, 0, 0)
    assert _fig6(-2.0, 2.0) == (1, 0, 0)
    assert _fig6(0.5, -3.0) == (0, 1, 0)


def test_velocity_point_classes_and_stencils(oracle_mod):
    cfg = W.SMALL_HEMI
    m = oracle_mod.Model(cfg)
    p = m.points()
    g = m.geometry()
    gz = m.gz
    vcls = p["vcls"]
    h = m.h
    nzc = vcls.shape[0]
    # corners at or below the terrain are class UG
    Kz = (np.arange(nzc) - gz)[:, None, None] * cfg.dz
    assert np.all((vcls == 0) == (Kz <= h[None]))
    # every boundary stencil: the intersection lies on the normal line, the four
    # points are predicted, weights in [0, 1)
    nx, ny = cfg.nx, cfg.ny
    for J in range(ny):
        for I in range(nx):
            K, i0, j0 = p["bK"][J, I], p["bI"][J, I], p["bJ"][J, I]
            a, b = p["ba"][J, I], p["bb"][J, I]
            n = p["bn"][J, I]
            assert abs(np.dot(n, n) - 1.0) < 1e-14 and n[2] > 0
            assert 0.0 <= a < 1.0 and 0.0 <= b < 1.0
            for (ii, jj, wgt) in ((i0, j0, (1 - a) * (1 - b)), (i0 + 1, j0, a * (1 - b)),
                                  (i0, j0 + 1, (1 - a) * b), (i0 + 1, j0 + 1, a * b)):
                assert wgt == 0.0 or vcls[K + gz, jj % ny, ii % nx] == 1
            # N - B is parallel to n (x and y offsets up to whole periods)
            t = (K * cfg.dz - h[J, I]) / n[2]
            xN = (i0 + a) * cfg.dx
            yN = (j0 + b) * cfg.dy
            dxN = (I * cfg.dx + t * n[0]) - xN
            dyN = (J * cfg.dy + t * n[1]) - yN
            assert abs(dxN / (nx * cfg.dx) - round(dxN / (nx * cfg.dx))) < 1e-12
            assert abs(dyN / (ny * cfg.dy) - round(dyN / (ny * cfg.dy))) < 1e-12
    # merged-face weights lie in (0, 1)
    mf = vcls == 2
    assert np.all((p["mg"][mf] > 0) & (p["mg"][mf] < 1))


def test_gradient_formulas_closed_form(oracle_mod):
    """Column gradients of Eqs. xgrad/ygrad equal the exact gradient of a plane."""
    nx = ny = 8
    cfg = W.RunConfig("t", nx, ny, 8, 50.0, 40.0, 50.0, 0.1, 1, "flat", 0.0, 1.0, U=0.0)
    # a periodic-safe check: a 'roof' with slope 0.3 in x over the interior columns
    h = np.zeros((ny, nx))
    for I in range(nx):
        h[:, I] = 20.0 + 0.3 * 50.0 * min(I, 4)
    g = oracle_mod.Model(cfg, h).geometry()
    assert np.allclose(g["gx"][:, :4], 0.3, atol=1e-15)
    assert np.allclose(g["gy"], 0.0, atol=1e-15)
    assert np.allclose(g["hc"][:, 0], 20.0 + 0.5 * 15.0)
