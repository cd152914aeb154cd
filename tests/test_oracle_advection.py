"""Pins of the oracle's advection at U != 0 (paper Sec 2.4: the scalar fluxes
of Eqs. ux1 - ux3 with the face value the mean of the two cells, and the
momentum equations momentum_u_d .. momentum_w_d with face densities the mean of
the four cells touching the face and advected values the mean of two corners).

A single Fourier mode riding on a uniform wind U over a flat floor, with
g = 0 and N = 0 (a uniform base state), stays a mode of the linearised
discrete system.  Its amplitudes s = (rho', p', (rho u)', (rho v)') obey
ds/dt = A s, with A worked out by hand from the discrete operators:
with a = 2 pi mx / nx, b = 2 pi my / ny (radians per cell), Cx = cos(a/2),
Cy = cos(b/2), Dx = 2i sin(a/2)/dx, Dy = 2i sin(b/2)/dy and c^2 = gamma p / rho,

  d rho'/dt   = -Dx U Cx (1 - Cy^2) rho' - Dx Cy mx - Dy Cx my
  d p'/dt     = -Dx U Cx p' - c^2 (Dx Cy (mx - U Cx Cy rho') + Dy Cx my)
  d mx/dt     = -Dx U^2 Cy (1 - 2 Cx^2) rho' - 2 Dx U Cx mx - Dy U Cy my - Dx Cy p'
  d my/dt     = -Dx U Cx my - Dy Cx p'

(the corner density is the four-column mean Cx Cy rho', the corner velocity
perturbation (mx - U Cx Cy rho')/rho; the mass and heat fluxes through an
x-face carry U Cx rho' + rho Cy u', the momentum flux through the east face of
a velocity cell U^2 Cy rho' + 2 rho U Cx u', through the north face rho U Cy v').
The step is one forward-Euler step, then leapfrog, no filter; the oracle must
follow the recurrence to O(eps^2).  Face densities from two cells instead of
four, a dropped one-half, or upwind face values change A and fail the test.
Over a raised floor the bottom cells are cut (fluid fraction 0.8, apertures
0.8): the mode survives only if every face flux carries its aperture.

The z-face terms are pinned by single-step impulses under the same wind
(test_*_impulse_under_wind below).
"""
import cmath
import math

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

U_DEFAULT = 12.0


def _cfg(nx, ny, nz, U, dt=0.05):
    return W.RunConfig("wind", nx, ny, nz, 100.0, 80.0, 50.0, dt, 1, "flat", 0.0, 1.0,
                       U=U, g=0.0, N=0.0, c4=0.0, sponge_frac=0.0, ra_nu=0.0)


def _system(cfg, mx_, my_, rho, p):
    a = 2.0 * math.pi * mx_ / cfg.nx
    b = 2.0 * math.pi * my_ / cfg.ny
    Cx, Cy = math.cos(0.5 * a), math.cos(0.5 * b)
    Dx = 2j * math.sin(0.5 * a) / cfg.dx
    Dy = 2j * math.sin(0.5 * b) / cfg.dy
    U = cfg.U
    c2 = cfg.cp / (cfg.cp - cfg.R) * p / rho
    A = np.zeros((4, 4), complex)
    A[0] = [-Dx * U * Cx * (1 - Cy * Cy), 0.0, -Dx * Cy, -Dy * Cx]
    A[1] = [c2 * Dx * Cy * U * Cx * Cy, -Dx * U * Cx, -c2 * Dx * Cy, -c2 * Dy * Cx]
    A[2] = [-Dx * U * U * Cy * (1 - 2 * Cx * Cx), -Dx * Cy, -2 * Dx * U * Cx, -Dy * U * Cy]
    A[3] = [0.0, -Dy * Cx, 0.0, -Dx * U * Cx]
    return A, a, b


def _evolve(A, s0, dt, n):
    s_prev, s = s0, s0 + dt * A @ s0
    for _ in range(n - 1):
        s_prev, s = s, s_prev + 2.0 * dt * A @ s
    return s


def _set_mode(oracle_mod, om, cfg, a, b, s0):
    """State = uniform wind + Re(s0 * exp(i (a x + b y))), x, y in cell units;
    the lid corners and the boundary velocity consistent with a z-uniform
    flow (free-slip lid: the velocity below; flat floor: the velocity of the
    first corner level above it)."""
    nx, ny, nz, gz = cfg.nx, cfg.ny, cfg.nz, om.gz
    rho, p = _base(om)
    ic, jc = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    Ec = np.exp(1j * (a * ic[None, :] + b * jc[:, None]))
    Ek = np.exp(1j * (a * np.arange(nx)[None, :] + b * np.arange(ny)[:, None]))
    r2 = (s0[0] * Ec).real
    p2 = (s0[1] * Ec).real
    om.set_field(oracle_mod.F_RHOP, 1, np.broadcast_to(r2, om.cell_shape))
    om.set_field(oracle_mod.F_PP, 1, np.broadcast_to(p2, om.cell_shape))
    mx2 = rho * cfg.U + (s0[2] * Ek).real
    my2 = (s0[3] * Ek).real
    # corner density of the interior (four columns, any two adjacent levels)
    # and of the lid (the cell level above the lid has no perturbation)
    r4 = 0.25 * (r2 + np.roll(r2, 1, 1) + np.roll(r2, 1, 0) + np.roll(np.roll(r2, 1, 0), 1, 1))
    rc_in, rc_lid = rho + r4, rho + 0.5 * r4
    MX = np.broadcast_to(mx2, om.corner_shape).copy()
    MY = np.broadcast_to(my2, om.corner_shape).copy()
    K = nz + gz
    MX[K] = rc_lid * mx2 / rc_in
    MY[K] = rc_lid * my2 / rc_in
    om.set_field(oracle_mod.F_MX, 1, MX)
    om.set_field(oracle_mod.F_MY, 1, MY)
    om.set_field(oracle_mod.F_MZ, 1, np.zeros(om.corner_shape))
    ub = np.zeros((ny, nx, 3))
    ub[..., 0] = mx2 / rc_in
    ub[..., 1] = my2 / rc_in
    om.set_field(oracle_mod.F_UB, 1, ub)
    return Ec, Ek


def _base(om):
    rhob, pb, koff = om.base()
    assert np.ptp(rhob) == 0.0 and np.ptp(pb) == 0.0  # g = 0: uniform base state
    return rhob[0], pb[0]


def _initial(rho, p, my_):
    eps = 1e-7
    s0 = np.array([eps * rho * cmath.exp(0.3j), eps * p * cmath.exp(-1.1j),
                   eps * rho * 300.0 * cmath.exp(0.7j), eps * rho * 200.0 * cmath.exp(2.0j)])
    if my_ == 0:
        s0[3] = 0.0  # an x-mode has no v (nothing drives it)
    return s0


def _scales(s0):
    return np.array([abs(s0[q]) if abs(s0[q]) else abs(s0[0]) * 300.0 for q in range(4)])


TOL = 1e-5

CASES = [
    (1, 0, U_DEFAULT), (0, 1, U_DEFAULT), (1, 1, U_DEFAULT), (2, 1, -7.0), (3, 2, U_DEFAULT), (1, 3, 20.0),
]


@pytest.mark.parametrize("floor", [0.0, 10.0], ids=["floor-at-0", "raised-floor"])
@pytest.mark.parametrize("mx_,my_,U", CASES)
def test_fourier_mode_on_a_uniform_wind(oracle_mod, mx_, my_, U, floor):
    cfg = _cfg(16, 12, 4, U)
    om = oracle_mod.Model(cfg, np.full((cfg.ny, cfg.nx), floor))
    om.init_state()
    if floor:
        g = om.geometry()
        assert np.allclose(g["vf"][0], 0.8) and np.allclose(g["ax"][0], 0.8) and np.allclose(g["ay"][0], 0.8)
    rho, p = _base(om)
    A, a, b = _system(cfg, mx_, my_, rho, p)
    s0 = _initial(rho, p, my_)
    Ec, Ek = _set_mode(oracle_mod, om, cfg, a, b, s0)
    n = 60
    om.step(n)
    s = _evolve(A, s0, cfg.dt, n)
    got = [om.field(oracle_mod.F_RHOP), om.field(oracle_mod.F_PP),
           om.field(oracle_mod.F_MX) - rho * cfg.U, om.field(oracle_mod.F_MY)]
    pred = om.points()["vcls"] == oracle_mod.V_PRED
    for q in range(4):
        E = Ec if q < 2 else Ek
        exp_ = np.broadcast_to((s[q] * E).real, got[q].shape)
        scale = _scales(s0)[q]
        err = np.abs(got[q] - exp_)
        if q >= 2:
            err = err[pred]
        assert err.max() <= TOL * scale, (q, err.max() / scale)
    # the mode moved: the recurrence is not the identity here
    assert abs(s[0] - s0[0]) > 0.05 * abs(s0[0])


def test_advection_recurrence_detects_slips():
    """The recurrence tells the scheme apart from its likely slips: from the
    initial state of the test above, each variant's amplitudes after 60 steps
    differ from the scheme's by ten times its tolerance or more."""
    cfg = _cfg(16, 12, 4, U_DEFAULT)
    rho, p = 1.2, 1.0e5
    A, a, b = _system(cfg, 1, 1, rho, p)
    s0 = _initial(rho, p, 1)
    ref = _evolve(A, s0, cfg.dt, 60)
    Cx, Cy = math.cos(0.5 * a), math.cos(0.5 * b)
    Dx, Dy = 2j * math.sin(0.5 * a) / cfg.dx, 2j * math.sin(0.5 * b) / cfg.dy
    U = cfg.U
    slips = {}
    B = A.copy(); B[2, 0] = -Dx * U * U * 1.0 * (1 - 2 * Cx * Cx); slips["east-face density of one cell column"] = B
    B = A.copy(); B[2, 2] = -Dx * U * Cx; slips["advected value without its one-half"] = B
    # upwind (U > 0) face value: the mass flux takes the upstream cell, symbol exp(-i a / 2)
    up = cmath.exp(-0.5j * a)
    B = A.copy(); B[0, 0] = -Dx * U * (up - Cx * Cy * Cy); slips["upwind face density"] = B
    for name, B in slips.items():
        s = _evolve(B, s0, cfg.dt, 60)
        assert np.max(np.abs(s - ref) / _scales(s0)) > 10 * TOL, name


# ---------------------------------------------------------------- impulses carried by an exactly uniform wind
def _uniform_wind_state(oracle_mod, om, cfg, wind, cell, dr=0.0, dp=0.0):
    """rho' = dr and p' = dp in one cell, and momentum rho_c * wind at every
    corner, so that every corner velocity above the floor and below the lid
    equals the wind exactly (boundary velocity and lid: the free-slip values
    of a wind parallel to them, zero for a vertical wind)."""
    nx, ny, nz, gz = cfg.nx, cfg.ny, cfg.nz, om.gz
    rho, _ = _base(om)
    i, j, k = cell
    r = np.zeros(om.cell_shape)
    r[k, j, i] = dr
    pp = np.zeros(om.cell_shape)
    pp[k, j, i] = dp
    om.set_field(oracle_mod.F_RHOP, 1, r)
    om.set_field(oracle_mod.F_PP, 1, pp)
    # corner density: mean of the 8 cells around (cells outside the fluid at the base state)
    rp = np.zeros((nz + 2, ny, nx))
    rp[1:nz + 1] = r
    rc = np.zeros(om.corner_shape)
    for K in range(0, nz + 1):
        s = np.zeros((ny, nx))
        for kk in (K - 1, K):
            a = rp[kk + 1]
            s += a + np.roll(a, 1, 1) + np.roll(a, 1, 0) + np.roll(np.roll(a, 1, 0), 1, 1)
        rc[K + gz] = rho + s / 8.0
    rc[:gz] = rho
    rc[nz + gz + 1:] = rho
    vertical = wind[2] != 0.0
    for f, wv in zip((oracle_mod.F_MX, oracle_mod.F_MY, oracle_mod.F_MZ), wind):
        M = rc * wv
        if f == oracle_mod.F_MZ or vertical:
            M[nz + gz] = 0.0  # lid: w = 0 (and no tangential flow under a vertical wind)
        om.set_field(f, 1, M)
    ub = np.zeros((ny, nx, 3))
    if not vertical:
        ub[..., 0], ub[..., 1] = wind[0], wind[1]
    om.set_field(oracle_mod.F_UB, 1, ub)


@pytest.mark.parametrize("axis", [0, 1, 2], ids=["wind-x", "wind-y", "wind-z"])
def test_density_impulse_in_a_uniform_wind(oracle_mod, axis):
    """One forward step with every velocity equal to the wind (speed V along
    the axis): the face value of the mass flux is the mean of the two cells,
    so the cells up- and downwind of the impulse change by -/+ dt V dr / (2 d)
    and the impulse cell not at all (centred, not upwind); the momentum of the
    eight corners of the velocity cells whose faces the impulse cell touches
    changes through the face densities (the means of the four cells on each
    face): -dt V^2 dr / (4 d) on the corners behind the cell's centre plane
    (the cell is on their downwind face), +dt V^2 dr / (4 d) on those ahead.
    Exact, with no linearisation: the velocities are the wind at every
    corner."""
    cfg = _cfg(12, 10, 10, 0.0, dt=0.05)
    om = oracle_mod.Model(cfg, np.zeros((cfg.ny, cfg.nx)))
    om.init_state()
    rho, _ = _base(om)
    V = 9.0
    wind = [0.0, 0.0, 0.0]
    wind[axis] = V
    i, j, k = 5, 4, 4
    dr = 1e-3
    _uniform_wind_state(oracle_mod, om, cfg, wind, (i, j, k), dr=dr)
    om.step(1)
    d = (cfg.dx, cfg.dy, cfg.dz)[axis]
    dt = cfg.dt
    # scalars: the 3x3x3 cells around the impulse
    r = om.field(oracle_mod.F_RHOP)
    e = np.zeros((3, 3, 3))
    e[1, 1, 1] = dr
    up = [1, 1, 1]
    up[2 - axis] = 0
    dn = [1, 1, 1]
    dn[2 - axis] = 2
    e[tuple(up)] += -dt * V * dr / (2 * d)
    e[tuple(dn)] += dt * V * dr / (2 * d)
    got = r[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
    assert np.max(np.abs(got - e)) <= 1e-12 * dr
    # a density impulse does not change rho theta: no pressure change near it
    # (a vertical wind compresses the layers at the floor and the lid)
    assert np.max(np.abs(om.field(oracle_mod.F_PP)[k - 2:k + 3])) == 0.0
    # momentum of the wind component on the corners I in i .. i+1 (and J, K alike)
    gz = om.gz
    F = (oracle_mod.F_MX, oracle_mod.F_MY, oracle_mod.F_MZ)[axis]
    M = om.field(F)
    rc_expect = np.zeros((4, 4, 4))  # corners K, J, I in k-1 .. k+2 etc.
    for Kk in range(2):
        for Jj in range(2):
            for Ii in range(2):
                lead = (Ii, Jj, Kk)[axis]  # 0: the corner's velocity cell has the impulse on its + face
                rc_expect[Kk + 1, Jj + 1, Ii + 1] = (-1.0 if lead == 0 else 1.0) * dt * V * V * dr / (4 * d)
    # the corner's own momentum before the step was rho_c V
    rc0 = rho + dr / 8.0
    got_m = M[k - 1 + gz:k + 3 + gz, j - 1:j + 3, i - 1:i + 3].copy()
    base = np.full((4, 4, 4), rho * V)
    base[1:3, 1:3, 1:3] = rc0 * V
    assert np.max(np.abs(got_m - base - rc_expect)) <= 1e-12 * V * V * dr
    for other in range(3):
        if other != axis:
            Mo = om.field((oracle_mod.F_MX, oracle_mod.F_MY, oracle_mod.F_MZ)[other])
            assert np.max(np.abs(Mo[k - 1 + gz:k + 3 + gz, j - 1:j + 3, i - 1:i + 3])) == 0.0


@pytest.mark.parametrize("axis", [0, 1, 2], ids=["wind-x", "wind-y", "wind-z"])
def test_pressure_impulse_in_a_uniform_wind(oracle_mod, axis):
    """The heat flux carries the mean of the two cells' rho theta: a pressure
    impulse dp is advected like the density, -/+ dt V dp / (2 d) on the cells
    up- and downwind (to first order in dp, since (c_p R/c_v)(p/p0)^(R/c_p)
    d(rho theta)/dp = 1)."""
    cfg = _cfg(12, 10, 10, 0.0, dt=0.05)
    om = oracle_mod.Model(cfg, np.zeros((cfg.ny, cfg.nx)))
    om.init_state()
    V = 9.0
    wind = [0.0, 0.0, 0.0]
    wind[axis] = V
    i, j, k = 5, 4, 4
    dp = 1e-2
    _uniform_wind_state(oracle_mod, om, cfg, wind, (i, j, k), dp=dp)
    om.step(1)
    d = (cfg.dx, cfg.dy, cfg.dz)[axis]
    p = om.field(oracle_mod.F_PP)[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
    e = np.zeros((3, 3, 3))
    e[1, 1, 1] = dp
    up = [1, 1, 1]
    up[2 - axis] = 0
    dn = [1, 1, 1]
    dn[2 - axis] = 2
    e[tuple(up)] += -cfg.dt * V * dp / (2 * d)
    e[tuple(dn)] += cfg.dt * V * dp / (2 * d)
    assert np.max(np.abs(p - e)) <= 1e-6 * cfg.dt * V * dp / d
