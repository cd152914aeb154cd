"""Pins of the oracle's time step (paper Sec 2.2, 2.4) against closed forms,
impulse responses, conservation and symmetry."""
import math

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W


def _flat(nx, ny, nz, dx, dy, dz, dt, **kw):
    base = dict(U=0.0, c4=0.0, sponge_frac=0.0, ra_nu=0.0)
    base.update(kw)
    return W.RunConfig("flat", nx, ny, nz, dx, dy, dz, dt, 1, "flat", 0.0, 1.0, **base)


# ---------------------------------------------------------------- acoustic modes
def _leapfrog_mode(a, b, P0, dt, n):
    """Exact discrete evolution of dP/dt = -a M, dM/dt = b P under one
    forward-Euler step followed by leapfrog (no filter)."""
    A = np.array([[0.0, -a], [b, 0.0]])
    x0 = np.array([P0, 0.0])
    x1 = x0 + dt * A @ x0
    xs = [x0, x1]
    for _ in range(n - 1):
        xs.append(xs[-2] + 2.0 * dt * A @ xs[-1])
    return xs[n]


@pytest.mark.parametrize("axis,m", [("x", 1), ("x", 3), ("y", 2), ("z", 1), ("z", 4)])
@pytest.mark.parametrize("floor", [0.0, 10.0])
def test_acoustic_mode_matches_closed_form(oracle_mod, axis, m, floor):
    """With g = 0 a standing sound wave along one axis is an exact mode of the
    discrete system: divergence and pressure gradient of Sec 2.4 act on it as
    multiplication by s = (2/d) sin(k d / 2), and the equation of state gives
    the sound speed squared gamma p / rho.  A raised flat floor (cut bottom
    cells, terrain below the first corner level) must not change it."""
    nx, ny, nz, d = (16, 4, 6, 100.0) if axis == "x" else ((4, 16, 6, 100.0) if axis == "y" else (4, 4, 12, 100.0))
    if axis == "z" and floor:
        pytest.skip("the raised floor pin is for horizontal modes")
    dt, n = 0.1, 30
    cfg = _flat(nx, ny, nz, d, d, d, dt, g=0.0, N=0.0)
    h = np.full((ny, nx), floor)
    om = oracle_mod.Model(cfg, h)
    om.init_state()
    gz = om.gz
    P0 = 1e-3
    nk = {"x": nx, "y": ny, "z": nz}[axis]
    if axis == "z":
        th = math.pi * m / nk
    else:
        th = 2.0 * math.pi * m / nk
    idx_c = np.arange(nk) + 0.5
    pp = np.zeros(om.cell_shape)
    if axis == "x":
        pp[:] = P0 * np.cos(th * idx_c)[None, None, :]
    elif axis == "y":
        pp[:] = P0 * np.cos(th * idx_c)[None, :, None]
    else:
        pp[:] = P0 * np.cos(th * idx_c)[:, None, None]
    om.set_field(oracle_mod.F_PP, 1, pp)
    om.step(n)
    # closed form
    gamma = cfg.cp / (cfg.cp - cfg.R)
    pbar = cfg.p_surf
    rhobar = pbar / (cfg.R * cfg.theta0)
    s = 2.0 / d * math.sin(0.5 * th)
    Pn, Mn = _leapfrog_mode(gamma * pbar * s / rhobar, s, P0, dt, n)
    got_p = om.field(oracle_mod.F_PP)
    if axis == "x":
        exp_p = Pn * np.cos(th * idx_c)[None, None, :] * np.ones(om.cell_shape)
    elif axis == "y":
        exp_p = Pn * np.cos(th * idx_c)[None, :, None] * np.ones(om.cell_shape)
    else:
        exp_p = Pn * np.cos(th * idx_c)[:, None, None] * np.ones(om.cell_shape)
    if floor:
        # the bottom layer is cut (fluid fraction 0.9) but keeps the same mode
        assert np.all(om.geometry()["vf"][0] < 1.0)
    assert np.max(np.abs(got_p - exp_p)) <= 2e-6 * P0
    # momentum on predicted corners
    vcls = om.points()["vcls"]
    fld = {"x": oracle_mod.F_MX, "y": oracle_mod.F_MY, "z": oracle_mod.F_MZ}[axis]
    M = om.field(fld)
    Kc = np.arange(om.corner_shape[0]) - gz
    if axis == "x":
        exp_m = Mn * np.sin(th * np.arange(nx))[None, None, :] * np.ones(om.corner_shape)
    elif axis == "y":
        exp_m = Mn * np.sin(th * np.arange(ny))[None, :, None] * np.ones(om.corner_shape)
    else:
        exp_m = Mn * np.sin(th * Kc)[:, None, None] * np.ones(om.corner_shape)
    pred = vcls == oracle_mod.V_PRED
    scale = max(abs(Mn), 1e-30)
    assert np.max(np.abs(M[pred] - exp_m[pred])) <= 2e-6 * scale + 1e-20


# ---------------------------------------------------------------- impulse responses
def _impulse_model(oracle_mod, **kw):
    cfg = _flat(12, 10, 8, 100.0, 80.0, 50.0, 0.2, **kw)
    om = oracle_mod.Model(cfg, np.zeros((cfg.ny, cfg.nx)))
    om.init_state()
    return cfg, om


def _tall_impulse_model(oracle_mod, **kw):
    """12 levels: an impulse at level 5 and every point its diffusion reaches
    (levels 3 .. 7) lie two or more points from the floor and the lid, so
    every stencil involved is the fourth-order one."""
    cfg = _flat(12, 10, 12, 100.0, 80.0, 50.0, 0.2, **kw)
    om = oracle_mod.Model(cfg, np.zeros((cfg.ny, cfg.nx)))
    om.init_state()
    return cfg, om


def test_buoyancy_impulse(oracle_mod):
    """A single-cell density perturbation at rest: after one forward step the
    eight corners of the cell carry w-momentum -dt g rho'/8 (the 8-point mean
    of Eq. momentum_w_d), nothing else moves."""
    cfg, om = _impulse_model(oracle_mod)
    i, j, k, dl = 5, 4, 3, 1e-3
    rp = np.zeros(om.cell_shape)
    rp[k, j, i] = dl
    om.set_field(oracle_mod.F_RHOP, 1, rp)
    om.step(1)
    gz = om.gz
    mz = om.field(oracle_mod.F_MZ)
    expect = np.zeros(om.corner_shape)
    for K in (k, k + 1):
        for J in (j, j + 1):
            for I in (i, i + 1):
                expect[K + gz, J, I] = -cfg.dt * cfg.g * dl / 8.0
    pred = om.points()["vcls"] == oracle_mod.V_PRED
    assert np.max(np.abs(mz[pred] - expect[pred])) <= 1e-18
    assert np.max(np.abs(om.field(oracle_mod.F_MX)[pred])) <= 1e-18
    assert np.max(np.abs(om.field(oracle_mod.F_MY)[pred])) <= 1e-18
    assert np.array_equal(om.field(oracle_mod.F_RHOP), rp)


def test_pressure_gradient_impulse(oracle_mod):
    """A single-cell pressure perturbation at rest pushes the momentum of its
    eight corners outward by dt p'/(4 d) along each axis (the four-cell means of
    Eqs. momentum_u_d .. w_d)."""
    cfg, om = _impulse_model(oracle_mod, g=0.0, N=0.0)
    i, j, k, dp = 6, 5, 4, 0.7
    pp = np.zeros(om.cell_shape)
    pp[k, j, i] = dp
    om.set_field(oracle_mod.F_PP, 1, pp)
    om.step(1)
    gz = om.gz
    pred = om.points()["vcls"] == oracle_mod.V_PRED
    for fld, d, ax in ((oracle_mod.F_MX, cfg.dx, 2), (oracle_mod.F_MY, cfg.dy, 1), (oracle_mod.F_MZ, cfg.dz, 0)):
        M = om.field(fld)
        expect = np.zeros(om.corner_shape)
        for K in (k, k + 1):
            for J in (j, j + 1):
                for I in (i, i + 1):
                    side = (I, J, K)[2 - ax] - (i, j, k)[2 - ax]  # 0: cell lies on the + side
                    expect[K + gz, J, I] = cfg.dt * dp / (4.0 * d) * (1.0 if side else -1.0)
        assert np.max(np.abs(M[pred] - expect[pred])) <= 1e-15 * abs(cfg.dt * dp / d)


def test_fourth_order_diffusion_impulse(oracle_mod):
    """Artificial diffusion of (rho theta)' away from every wall: linearised
    about the base state the pressure responds with the 5-point stencil
    (1,-4,6,-4,1) times c4/16 on each axis (since
    (c_p R/c_v)(p/p0)^(R/c_p) d(rho theta)/dp = 1)."""
    c4 = 0.02
    cfg, om = _tall_impulse_model(oracle_mod, g=0.0, N=0.0, c4=c4)
    i, j, k, dp = 6, 5, 5, 1e-2
    pp = np.zeros(om.cell_shape)
    pp[k, j, i] = dp
    om.set_field(oracle_mod.F_PP, 1, pp)
    om.step(1)
    got = om.field(oracle_mod.F_PP)
    w = c4 / 16.0 * dp
    expect = np.zeros(om.cell_shape)
    expect[k, j, i] = dp - 18.0 * w
    for a, c in ((1, -4.0), (2, 1.0)):
        for s in (-1, 1):
            expect[k, j, i + s * a] += -c * w
            expect[k, j + s * a, i] += -c * w
            expect[k + s * a, j, i] += -c * w
    assert np.max(np.abs(got - expect)) <= 1e-6 * w


def test_momentum_diffusion_impulse(oracle_mod):
    c4 = 0.02
    cfg, om = _tall_impulse_model(oracle_mod, g=0.0, N=0.0, c4=c4)
    gz = om.gz
    I, J, K, dm = 6, 5, 5, 1e-7
    mx = np.zeros(om.corner_shape)
    mx[K + gz, J, I] = dm
    om.set_field(oracle_mod.F_MX, 1, mx)
    om.step(1)
    got = om.field(oracle_mod.F_MX)
    w = c4 / 16.0 * dm
    expect = np.zeros(om.corner_shape)
    expect[K + gz, J, I] = dm - 18.0 * w
    for a, c in ((1, -4.0), (2, 1.0)):
        for s in (-1, 1):
            expect[K + gz, J, I + s * a] += -c * w
            expect[K + gz, J + s * a, I] += -c * w
            expect[K + s * a + gz, J, I] += -c * w
    pred = om.points()["vcls"] == oracle_mod.V_PRED
    assert np.max(np.abs(got[pred] - expect[pred])) <= 1e-6 * w


# ---------------------------------------------------------------- rest state, conservation, symmetry
def test_rest_state_over_steep_terrain_stays_at_rest(oracle_mod):
    """No wind, no perturbation over the steep hemisphere: every tendency is zero
    (perturbation form of Sec 2.1), so the state stays exactly at rest."""
    cfg = W.SMALL_HEMI.replace(U=0.0)
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(15)
    for f in (oracle_mod.F_RHOP, oracle_mod.F_PP, oracle_mod.F_MX, oracle_mod.F_MY, oracle_mod.F_MZ,
              oracle_mod.F_UB):
        assert np.max(np.abs(om.field(f))) == 0.0


@pytest.mark.parametrize("cfg", [W.SMALL_HEMI, W.C1_BELL.replace(steps=20)], ids=["hemisphere", "bell"])
def test_mass_conserved_to_round_off(oracle_mod, cfg):
    """Perturbation mass sum V_G rho'_G is conserved across cut cells and merges
    (Sec 2.4: the first-order face scalar does not violate conservation),
    also with the Robert-Asselin filter because the first step conserves it."""
    om = oracle_mod.Model(cfg)
    om.init_state()
    m0 = om.mass(1)
    V0 = cfg.dx * cfg.dy * cfg.dz
    masses = []
    for _ in range(4):
        om.step(5)
        masses.append(om.mass(1))
    rp = om.field(oracle_mod.F_RHOP)
    scale = np.abs(rp).max() * V0 * cfg.cells
    assert scale > 0
    for m in masses:
        assert abs(m - m0) <= 1e-13 * scale, (m, m0, scale)


def _bubble(om, cfg, zc, amp, r):
    kk, jj, ii = np.meshgrid(np.arange(cfg.nz) + 0.5, np.arange(cfg.ny) + 0.5, np.arange(cfg.nx) + 0.5,
                             indexing="ij")
    x = ii * cfg.dx - 0.5 * cfg.nx * cfg.dx
    y = jj * cfg.dy - 0.5 * cfg.ny * cfg.dy
    z = kk * cfg.dz - zc
    d2 = (x * x + y * y + z * z) / (r * r)
    return amp * np.exp(-d2)


def test_mirror_symmetry_over_hemisphere(oracle_mod):
    """The merge rules are sign-symmetric (Fig. 6), so a pressure bubble above the
    hemisphere at rest evolves mirror-symmetrically in x and in y."""
    cfg = W.SMALL_HEMI.replace(U=0.0)
    om = oracle_mod.Model(cfg)
    om.init_state()
    g = om.geometry()
    pp = _bubble(om, cfg, 700.0, 50.0, 150.0)
    owners = (g["cls"] != 0)
    om.set_field(oracle_mod.F_PP, 1, np.where(owners, pp, 0.0))
    om.step(12)
    p = om.field(oracle_mod.F_PP)
    mx = om.field(oracle_mod.F_MX)
    my = om.field(oracle_mod.F_MY)
    mz = om.field(oracle_mod.F_MZ)
    sp, sm = np.abs(p).max(), max(np.abs(mx).max(), np.abs(mz).max())
    # cells: i -> nx-1-i ; corners: I -> nx-I (mod nx)
    assert np.max(np.abs(p - p[:, :, ::-1])) <= 1e-11 * sp
    assert np.max(np.abs(p - p[:, ::-1, :])) <= 1e-11 * sp
    Im = (-np.arange(cfg.nx)) % cfg.nx
    Jm = (-np.arange(cfg.ny)) % cfg.ny
    assert np.max(np.abs(mx + mx[:, :, Im])) <= 1e-11 * sm
    assert np.max(np.abs(mz - mz[:, :, Im])) <= 1e-11 * sm
    assert np.max(np.abs(my + my[:, Jm, :])) <= 1e-11 * sm
    assert np.max(np.abs(mz - mz[:, Jm, :])) <= 1e-11 * sm
    assert sm > 0


def test_transpose_symmetry_over_bell(oracle_mod):
    """With nx = ny and dx = dy the bell hill (vertical merges only) is symmetric
    under x <-> y; a symmetric bubble must stay symmetric with u and v swapped."""
    cfg = W.RunConfig("bellT", 24, 24, 16, 100.0, 100.0, 100.0, 0.1, 1, "bell", 150.0, 600.0, U=0.0)
    om = oracle_mod.Model(cfg)
    om.init_state()
    pp = _bubble(om, cfg, 600.0, 30.0, 200.0)
    g = om.geometry()
    om.set_field(oracle_mod.F_PP, 1, np.where(g["cls"] != 0, pp, 0.0))
    om.step(10)
    p = om.field(oracle_mod.F_PP)
    mx, my, mz = om.field(oracle_mod.F_MX), om.field(oracle_mod.F_MY), om.field(oracle_mod.F_MZ)
    sp, sm = np.abs(p).max(), np.abs(mx).max()
    assert np.max(np.abs(p - p.transpose(0, 2, 1))) <= 1e-11 * sp
    assert np.max(np.abs(mx - my.transpose(0, 2, 1))) <= 1e-11 * sm
    assert np.max(np.abs(mz - mz.transpose(0, 2, 1))) <= 1e-11 * sm


def test_free_slip_boundary_velocity_is_tangential(oracle_mod):
    cfg = W.SMALL_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(3)
    ub = om.field(oracle_mod.F_UB)
    n = om.points()["bn"]
    un = np.einsum("jid,jid->ji", ub, n)
    assert np.max(np.abs(un)) <= 1e-13 * np.abs(ub).max()
    assert np.abs(ub).max() > 1.0


def test_no_slip_boundary_velocity_is_zero(oracle_mod):
    cfg = W.SMALL_HEMI.replace(bc_slip=0)
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(3)
    assert np.all(om.field(oracle_mod.F_UB) == 0.0)


def test_base_state_hydrostatic_and_stable(oracle_mod):
    """Base state: dp/dz = -rho g (to the second-order accuracy of a centred
    difference) and theta = theta0 exp(N^2 z / g) through the equation of state."""
    # 5 m levels: the centred difference is accurate to ~(dz/H)^2/6 ~ 1e-7
    cfg = W.C1_BELL.replace(nx=4, ny=4, nz=40, dz=5.0, terrain="flat")
    om = oracle_mod.Model(cfg)
    rhob, pb, koff = om.base()
    dz = cfg.dz
    k = np.arange(len(rhob)) - koff
    z = (k + 0.5) * dz
    dpdz = (pb[2:] - pb[:-2]) / (2 * dz)
    assert np.max(np.abs(dpdz + rhob[1:-1] * cfg.g) / (rhob[1:-1] * cfg.g)) < 1e-6
    kap = cfg.R / cfg.cp
    theta = pb / (rhob * cfg.R) * (cfg.p0 / pb) ** kap
    assert np.max(np.abs(theta / (cfg.theta0 * np.exp(cfg.N ** 2 * z / cfg.g)) - 1.0)) < 1e-13
    # 288 K surface air at 1000 hPa (config C1)
    assert abs(cfg.theta0 - 288.0) < 1e-12
