"""Pins of the oracle's artificial diffusion next to walls (paper Sec 2.1: a
fourth-order term in the horizontal and vertical directions; Sec 2.4: where a
cell lacks the neighbouring fluid points the fourth-order term needs, a
second-order term with the boundary conditions of the terrain surface).

Each case plants one impulse in a resting, weightless atmosphere (g = 0,
N = 0, U = 0) and checks the first (forward-Euler) step against the response
worked out by hand for that geometry.  With w = (c4 / 16) x amplitude the
fourth-order stencil gives (-1, +4, -6, +4, -1) w along an axis and the
second-order one (reading C-4: K2 = 4 K4 / d^2) gives 4 x (+1, -2, +1) w,
with a scalar neighbour outside the fluid taking the centre value (no flux
through the wall) and a velocity neighbour outside the fluid keeping its
stored (boundary) value, here zero.

A plausible slip in the rule fails one of them: the fourth order kept at the
wall (-18 w instead of -20 w at the impulse), the second order taken only
when a distance-1 neighbour is missing (the level-1 and plateau cases), a
Dirichlet zero instead of the zero gradient for scalars (-8 w instead of
-4 w on the first layer), absorbed cells counted as fluid (the ramp cases),
the floor corner counted as fluid (the floor at zero height).
"""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

C4 = 0.02
DP = 1e-2    # pressure impulse, Pa
DM = 1e-7    # momentum impulse, kg m^-2 s^-1


def _cfg(nx, ny, nz, **kw):
    base = dict(U=0.0, c4=C4, sponge_frac=0.0, ra_nu=0.0, g=0.0, N=0.0)
    base.update(kw)
    return W.RunConfig("walls", nx, ny, nz, 100.0, 80.0, 50.0, 0.2, 1, "flat", 0.0, 1.0, **base)


def _model(oracle_mod, cfg, h):
    om = oracle_mod.Model(cfg, h)
    om.init_state()
    return om


def _in_layer(expect, at, amp, horizontal=("x", "y")):
    """fourth-order responses along x and y through `at` (k or K, j, i index
    order); the impulse's own -6 w per axis is added by the caller"""
    k, j, i = at
    ny, nx = expect.shape[1], expect.shape[2]
    w = C4 / 16.0 * amp
    for a, c in ((1, 4.0), (2, -1.0)):
        for s in (-1, 1):
            if "x" in horizontal:
                expect[k, j, (i + s * a) % nx] += c * w
            if "y" in horizontal:
                expect[k, (j + s * a) % ny, i] += c * w


# ---------------------------------------------------------------- floor and lid, scalar
# z responses (in units of w) of an impulse at level k; 'top' levels count from the lid
Z_SCALAR = {
    0: {0: -4.0, 1: 4.0, 2: -1.0},              # zero gradient below: 4 (psi1 - psi0)
    1: {0: 4.0, 1: -8.0, 2: 4.0, 3: -1.0},      # second order at 1, fourth order from 2 up
    "top": {0: -4.0, 1: 4.0, 2: -1.0},
    "top-1": {0: 4.0, 1: -8.0, 2: 4.0, 3: -1.0},
}


@pytest.mark.parametrize("floor", [0.0, 10.0], ids=["floor-at-0", "raised-floor"])
@pytest.mark.parametrize("where", [0, 1, "top", "top-1"])
def test_scalar_second_order_at_floor_and_lid(oracle_mod, floor, where):
    cfg = _cfg(8, 6, 10)
    om = _model(oracle_mod, cfg, np.full((cfg.ny, cfg.nx), floor))
    if floor:
        # the bottom layer is cut (fluid fraction 0.8) but owns its pressure points
        g = om.geometry()
        assert np.all(g["cls"][0] == oracle_mod.C_CUT) and np.allclose(g["vf"][0], 0.8)
    i, j = 3, 2
    k = {0: 0, 1: 1, "top": cfg.nz - 1, "top-1": cfg.nz - 2}[where]
    sgn = -1 if isinstance(where, str) else 1  # lid cases count down from the top
    pp = np.zeros(om.cell_shape)
    pp[k, j, i] = DP
    om.set_field(oracle_mod.F_PP, 1, pp)
    om.step(1)
    w = C4 / 16.0 * DP
    expect = np.zeros(om.cell_shape)
    expect[k, j, i] = DP - 12.0 * w
    _in_layer(expect, (k, j, i), DP)
    # the z responses: the table is indexed by the level counted from the wall
    wall0 = 0 if not isinstance(where, str) else cfg.nz - 1
    for lvl, c in Z_SCALAR[where].items():
        kk = wall0 + sgn * lvl
        expect[kk, j, i] += c * w
    got = om.field(oracle_mod.F_PP)
    assert np.max(np.abs(got - expect)) <= 1e-6 * w


# ---------------------------------------------------------------- floor and lid, momentum
Z_MOMENTUM = {
    1: {1: -8.0, 2: 4.0, 3: -1.0},              # corner 0 lies on the wall: second order at 1 and 2
    2: {1: 4.0, 2: -8.0, 3: 4.0, 4: -1.0},
    "top": {1: -8.0, 2: 4.0, 3: -1.0},          # corner nz lies on the lid
    "top-1": {1: 4.0, 2: -8.0, 3: 4.0, 4: -1.0},
}


@pytest.mark.parametrize("floor", [0.0, 10.0], ids=["floor-at-0", "raised-floor"])
@pytest.mark.parametrize("where", [1, 2, "top", "top-1"])
def test_momentum_second_order_at_floor_and_lid(oracle_mod, floor, where):
    cfg = _cfg(8, 6, 10)
    om = _model(oracle_mod, cfg, np.full((cfg.ny, cfg.nx), floor))
    gz = om.gz
    I, J = 3, 2
    K = {1: 1, 2: 2, "top": cfg.nz - 1, "top-1": cfg.nz - 2}[where]
    mx = np.zeros(om.corner_shape)
    mx[K + gz, J, I] = DM
    om.set_field(oracle_mod.F_MX, 1, mx)
    om.step(1)
    w = C4 / 16.0 * DM
    expect = np.zeros(om.corner_shape)
    expect[K + gz, J, I] = DM - 12.0 * w
    _in_layer(expect, (K + gz, J, I), DM)
    # levels counted from the wall corner (corner 0 on the floor, corner nz on the lid)
    for lvl, c in Z_MOMENTUM[where].items():
        KK = lvl if not isinstance(where, str) else cfg.nz - lvl
        expect[KK + gz, J, I] += c * w
    pred = om.points()["vcls"] == oracle_mod.V_PRED
    got = om.field(oracle_mod.F_MX)
    assert np.max(np.abs(got[pred] - expect[pred])) <= 1e-6 * w


# ---------------------------------------------------------------- horizontal: a one-column ramp
def _ramp(oracle_mod):
    """Flat floor for corners I <= 7, a plateau of 800 m (16 levels) for
    8 <= I <= 15, flat again from 16: column 7 rises by 8 levels per cell, so
    its cells have fluid fractions (2k + 1)/32 below the plateau top: absorbed
    (fraction below one half) for k <= 7 and merged into column 6 (the side of
    the lower terrain, Fig. 6), cut for 8 <= k <= 15; columns 8 .. 14 are below
    the terrain up to level 15."""
    cfg = _cfg(24, 6, 24)
    h = np.zeros((cfg.ny, cfg.nx))
    h[:, 8:16] = 800.0
    om = _model(oracle_mod, cfg, h)
    g = om.geometry()
    cls = g["cls"][:, 3, :]
    for k in range(16):
        assert cls[k, 7] == (oracle_mod.C_ABS if k <= 7 else oracle_mod.C_CUT), k
        assert np.isclose(g["vf"][k, 3, 7], (2 * k + 1) / 32.0)
        assert cls[k, 8] == oracle_mod.C_UG and cls[k, 6] == oracle_mod.C_FULL
    nx, ny = cfg.nx, cfg.ny
    for k in range(8):
        assert g["root"][k, 3, 7] == (k * ny + 3) * nx + 6  # host: the full cell at -x
    return cfg, om


@pytest.mark.parametrize("k", [5, 10], ids=["absorbed-at-+2", "cut-at-+2"])
def test_scalar_diffusion_next_to_ramp(oracle_mod, k):
    """Impulse in cell (5, 3, k).  At k = 5 its +2 neighbour (7, 3, 5) is
    absorbed, so x takes the second order (-8 w); the host (6, 3, 5) of that
    absorbed cell has neither (7) nor (8) as a fluid point: 4 (psi5 - psi6),
    i.e. +4 w, carried by its member too.  At k = 10 the +2 neighbour is cut
    (a fluid point): fourth order at the impulse, while the cut cell (7, 3, 10)
    itself, with (8) and (9) below the plateau, takes the second order with the
    zero gradient and sees nothing of the impulse (fourth order would give
    -w)."""
    cfg, om = _ramp(oracle_mod)
    i, j = 5, 3
    pp = np.zeros(om.cell_shape)
    pp[k, j, i] = DP
    om.set_field(oracle_mod.F_PP, 1, pp)
    om.step(1)
    w = C4 / 16.0 * DP
    e = np.zeros(om.cell_shape)
    e[k, j, i] = DP - 12.0 * w + (-8.0 if k == 5 else -6.0) * w
    _in_layer(e, (k, j, i), DP, horizontal=("y",))
    for dk, c in ((-2, -1.0), (-1, 4.0), (1, 4.0), (2, -1.0)):
        e[k + dk, j, i] += c * w
    e[k, j, 3] += -1.0 * w
    e[k, j, 4] += 4.0 * w
    e[k, j, 6] += 4.0 * w
    if k == 5:
        e[k, j, 7] += 4.0 * w  # member of the group hosted by (6, 3, 5)
    got = om.field(oracle_mod.F_PP)
    assert np.max(np.abs(got - e)) <= 1e-6 * w
    if k == 10:
        assert abs(got[k, j, 7]) <= 1e-6 * w


@pytest.mark.parametrize("K", [5, 18], ids=["beside-the-plateau", "above-the-plateau"])
def test_momentum_diffusion_next_to_ramp(oracle_mod, K):
    """x-momentum impulse at corner (6, 3, K).  At K = 5 the corner (8, 3, 5)
    lies below the plateau (800 m), so x takes the second order (-8 w);
    (7, 3, 5) lies above the flat floor and is a fluid point, so corner 5
    keeps the fourth order.  At K = 18 every corner of the x stencil is above
    the plateau: fourth order everywhere."""
    cfg, om = _ramp(oracle_mod)
    gz = om.gz
    I, J = 6, 3
    mx = np.zeros(om.corner_shape)
    mx[K + gz, J, I] = DM
    om.set_field(oracle_mod.F_MX, 1, mx)
    om.step(1)
    w = C4 / 16.0 * DM
    e = np.zeros(om.corner_shape)
    e[K + gz, J, I] = DM - 12.0 * w + (-8.0 if K == 5 else -6.0) * w
    _in_layer(e, (K + gz, J, I), DM, horizontal=("y",))
    for dk, c in ((-2, -1.0), (-1, 4.0), (1, 4.0), (2, -1.0)):
        e[K + dk + gz, J, I] += c * w
    for di, c in ((-2, -1.0), (-1, 4.0), (1, 4.0), (2, -1.0)):
        e[K + gz, J, I + di] += c * w
    pts = om.points()["vcls"]
    pred = pts == oracle_mod.V_PRED
    if K == 5:
        assert not pred[K + gz, J, 7] and not pred[K + gz, J, 8]
    else:
        assert pred[K + gz, J, 7] and pred[K + gz, J, 8]
    got = om.field(oracle_mod.F_MX)
    assert np.max(np.abs(got[pred] - e[pred])) <= 1e-6 * w
