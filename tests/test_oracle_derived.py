"""Pins of the oracle's derived output fields (corner velocity, potential
temperature perturbation) and heat content against closed forms: the base
state's potential temperature theta0 exp(N^2 z / g) (Sec 3), the equation of
state rho theta = (p0/R)(p/p0)^(cv/cp) (Sec 2.1) and known momentum fields."""
import math

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W


def _flat(nx=8, ny=6, nz=10, d=100.0, **kw):
    return W.RunConfig("flat", nx, ny, nz, d, d, d, 0.1, 1, "flat", 0.0, 1.0, **kw)


def theta_bar(cfg, k):
    """Base potential temperature at the centre of cell level k."""
    z = (np.asarray(k) + 0.5) * cfg.dz
    return cfg.theta0 * np.exp(cfg.N ** 2 * z / cfg.g)


def _levels(om):
    rhob, pb, koff = om.base()
    nz = om.cfg.nz
    return rhob, pb, koff, np.arange(nz)


def test_theta_prime_zero_at_rest(oracle_mod):
    om = oracle_mod.Model(W.SMALL_HEMI)
    om.init_state()
    assert np.array_equal(om.derived(oracle_mod.D_THETA), np.zeros(om.cell_shape))


def test_theta_prime_of_density_perturbation(oracle_mod):
    """Unchanged pressure (so unchanged rho theta) and rho' = -eps rho_bar give
    theta = theta_bar / (1 - eps), i.e. theta' = theta_bar eps / (1 - eps),
    with eps different in every cell."""
    cfg = _flat()
    om = oracle_mod.Model(cfg)
    om.init_state()
    rhob, pb, koff, ks = _levels(om)
    nz, ny, nx = om.cell_shape
    idx = np.arange(nz * ny * nx).reshape(om.cell_shape)
    eps = 1e-3 * (1 + (idx * 7919) % 37) / 37.0
    rp = -eps * rhob[ks + koff][:, None, None]
    om.set_field(oracle_mod.F_RHOP, 1, rp)
    got = om.derived(oracle_mod.D_THETA)
    want = theta_bar(cfg, ks)[:, None, None] * eps / (1 - eps)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-9


def test_theta_prime_of_pressure_perturbation(oracle_mod):
    """rho' = 0 and p' = delta p_bar give theta' = theta_bar ((1+delta)^(cv/cp) - 1);
    delta differs from cell to cell and changes sign."""
    cfg = _flat()
    om = oracle_mod.Model(cfg)
    om.init_state()
    rhob, pb, koff, ks = _levels(om)
    nz, ny, nx = om.cell_shape
    idx = np.arange(nz * ny * nx).reshape(om.cell_shape)
    delta = 2e-3 * (((idx * 104729) % 41) / 20.0 - 1.0)
    delta[delta == 0] = 1e-4
    om.set_field(oracle_mod.F_PP, 1, delta * pb[ks + koff][:, None, None])
    got = om.derived(oracle_mod.D_THETA)
    cvcp = (cfg.cp - cfg.R) / cfg.cp
    want = theta_bar(cfg, ks)[:, None, None] * np.expm1(cvcp * np.log1p(delta))
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-8
    # the time level is honoured: the filtered previous level is still at rest
    assert np.array_equal(om.derived(oracle_mod.D_THETA, 0), np.zeros(om.cell_shape))


def test_corner_velocity_of_known_momentum(oracle_mod):
    """Over a flat floor at zero height the corners K >= 1 hold momentum /
    corner density, the corner density being the mean of the two cell levels
    around the corner (all eight cells at base density); corners K = 0 (on the
    terrain) give the boundary-point velocity of their column."""
    cfg = _flat()
    om = oracle_mod.Model(cfg)
    om.init_state()
    rhob, pb, koff, _ = _levels(om)
    nz, ny, nx = om.cell_shape
    gz = om.gz
    K = np.arange(-gz, nz + gz + 1)
    rc = 0.5 * (rhob[K - 1 + koff] + rhob[K + koff])
    I = np.arange(nx)[None, None, :]
    J = np.arange(ny)[None, :, None]
    KK = K[:, None, None]
    want = [1.0 + I + 100.0 * J + 1e4 * KK, -2.0 * I + 0.5 * J, 0.01 * (I + J + KK)]
    for f, w in zip((oracle_mod.F_MX, oracle_mod.F_MY, oracle_mod.F_MZ), want):
        om.set_field(f, 1, rc[:, None, None] * (w + 0.0 * KK * I * J))
    ub = np.stack([np.full((ny, nx), 3.0), 0.25 * np.arange(nx)[None, :] + 0 * J[0], -0.5 + 0 * I[0] * J[0]], -1)
    om.set_field(oracle_mod.F_UB, 1, ub)
    for c, which in enumerate((oracle_mod.D_U, oracle_mod.D_V, oracle_mod.D_W)):
        got = om.derived(which)
        assert got.shape == (nz + 1, ny, nx)
        w = np.broadcast_to(want[c], (len(K), ny, nx))[gz:gz + nz + 1]
        np.testing.assert_allclose(got[1:], w[1:], rtol=1e-13, atol=1e-13)
        assert np.array_equal(got[0], ub[:, :, c])
        with pytest.raises(oracle_mod.OracleError):
            om.derived(which, 0)  # the boundary velocity exists for the current level only


def test_corner_velocity_of_initial_state_over_a_hill(oracle_mod):
    """The initial state over the bell hill: uniform wind U on the predicted
    corners, the free-slip boundary velocity (tangential) on corners at or
    below the terrain, and v = w = 0 away from the terrain."""
    cfg = W.C1_BELL
    om = oracle_mod.Model(cfg)
    om.init_state()
    pts = om.points()
    gz = om.gz
    vcls = pts["vcls"][gz:gz + cfg.nz + 1]
    u, v, w = (om.derived(x) for x in (oracle_mod.D_U, oracle_mod.D_V, oracle_mod.D_W))
    pred = vcls == oracle_mod.V_PRED
    assert np.max(np.abs(u[pred] - cfg.U)) <= 4e-16 * cfg.U * 4
    assert np.max(np.abs(v[pred])) == 0.0 and np.max(np.abs(w[pred])) == 0.0
    h = cfg.heights()
    K = np.arange(cfg.nz + 1)[:, None, None]
    below = K * cfg.dz <= h[None]
    n = pts["bn"]
    un = u * n[None, :, :, 0] + v * n[None, :, :, 1] + w * n[None, :, :, 2]
    assert below.any()
    assert np.max(np.abs(un[below])) < 1e-12 * cfg.U
    assert np.all(np.abs(u[below]) > 0.5 * cfg.U)  # free slip keeps the wind along the surface


def test_heat_closed_form_flat(oracle_mod):
    """p' = delta_k p_bar over a flat floor: the heat content is the sum over
    cells of V rho_bar theta_bar ((1 + delta_k)^(cv/cp) - 1), with
    rho_bar theta_bar the base state's own product."""
    cfg = _flat(nz=12)
    om = oracle_mod.Model(cfg)
    om.init_state()
    assert om.heat() == 0.0
    rhob, pb, koff, ks = _levels(om)
    delta = 1e-3 * (1.0 + 0.37 * ks) * np.where(ks % 3 == 1, -1.0, 1.0)
    pp = np.broadcast_to((delta * pb[ks + koff])[:, None, None], om.cell_shape)
    om.set_field(oracle_mod.F_PP, 1, pp)
    cvcp = (cfg.cp - cfg.R) / cfg.cp
    V = cfg.dx * cfg.dy * cfg.dz
    want = V * cfg.nx * cfg.ny * np.sum(rhob[ks + koff] * theta_bar(cfg, ks) * np.expm1(cvcp * np.log1p(delta)))
    assert abs(om.heat() - want) <= 1e-9 * abs(want)
    assert om.heat(0) == 0.0


def test_heat_over_a_hill_uses_merged_volumes(oracle_mod):
    """Over the hemisphere with a uniform relative pressure perturbation, the
    heat content is the sum over merge groups of V_G rho_bar theta_bar
    ((1+delta)^(cv/cp) - 1) at the host cell's level."""
    cfg = W.SMALL_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    g = om.geometry()
    rhob, pb, koff, ks = _levels(om)
    delta = 5e-4
    pp = np.broadcast_to((delta * pb[ks + koff])[:, None, None], om.cell_shape).copy()
    om.set_field(oracle_mod.F_PP, 1, pp)
    nz, ny, nx = om.cell_shape
    ids = np.arange(nz * ny * nx).reshape(om.cell_shape)
    host = (g["root"] == ids) & (g["cls"] != oracle_mod.C_UG)
    kk = np.broadcast_to(ks[:, None, None], om.cell_shape)
    cvcp = (cfg.cp - cfg.R) / cfg.cp
    want = np.sum(g["vg"][host] * rhob[kk[host] + koff] * theta_bar(cfg, kk[host])) * math.expm1(cvcp * math.log1p(delta))
    assert abs(om.heat() - want) <= 1e-9 * abs(want)
    # merging moves volume between cells but keeps the fluid volume
    assert abs(np.sum(g["vg"][host]) - np.sum(g["vf"]) * cfg.dx * cfg.dy * cfg.dz) <= 1e-9 * np.sum(g["vg"][host])


def _set_u(oracle_mod, om, fu):
    """Momentum rho_c * fu(I, J, K) on every corner level of a flat-floor
    model at rest density (rho_c = mean base density of the levels K-1, K)."""
    rhob, pb, koff, _ = _levels(om)
    nz, ny, nx = om.cell_shape
    K = np.arange(-om.gz, nz + om.gz + 1)
    rc = 0.5 * (rhob[K - 1 + koff] + rhob[K + koff])
    I = np.arange(nx)[None, None, :]
    J = np.arange(ny)[None, :, None]
    om.set_field(oracle_mod.F_MX, 1, rc[:, None, None] * fu(I, J, K[:, None, None]))


def test_error_norms_of_a_known_difference(oracle_mod):
    """The appendix's L1 and L2 norms: a coarse model holding u = U and a
    model refined by 2 holding U + delta at the coincident corners give the
    mean of |delta| and the root mean square of delta over the coarse
    corners above zmin; equal fields give zero."""
    a = oracle_mod.Model(_flat(8, 6, 10, 200.0))
    b = oracle_mod.Model(_flat(16, 12, 20, 100.0))
    a.init_state()
    b.init_state()
    U = 7.0
    _set_u(oracle_mod, a, lambda I, J, K: U + 0.0 * (I + J + K))
    _set_u(oracle_mod, b, lambda I, J, K: U + 0.0 * (I + J + K))
    l1, l2, n = oracle_mod.error_norms(a, b, oracle_mod.D_U, 250.0)
    assert n == 8 * 6 * 9  # corner levels K = 2 .. 10 lie above 250 m
    assert l1 <= 4e-16 * U and l2 <= 4e-16 * U
    assert oracle_mod.error_norms(a, b, oracle_mod.D_W, 250.0)[:2] == (0.0, 0.0)

    def delta(I, J, K):
        return 1e-2 * np.sin(0.7 * I + 1.3 * J) * np.cos(0.4 * K) + 1e-3 * (I % 3)

    _set_u(oracle_mod, b, lambda I, J, K: U + delta(I, J, K))
    Ia, Ja, Ka = np.meshgrid(np.arange(8), np.arange(6), np.arange(2, 11), indexing="ij")
    d = delta(2 * Ia, 2 * Ja, 2 * Ka)
    l1, l2, n = oracle_mod.error_norms(a, b, oracle_mod.D_U, 250.0)
    assert n == d.size
    assert abs(l1 - np.mean(np.abs(d))) <= 1e-12 * np.mean(np.abs(d))
    assert abs(l2 - np.sqrt(np.mean(d ** 2))) <= 1e-12 * np.sqrt(np.mean(d ** 2))
    # every level above the floor when zmin is below it
    assert oracle_mod.error_norms(a, b, oracle_mod.D_U, -1.0)[2] == 8 * 6 * 11


def test_error_norms_reject_incommensurate_grids(oracle_mod):
    a = oracle_mod.Model(_flat(8, 6, 10, 200.0))
    for b in (oracle_mod.Model(_flat(12, 9, 15, 133.33)), oracle_mod.Model(_flat(16, 12, 18, 100.0))):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.error_norms(a, b, oracle_mod.D_U, 0.0)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.error_norms(a, a, oracle_mod.D_THETA, 0.0)


def test_error_norms_at_a_rational_ratio(oracle_mod):
    """Spacings in the ratio 5/2 (250 m against 100 m, as in the appendix):
    only every second coarse corner coincides with a fine corner (every
    500 m), and the norms are taken over those."""
    a = oracle_mod.Model(_flat(8, 6, 10, 250.0))
    b = oracle_mod.Model(_flat(20, 15, 25, 100.0))
    a.init_state()
    b.init_state()
    U = 5.0
    _set_u(oracle_mod, a, lambda I, J, K: U + 0.0 * (I + J + K))

    def delta(I, J, K):
        return 1e-2 * np.cos(0.3 * I - 0.2 * J) * (1.0 + 0.1 * K)

    _set_u(oracle_mod, b, lambda I, J, K: U + delta(I, J, K))
    Ia, Ja, Ka = np.meshgrid(np.arange(0, 8, 2), np.arange(0, 6, 2), np.arange(2, 11, 2), indexing="ij")
    d = delta(Ia // 2 * 5, Ja // 2 * 5, Ka // 2 * 5)
    l1, l2, n = oracle_mod.error_norms(a, b, oracle_mod.D_U, 300.0)  # K dz > 300 m: K = 2, 4, .., 10
    assert n == d.size == 4 * 3 * 5
    assert abs(l1 - np.mean(np.abs(d))) <= 1e-12 * np.mean(np.abs(d))
    assert abs(l2 - np.sqrt(np.mean(d ** 2))) <= 1e-12 * np.sqrt(np.mean(d ** 2))
