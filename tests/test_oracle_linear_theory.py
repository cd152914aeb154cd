"""The oracle against linear mountain-wave theory (paper Sec 3.1.1: the flow
over a small bell-shaped hill agrees with the linear theory of Smith 1980).

A 20 m bell of half-width 2 km on 400 m cells (a = 5 cells, as in the paper's
1 km / 200 m test), U = 10 m/s, N = 0.01 1/s, run for 800 s from rest
relative to the uniform flow.  The vertical velocity at z = 1.6 km is
compared with the steady linear solution on the same periodic domain
(tests/linear_theory.py).  Tolerances: the remaining differences are the
transient still leaving the domain at 800 s, second-order truncation at five
cells per half-width, and the reflection from the lid and sponge; measured
0.33 (relative L2) and 0.95 (correlation), bounds set with margin.  A missing
or reversed buoyancy, pressure gradient or advection term gives a different
wave pattern (potential flow or the wrong phase) and fails both."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

import linear_theory as LT


def test_linear_solution_single_mode_and_surface_condition():
    """The helper itself: one Fourier mode propagates as cos(k x + m z)
    (phase lines tilting upstream with height, energy upward) and the surface
    vertical velocity is U dh/dx."""
    nx, ny, d = 64, 4, 250.0
    Lx = nx * d
    x = np.arange(nx) * d
    k = 2 * np.pi / Lx  # below N/U: a propagating mode
    h = np.tile(10.0 * np.cos(k * x), (ny, 1))
    U, N, z = 10.0, 0.01, 700.0
    w = LT.vertical_velocity(h, d, d, U, N, z)
    m = np.sqrt(N * N / (U * U) - k * k)
    expect = -U * 10.0 * k * np.sin(k * x + m * z)
    assert np.max(np.abs(w[0] - expect)) < 1e-9 * np.abs(expect).max()
    w0 = LT.vertical_velocity(h, d, d, U, N, 0.0)
    assert np.max(np.abs(w0[0] - (-U * 10.0 * k * np.sin(k * x)))) < 1e-9


@pytest.mark.timeout(300)
def test_oracle_bell_hill_matches_linear_theory(oracle_mod):
    d, a = 400.0, 2000.0
    cfg = W.RunConfig("linear-bell", 40, 24, 16, d, d, d, 0.4, 0, "bell", 20.0, a)
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(2000)  # 800 s
    rb, pb, koff = om.base()
    K = 4
    rc = 0.5 * (rb[K - 1 + koff] + rb[K + koff])
    r0 = 0.5 * (rb[-1 + koff] + rb[koff])
    wm = om.field(oracle_mod.F_MZ)[K + 2] / rc  # corner level K (host levels start at -2)
    wl = LT.vertical_velocity(cfg.heights(), d, d, cfg.U, cfg.N, K * d, r0 / rc)
    l2 = np.sqrt(((wm - wl) ** 2).sum() / (wl ** 2).sum())
    corr = (wm * wl).sum() / np.sqrt((wm ** 2).sum() * (wl ** 2).sum())
    assert l2 <= 0.45 and corr >= 0.92, (l2, corr)
    assert 0.8 <= np.abs(wm).max() / np.abs(wl).max() <= 1.2
