"""Derived output fields (corner velocity, potential-temperature
perturbation), the heat content and the analytic terrain on the GPU against
the FP64 oracle and the input generator, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def gpu_model(cc, cfgs, prec):
    cfgs = cfgs if isinstance(cfgs, list) else [cfgs]
    m = cc.Model(cfgs, prec)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    return m


def _atol(cc, which, cfg):
    """theta' is the difference of two values near theta0: the oracle forms
    it directly, so it carries a few ulp of theta0."""
    return 16 * np.finfo(float).eps * cfg.theta0 if which == cc.CC_THETA_P else 0.0


def _heat_tol(cfg, nx, ny, nz, dx, dy, dz):
    """Each cell's (rho theta)' is a difference of two values of the
    equation of state near rho_theta_bar; the two sides' powers may differ by
    an ulp or two, so the sums may differ by up to a few ulp of rho_theta_bar
    times the volume (rho_theta_bar is largest at the surface)."""
    cvcp = (cfg.cp - cfg.R) / cfg.cp
    rth_s = cfg.p0 / cfg.R * (cfg.p_surf / cfg.p0) ** cvcp
    return 4 * np.finfo(float).eps * rth_s * nx * ny * nz * dx * dy * dz


def _pairs(cc, om):
    return [(cc.CC_U, om.D_U), (cc.CC_V, om.D_V), (cc.CC_W, om.D_W), (cc.CC_THETA_P, om.D_THETA)]


@pytest.mark.parametrize("cfg,steps", [(W.SMALL_HEMI, 20), (W.C1_BELL, 30)], ids=["hemisphere", "bell"])
def test_fp64_derived_fields_and_heat_match_oracle(cc, oracle_mod, cfg, steps):
    om = oracle_mod.Model(cfg)
    om.init_state()
    m = gpu_model(cc, cfg, cc.CC_FP64)
    m.init_state()
    assert m.diagnostics(0)["heat"] == 0.0 and om.heat() == 0.0
    om.step(steps)
    m.step(steps)
    for fg, fo in _pairs(cc, oracle_mod):
        for lev in ((0, 1) if fg == cc.CC_THETA_P else (1,)):
            a, b = m.derived(0, fg, lev), om.derived(fo, lev)
            assert a.shape == b.shape
            scale = np.abs(b).max()
            assert scale > 0, (fg, lev)
            assert np.abs(a - b).max() <= 1e-9 * scale + _atol(cc, fg, cfg), (fg, lev)
    hg, ho = m.diagnostics(0)["heat"], om.heat()
    assert ho != 0.0
    tol = _heat_tol(cfg, cfg.nx, cfg.ny, cfg.nz, cfg.dx, cfg.dy, cfg.dz)
    assert tol < 1e-3 * abs(ho)
    assert abs(hg - ho) <= tol, (hg, ho, tol)
    m.close()


def test_fp32_derived_fields_and_heat_against_oracle(cc, oracle_mod):
    cfg = W.SMALL_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(20)
    m = gpu_model(cc, cfg, cc.CC_FP32)
    m.init_state()
    assert m.diagnostics(0)["heat"] == 0.0
    m.step(20)
    for fg, fo in _pairs(cc, oracle_mod):
        a, b = m.derived(0, fg), om.derived(fo)
        l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert l2 <= 2e-3, (fg, l2)
    hg, ho = m.diagnostics(0)["heat"], om.heat()
    assert abs(hg - ho) <= 2e-3 * abs(ho), (hg, ho)
    m.close()


def test_derived_on_refined_levels(cc, oracle_mod):
    rc = W.SMALL_REFINED
    R = oracle_mod.Refine(rc.base, rc.boxes, rc.finest_heights(pad=4))
    R.init_state()
    R.step(2)
    m = cc.RefinedModel(rc.base, rc.boxes, cc.CC_FP64)
    for l, c in enumerate(m.cfgs):
        m.set_terrain(l, rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx)))
    m.build_geometry()
    m.init_state()
    m.step(2)
    for l, lev in enumerate(R.levels):
        for fg, fo in _pairs(cc, oracle_mod):
            a, b = m.derived(l, fg), lev.derived(fo)
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= 1e-9 * scale + _atol(cc, fg, rc.base), (l, fg)
        hg, ho = m.diagnostics(l)["heat"], lev.heat()
        c = m.cfgs[l]
        assert abs(hg - ho) <= _heat_tol(rc.base, c.nx, c.ny, c.nz, c.dx, c.dy, c.dz), (l, hg, ho)
    m.close()


def test_derived_errors(cc):
    m = gpu_model(cc, W.SMALL_HEMI, cc.CC_FP32)
    with pytest.raises(cc.CutcellError) as e:
        m.derived(0, cc.CC_U)
    assert e.value.status == cc.CC_ESTATE
    m.init_state()
    for d, which, lev in ((1, cc.CC_U, 1), (0, 4, 1), (0, cc.CC_W, 2), (0, cc.CC_V, 0)):
        out = np.zeros((W.SMALL_HEMI.nz + 1, W.SMALL_HEMI.ny, W.SMALL_HEMI.nx))
        st = m.L.cc_download_derived(m.h, d, which, lev, out.ctypes.data)
        assert st == cc.CC_EINVAL
    m.close()


HILLS = [W.C1_BELL, W.SMALL_HEMI, W.C1_BELL.replace(name="cosine-32x32x24", terrain="cosine", h0=300.0, a=1500.0),
         W.SMALL_HEMI.replace(name="ellipsoid-40x36x24", terrain="ellipsoid", h0=250.0, a=600.0)]


def test_analytic_terrain_matches_generator_and_geometry(cc, oracle_mod):
    """The hill evaluated on the GPU equals the input generator's heights to
    a few ulp, and the geometry built on it equals the oracle's on the same
    heights, for an ensemble with one domain per hill shape."""
    m = cc.Model(HILLS, cc.CC_FP64)
    for d, c in enumerate(HILLS):
        m.set_terrain_analytic(d, c.terrain, c.h0, c.a)
    for d, c in enumerate(HILLS):
        h = m.terrain(d)
        ref = c.heights()
        assert np.max(np.abs(h - ref)) <= 8 * np.finfo(float).eps * c.h0, c.name
        assert (h > 0).sum() == (ref > 0).sum()
    m.build_geometry()
    for d, c in enumerate(HILLS):
        om = oracle_mod.Model(c, m.terrain(d))
        og, g = om.geometry(), m.geometry(d)
        assert np.array_equal(g["cls"], og["cls"]), c.name
        assert np.array_equal(g["root"], og["root"]), c.name
        assert np.max(np.abs(g["vf"] - og["vf"])) <= 1e-14
    m.init_state()
    m.step(3)
    assert all(m.diagnostics(d)["nonfinite"] == 0 for d in range(len(HILLS)))
    m.close()


def test_analytic_terrain_errors(cc):
    c = W.SMALL_HEMI
    m = cc.Model([c], cc.CC_FP64)
    with pytest.raises(cc.CutcellError) as e:
        m.terrain(0)
    assert e.value.status == cc.CC_ESTATE
    for kind, h0, a in ((7, 100.0, 100.0), (cc.CC_HILL_BELL, -1.0, 100.0), (cc.CC_HILL_BELL, 100.0, 0.0),
                        (cc.CC_HILL_BELL, float("nan"), 100.0), (cc.CC_HILL_ELLIPSOID, 5000.0, 400.0)):
        with pytest.raises(cc.CutcellError) as e:
            m.set_terrain_analytic(0, kind, h0, a)
        assert e.value.status == cc.CC_EINVAL
    with pytest.raises(cc.CutcellError) as e:
        m.build_geometry()  # the failed hill left no terrain
    assert e.value.status == cc.CC_ESTATE
    m.close()
    rc = W.SMALL_REFINED
    r = cc.RefinedModel(rc.base, rc.boxes, cc.CC_FP64)
    fine = r.cfgs[-1]
    with pytest.raises(cc.CutcellError) as e:  # a hill reaching the box edges
        r.set_terrain_analytic(r.nlev - 1, "bell", 50.0, fine.nx * fine.dx)
    assert e.value.status == cc.CC_EINVAL
    r.close()


def _pair_cfgs(coarse_d=400.0, nx=20, ny=16, nz=10, T=60.0):
    base = W.RunConfig("cosine", nx, ny, nz, coarse_d, coarse_d, coarse_d, 0.15 * coarse_d / 200.0, 1, "cosine",
                       300.0, 1600.0)
    fine = base.replace(name="cosine-fine", nx=2 * nx, ny=2 * ny, nz=2 * nz, dx=coarse_d / 2, dy=coarse_d / 2,
                        dz=coarse_d / 2, dt=base.dt / 2)
    return base, fine, int(round(T / base.dt))


def test_error_norms_match_oracle(cc, oracle_mod):
    """L1 / L2 norms of u, v, w of a 400 m cosine-hill run against the 200 m
    run at the same time, above the hill top: GPU (FP64 and FP32 coarse
    models) against the oracle's norms of the oracle's runs."""
    a_cfg, b_cfg, n = _pair_cfgs()
    oa, ob = oracle_mod.Model(a_cfg), oracle_mod.Model(b_cfg)
    oa.init_state()
    ob.init_state()
    oa.step(n)
    ob.step(2 * n)
    b = gpu_model(cc, b_cfg, cc.CC_FP64)
    b.init_state()
    b.step(2 * n)
    for prec, tol in ((cc.CC_FP64, 1e-9), (cc.CC_FP32, 2e-3)):
        a = gpu_model(cc, a_cfg, prec)
        a.init_state()
        a.step(n)
        for wg, wo in ((cc.CC_U, oracle_mod.D_U), (cc.CC_V, oracle_mod.D_V), (cc.CC_W, oracle_mod.D_W)):
            l1, l2, cnt = cc.error_norms(a, 0, b, 0, wg, a_cfg.h0)
            r1, r2, rn = oracle_mod.error_norms(oa, ob, wo, a_cfg.h0)
            assert cnt == rn == a_cfg.nx * a_cfg.ny * (a_cfg.nz - 0)
            assert r1 > 0 and r2 > 0
            assert abs(l1 - r1) <= tol * r1 and abs(l2 - r2) <= tol * r2, (prec, wg, l1, r1, l2, r2)
        assert cc.error_norms(a, 0, a, 0, cc.CC_W)[:2] == (0.0, 0.0)
        a.close()
    with pytest.raises(cc.CutcellError) as e:
        cc.error_norms(b, 0, b.__class__([a_cfg], cc.CC_FP64), 0, cc.CC_U)  # coarser, not finer
    assert e.value.status in (cc.CC_EINVAL, cc.CC_ESTATE)
    b.close()


def test_cosine_hill_errors_fall_with_resolution(cc):
    """The appendix accuracy experiment at reduced size: the cosine hill
    (h_m = 400 m, a = 2 km) on a 16 x 16 x 8 km periodic domain at 400, 200
    and 100 m (FP32, hills evaluated on the GPU), 1200 s of flow; the L1 and
    L2 errors of u and w above the hill top against the 100 m run fall from
    400 m to 200 m by at least a factor 1.5 (measured: 2.2 - 3.0)."""
    runs = {}
    for d in (400.0, 200.0, 100.0):
        n = int(16000 / d)
        cfg = W.RunConfig(f"cosine-{d:g}m", n, n, n // 2, d, d, d, 0.15 * d / 200.0, 1, "cosine", 400.0, 2000.0)
        m = cc.Model([cfg], cc.CC_FP32)
        m.set_terrain_analytic(0, "cosine", cfg.h0, cfg.a)
        m.build_geometry()
        m.init_state()
        m.step(int(round(1200.0 / cfg.dt)))
        assert m.diagnostics(0)["nonfinite"] == 0
        runs[d] = m
    for w in (cc.CC_U, cc.CC_W):
        e4 = cc.error_norms(runs[400.0], 0, runs[100.0], 0, w, 400.0)
        e2 = cc.error_norms(runs[200.0], 0, runs[100.0], 0, w, 400.0)
        assert e4[2] == 40 * 40 * 19 and e2[2] == 80 * 80 * 38
        for k in (0, 1):
            assert e4[k] >= 1.5 * e2[k] > 0, (w, k, e4, e2)
    for m in runs.values():
        m.close()


def test_error_norms_at_a_rational_ratio_match_oracle(cc, oracle_mod):
    """250 m against 100 m (the appendix's 250 m run): the norms over the
    corners the grids share (every 500 m) equal the oracle's."""
    a_cfg = W.RunConfig("cosine-250m", 16, 12, 8, 250.0, 250.0, 250.0, 0.1875, 1, "cosine", 300.0, 1200.0)
    b_cfg = a_cfg.replace(name="cosine-100m", nx=40, ny=30, nz=20, dx=100.0, dy=100.0, dz=100.0, dt=0.075)
    oa, ob = oracle_mod.Model(a_cfg), oracle_mod.Model(b_cfg)
    oa.init_state()
    ob.init_state()
    oa.step(160)
    ob.step(400)
    a, b = gpu_model(cc, a_cfg, cc.CC_FP64), gpu_model(cc, b_cfg, cc.CC_FP64)
    a.init_state()
    b.init_state()
    a.step(160)
    b.step(400)
    for wg, wo in ((cc.CC_U, oracle_mod.D_U), (cc.CC_W, oracle_mod.D_W)):
        l1, l2, n = cc.error_norms(a, 0, b, 0, wg, a_cfg.h0)
        r1, r2, rn = oracle_mod.error_norms(oa, ob, wo, a_cfg.h0)
        assert n == rn == 8 * 6 * 4  # corners K = 2, 4, 6, 8 lie above 300 m
        assert abs(l1 - r1) <= 1e-9 * r1 and abs(l2 - r2) <= 1e-9 * r2, (wg, l1, r1, l2, r2)
    a.close()
    b.close()


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_diagnostics_repeat_bit_for_bit(cc, prec_name):
    """The conservation sums (Neumaier per thread, fixed-order warp-shuffle
    TwoSum trees over fixed blocks) do not depend on scheduling: two models
    stepped alike report the same bits, and so does a second call on one."""
    prec = cc.CC_FP64 if prec_name == "fp64" else cc.CC_FP32
    cfgs = [W.SMALL_HEMI, W.C1_BELL]
    out = []
    for _ in range(2):
        m = gpu_model(cc, cfgs, prec)
        m.init_state()
        m.step(12)
        out.append([m.diagnostics(d) for d in range(2)])
        out.append([m.diagnostics(d) for d in range(2)])
        m.close()
    for run in out[1:]:
        for d in range(2):
            for key in ("mass", "mass_comp", "heat", "heat_comp", "max_u", "max_w"):
                assert run[d][key] == out[0][d][key], (d, key)
    assert out[0][0]["max_u"] > 0.0
