"""Block-structured refinement on the GPU (Sec 2.2) against the FP64 oracle,
through the C ABI: per-level geometry, subcycled steps with the coarse-fine
ghost fill, restriction and flux register, rest state and conservation
(needs a GB300)."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RC = W.SMALL_REFINED


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def gpu_refined(cc, rc, prec=None, **kw):
    base = rc.base.replace(**kw) if kw else rc.base
    m = cc.RefinedModel(base, rc.boxes, cc.CC_FP64 if prec is None else prec)
    for l, c in enumerate(m.cfgs):
        h = rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx))
        m.set_terrain(l, h)
    m.build_geometry()
    return m


def oracle_refined(oracle_mod, rc, **kw):
    base = rc.base.replace(**kw) if kw else rc.base
    return oracle_mod.Refine(base, rc.boxes, rc.finest_heights(pad=4))


def _pairs(cc, oracle_mod):
    return [(cc.CC_RHOP, oracle_mod.F_RHOP), (cc.CC_PP, oracle_mod.F_PP), (cc.CC_MX, oracle_mod.F_MX),
            (cc.CC_MY, oracle_mod.F_MY), (cc.CC_MZ, oracle_mod.F_MZ), (cc.CC_UB, oracle_mod.F_UB)]


def _compare(cc, oracle_mod, m, R, rel_l2, rel_inf, report=False):
    """Per level, field and time level: L2 and max error relative to the
    field's L2 norm and largest magnitude over all levels (the coarse levels
    see the hill's disturbance only through restriction, so their own norms
    can be many orders below it)."""
    errs = {}
    for fg, fo in _pairs(cc, oracle_mod):
        for tl in ((1,) if fg == cc.CC_UB else (0, 1)):
            a = [m.download(l, fg, tl) for l in range(len(R.levels))]
            b = [lev.field(fo, tl) for lev in R.levels]
            scale = max(np.abs(x).max() for x in b)
            norm = np.sqrt(sum(np.sum(x ** 2) for x in b))
            for l in range(len(b)):
                if scale == 0.0:
                    assert np.abs(a[l]).max() == 0.0, (l, fg, tl)
                    continue
                l2 = np.sqrt(np.sum((a[l] - b[l]) ** 2)) / norm
                li = np.abs(a[l] - b[l]).max() / scale
                errs[(l, fg, tl)] = (l2, li)
                if not report:
                    assert l2 <= rel_l2 and li <= rel_inf, (l, fg, tl, l2, li)
    return errs


def test_level_geometry_bit_exact(cc, oracle_mod):
    """Every level's cell classes, merge roots, velocity-point classes and
    boundary stencils equal the oracle's, which evaluates the box levels over
    their padded terrain."""
    R = oracle_refined(oracle_mod, RC)
    m = gpu_refined(cc, RC)
    for l, lev in enumerate(R.levels):
        og, op = lev.geometry(), lev.points()
        g, s = m.geometry(l), m.stencils(l)
        assert np.array_equal(g["cls"], og["cls"]), l
        assert np.array_equal(g["root"], og["root"]), l
        assert np.array_equal(g["vcls"], op["vcls"]), l
        for k in ("bK", "bI", "bJ"):
            assert np.array_equal(s[k], op[k]), (l, k)
        for k in ("vf", "ax", "ay", "az"):
            assert np.max(np.abs(g[k] - og[k])) <= 1e-14, (l, k)
    assert (m.geometry(m.nlev - 1)["cls"] == 2).any()  # the hill is cut on the finest level
    m.close()


def test_fp64_refined_parity(cc, oracle_mod):
    """Three levels, each subcycled step against the oracle element by element
    on every level and both time levels."""
    R = oracle_refined(oracle_mod, RC)
    R.init_state()
    m = gpu_refined(cc, RC)
    m.init_state()
    _compare(cc, oracle_mod, m, R, 1e-13, 1e-11)
    R.step(1)
    m.step(1)
    _compare(cc, oracle_mod, m, R, 1e-12, 1e-10)
    R.step(4)
    m.step(4)
    _compare(cc, oracle_mod, m, R, 1e-10, 1e-8)
    m.close()


def test_refined_rest_state_exact(cc):
    for prec in (cc.CC_FP64, cc.CC_FP32):
        m = gpu_refined(cc, RC, prec, U=0.0)
        m.init_state()
        m.step(3)
        for l in range(m.nlev):
            for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ, cc.CC_UB):
                assert np.abs(m.download(l, f)).max() == 0.0, (prec, l, f)
        m.close()


def _flux_scale(rc):
    nx, ny, nz, ox, oy = rc.boxes[0]
    b = rc.base
    return 1.2 * b.U * (ny * b.dy / 2) * (nz * b.dz / 2) * 2 * b.dt


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_refined_mass_conserved_filter_off(cc, oracle_mod, prec, tol):
    """With the filter off, the two-time-level mass over the active cells of
    all levels is conserved to round-off on the GPU (the register makes the
    coarse flux through the box boundary the mean of the fine substeps), and
    its value follows the oracle's."""
    m = gpu_refined(cc, RC, cc.CC_FP64 if prec == "fp64" else cc.CC_FP32, ra_nu=0.0)
    m.init_state()
    m.step(1)
    q0 = m.mass()
    for _ in range(4):
        m.step(1)
        assert abs(m.mass() - q0) <= tol * _flux_scale(RC), (m.mass(), q0)
    if prec == "fp64":
        R = oracle_refined(oracle_mod, RC, ra_nu=0.0)
        R.init_state()
        R.step(5)
        assert abs(m.mass() - R.mass()) <= 1e-10 * _flux_scale(RC)
    m.close()


def test_fp32_refined_error_against_oracle(cc, oracle_mod):
    R = oracle_refined(oracle_mod, RC)
    R.init_state()
    R.step(6)
    m = gpu_refined(cc, RC, cc.CC_FP32)
    m.init_state()
    m.step(6)
    errs = _compare(cc, oracle_mod, m, R, 0, 0, report=True)
    for key, (l2, li) in errs.items():
        assert l2 <= 1e-3 and li <= 1e-2, (key, l2, li)
    m.close()


def test_full_size_refined_properties(cc):
    """The three-level 200/100/50 m hemisphere as the benchmark runs it (FP32):
    rest state exact, mass over the active cells conserved with the filter
    off, finite state with the filter on."""
    rc = W.C4_REFINED
    m = gpu_refined(cc, rc, cc.CC_FP32, ra_nu=0.0)
    m.init_state()
    m.step(1)
    q0 = m.mass()
    m.step(2)
    assert abs(m.mass() - q0) <= 2e-6 * _flux_scale(rc) * 4
    for l in range(m.nlev):
        d = m.diagnostics(l)
        assert d["nonfinite"] == 0
    m.close()


def test_refined_error_paths(cc):
    b = RC.base
    with pytest.raises(cc.CutcellError) as e:
        cc.RefinedModel(b, [(32, 32, 16, 15, 16)])  # odd offset
    assert e.value.status == cc.CC_EINVAL
    with pytest.raises(cc.CutcellError) as e:
        cc.RefinedModel(b, [(32, 32, 16, 2, 16)])  # covered box touches the coarse edge region
    assert e.value.status == cc.CC_EINVAL
    m = cc.RefinedModel(b, RC.boxes)
    h = np.zeros((32, 32))
    h[2, 2] = 10.0  # terrain near a box edge
    with pytest.raises(cc.CutcellError) as e:
        m.set_terrain(2, h)
    assert e.value.status == cc.CC_EINVAL
    hc = np.zeros((32, 32))
    hc[16, 16] = 5.0  # coarse terrain next to the covered box
    m.set_terrain(0, hc)
    m.set_terrain(1, np.zeros((32, 32)))
    m.set_terrain(2, RC.finest_heights())
    with pytest.raises(cc.CutcellError) as e:
        m.build_geometry()
    assert e.value.status == cc.CC_EGEOM
    m.close()


def test_refined_autotune_per_level_keeps_bits(cc):
    """Each level picks its own schedule; the result is the same bits as the
    default schedules."""
    m = gpu_refined(cc, RC, cc.CC_FP32)
    m.init_state()
    m.step(3)
    ref = [m.download(l, f) for l in range(m.nlev) for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX)]
    m.close()
    m = gpu_refined(cc, RC, cc.CC_FP32)
    m.init_state()
    m.step(1)
    sched = m.autotune(2)
    assert len(sched) == m.nlev and all(s[0] in (16, 8) for s in sched)
    m.step(2)
    out = [m.download(l, f) for l in range(m.nlev) for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX)]
    for x, y in zip(out, ref):
        assert np.array_equal(x, y)
    m.close()


def test_refined_graph_replay_equals_direct_launches(cc):
    outs = []
    for on in (False, True):
        m = gpu_refined(cc, RC, cc.CC_FP32)
        m.graphs(on)
        m.init_state()
        for _ in range(6):
            m.step(1)
        launches = m.last_launch_count
        outs.append([m.download(l, f) for l in range(m.nlev) for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MZ)])
        m.close()
        assert launches > 20
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


PAPER_BASE = W.RunConfig("hemisphere-400m", 160, 80, 40, 400.0, 400.0, 400.0, 0.3, 1, "hemisphere", 1000.0, 1000.0,
                         theta0=300.0)
# the regions behind the fine levels' inflow faces (m): x, y ranges and z < 3.2 km
INFLOW = {1: (16000.0, 22000.0, 8000.0, 24000.0), 2: (24000.0, 30000.0, 12000.0, 20000.0)}
TIMES = (1200, 2400, 3600)


def _max_w(w, dx, dz, x0, ox, oy, region):
    """Largest |w| at the corners of a level whose corner (0, 0) lies at
    (ox, oy) m, inside the region (x0 .. x1, y0 .. y1, z below 3.2 km)."""
    xa, xb, ya, yb = region
    nk, ny, nx = w.shape
    X, Y, Z = ox + np.arange(nx) * dx, oy + np.arange(ny) * dx, np.arange(nk) * dz
    sel = w[np.ix_(Z < 3200.0, (Y >= ya) & (Y <= yb), (X >= xa) & (X < xb))]
    return float(np.abs(sel).max())


@pytest.fixture(scope="module")
def uniform200(cc):
    """The uniform 200 m run of the same flow: largest |w| in the two regions
    at 1,200, 2,400 and 3,600 s."""
    u = PAPER_BASE.replace(nx=320, ny=160, nz=80, dx=200.0, dy=200.0, dz=200.0, dt=0.15)
    m = cc.Model([u], cc.CC_FP32)
    m.set_terrain(0, u.heights())
    m.build_geometry()
    m.init_state()
    out = {}
    for T in TIMES:
        m.step(8000)
        w = m.derived(0, cc.CC_W)
        out[T] = {l: _max_w(w, 200.0, 200.0, 0.0, 0.0, 0.0, INFLOW[l]) for l in (1, 2)}
    m.close()
    return out


# measured bounds on the largest |w| (m/s) behind the inflow faces, with some
# headroom: run (levels) -> level -> time -> bound
INFLOW_BOUND = {2: {1: {2400: 6.0, 3600: 18.0}},
                3: {1: {2400: 0.8, 3600: 1.0}, 2: {1200: 2.0, 2400: 2.6, 3600: 11.0}}}


@pytest.mark.timeout(900)
@pytest.mark.parametrize("nbox", [1, 2], ids=["two-levels", "three-levels"])
def test_refined_paper_domain_one_hour(cc, uniform200, nbox):
    """The 1 km hemisphere on the paper's 64 x 32 x 16 km domain at 400 m with
    a 200 m box (x 16-48 km, y 8-24 km, z 0-8 km) and, for three levels, a
    100 m box (x 24-40 km, y 12-20 km, z 0-4 km), FP32, one hour (12,000
    coarse steps).  Every level stays finite.  The largest |w| below 3.2 km in
    the 6 km behind each fine level's inflow face is compared with the uniform
    200 m run at the same points.  At 1,200 s the 200 m levels match it (two
    levels 0.12 against 0.12 m/s; three levels 0.02).  The open defect (a
    disturbance behind the fine inflow faces, still unexplained) then shows:
    at 2,400 s the two-level run reaches 4.2 m/s there against 0.014 for the uniform grid, about 300 times
    more, and 12.5 m/s at 3,600 s; in the three-level run the 200 m level
    reaches 0.52 m/s (about 37 times the uniform run) and the 100 m box,
    already at 1.3 against 0.48 m/s at 1,200 s, 7.3 m/s at 3,600 s.  The test
    asserts the 1,200 s agreement of the 200 m levels and bounds the rest at
    the measured values (so that the defect cannot grow unnoticed); it does
    not claim that the refined runs are right behind their inflow faces."""
    boxes = [(160, 80, 40, 80, 40)] * nbox
    rc = W.RefinedConfig("paper-domain", PAPER_BASE, boxes)
    m = cc.RefinedModel(PAPER_BASE, boxes, cc.CC_FP32)
    for l, c in enumerate(m.cfgs):
        m.set_terrain(l, rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx)))
    m.build_geometry()
    m.init_state()
    got = {}
    for T in TIMES:
        m.step(4000)
        for l in range(1, m.nlev):
            c = m.cfgs[l]
            ox, oy = rc.level_origin(l)
            got[(l, T)] = _max_w(m.derived(l, cc.CC_W), c.dx, c.dz, 0.0, ox, oy, INFLOW[l])
    ds = [m.diagnostics(l, check=False) for l in range(m.nlev)]
    m.close()
    for l, d in enumerate(ds):
        assert d["nonfinite"] == 0, l
        assert d["max_w"] < 20.0, (l, d["max_w"])
    # the 200 m level agrees with the uniform 200 m run at 1,200 s
    assert got[(1, 1200)] <= 1.5 * uniform200[1200][1] + 0.02, (got[(1, 1200)], uniform200[1200][1])
    for l, per in INFLOW_BOUND[nbox + 1].items():
        for T, bound in per.items():
            assert got[(l, T)] <= bound, (l, T, got[(l, T)], uniform200[T][l])
