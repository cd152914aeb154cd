"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GZ_HOST = 2


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def gpu_model(cc, cfgs, prec=None, heights=None):
    prec = cc.CC_FP64 if prec is None else prec
    cfgs = cfgs if isinstance(cfgs, list) else [cfgs]
    m = cc.Model(cfgs, prec)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights() if heights is None else heights[d])
    m.build_geometry()
    return m


def expected_groups(og):
    cls, root = og["cls"].ravel(), og["root"].ravel()
    sel = (cls == 2) | (cls == 3)
    hosts = np.unique(root[sel])
    start = [0]
    mem = []
    for h in hosts:
        mm = np.flatnonzero(root == h)
        mem.extend(mm.tolist())
        start.append(len(mem))
    return hosts.astype(np.int32), np.array(start, np.int32), np.array(mem, np.int32)


GEOM_CASES = [W.C1_BELL, W.SMALL_HEMI, W.C2_HEMI]


@pytest.mark.parametrize("cfg", GEOM_CASES, ids=lambda c: c.name)
def test_geometry_bit_exact(cc, oracle_mod, cfg):
    om = oracle_mod.Model(cfg)
    og, op = om.geometry(), om.points()
    m = gpu_model(cc, cfg)
    g, s = m.geometry(), m.stencils()
    # integer maps: bit-exact
    assert np.array_equal(g["cls"], og["cls"])
    assert np.array_equal(g["root"], og["root"])
    assert np.array_equal(g["vcls"], op["vcls"])
    for k in ("bK", "bI", "bJ"):
        assert np.array_equal(s[k], op[k]), k
    mf = op["vcls"] == 2
    assert np.array_equal(s["mK"][mf], op["mK"][mf])
    # compacted merge-group lists: bit-exact
    host, start, mem = m.groups()
    eh, es, em = expected_groups(og)
    assert np.array_equal(host, eh) and np.array_equal(start, es) and np.array_equal(mem, em)
    # volumes, apertures and stencil weights: same operations in the same order
    for k in ("vf", "ax", "ay", "az"):
        assert np.max(np.abs(g[k] - og[k])) <= 1e-14, k
    assert np.max(np.abs(s["ba"] - op["ba"])) <= 1e-14
    assert np.max(np.abs(s["bb"] - op["bb"])) <= 1e-14
    assert np.max(np.abs(s["bn"] - op["bn"])) <= 1e-15
    if mf.any():
        assert np.max(np.abs(s["mg"][mf] - op["mg"][mf])) <= 1e-14
    m.close()


FIELDS = None


def _compare(cc, oracle_mod, m, om, d=0, rel_l2=1e-10, rel_inf=1e-8, report=None):
    pairs = [(cc.CC_RHOP, oracle_mod.F_RHOP), (cc.CC_PP, oracle_mod.F_PP), (cc.CC_MX, oracle_mod.F_MX),
             (cc.CC_MY, oracle_mod.F_MY), (cc.CC_MZ, oracle_mod.F_MZ), (cc.CC_UB, oracle_mod.F_UB)]
    errs = {}
    for fg, fo in pairs:
        for level in ((1,) if fg == cc.CC_UB else (0, 1)):
            a = m.download(d, fg, level)
            b = om.field(fo, level)
            scale = np.abs(b).max()
            if scale == 0.0:
                assert np.abs(a).max() == 0.0, (fg, level)
                continue
            l2 = np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
            li = np.abs(a - b).max() / scale
            errs[(fg, level)] = (l2, li)
            if report is None:
                assert l2 <= rel_l2 and li <= rel_inf, (fg, level, l2, li)
    return errs


@pytest.mark.parametrize("cfg,steps", [(W.C1_BELL, 100), (W.SMALL_HEMI, 40),
                                       (W.SMALL_HEMI.replace(bc_slip=0, name="hemi-noslip"), 10)],
                         ids=["bell-100", "hemisphere-40", "hemisphere-noslip-10"])
def test_fp64_step_parity(cc, oracle_mod, cfg, steps):
    om = oracle_mod.Model(cfg)
    om.init_state()
    m = gpu_model(cc, cfg)
    m.init_state()
    _compare(cc, oracle_mod, m, om, rel_l2=1e-13, rel_inf=1e-11)  # initial diagnosis
    om.step(1)
    m.step(1)
    _compare(cc, oracle_mod, m, om, rel_l2=1e-12, rel_inf=1e-10)  # forward-Euler start
    om.step(steps - 1)
    m.step(steps - 1)
    _compare(cc, oracle_mod, m, om)
    m.close()


def test_fp64_parity_full_size_hemisphere(cc, oracle_mod):
    """The 128x128x64 hemisphere at full size (the benchmark's domain), as the
    benchmark launches it, a few steps against the oracle element by element."""
    cfg = W.C2_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    m = gpu_model(cc, cfg)
    m.init_state()
    om.step(4)
    m.step(4)
    _compare(cc, oracle_mod, m, om)
    m.close()


def test_upload_download_roundtrip_and_resume(cc, oracle_mod):
    """A state uploaded from the oracle continues exactly like the oracle."""
    cfg = W.SMALL_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(7)
    m = gpu_model(cc, cfg)
    m.init_state()
    m.step(1)  # leave the forward-Euler start behind
    for fg, fo in [(cc.CC_RHOP, oracle_mod.F_RHOP), (cc.CC_PP, oracle_mod.F_PP), (cc.CC_MX, oracle_mod.F_MX),
                   (cc.CC_MY, oracle_mod.F_MY), (cc.CC_MZ, oracle_mod.F_MZ)]:
        for level in (0, 1):
            a = om.field(fo, level)
            m.upload(0, fg, level, a)
            assert np.array_equal(m.download(0, fg, level), a)
    m.upload(0, cc.CC_UB, 1, om.field(oracle_mod.F_UB, 1))
    om.step(5)
    m.step(5)
    _compare(cc, oracle_mod, m, om)
    m.close()


def test_rest_state_exact_on_gpu(cc):
    cfg = W.SMALL_HEMI.replace(U=0.0)
    for prec in (cc.CC_FP64, cc.CC_FP32):
        m = gpu_model(cc, cfg, prec)
        m.init_state()
        m.step(20)
        for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ, cc.CC_UB):
            assert np.abs(m.download(0, f)).max() == 0.0, (prec, f)
        m.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_mass_conservation_on_gpu(cc, prec, tol):
    cfg = W.SMALL_HEMI
    m = gpu_model(cc, cfg, cc.CC_FP64 if prec == "fp64" else cc.CC_FP32)
    m.init_state()
    d0 = m.diagnostics()
    m.step(60)
    d1 = m.diagnostics()
    rp = m.download(0, cc.CC_RHOP)
    scale = np.abs(rp).max() * cfg.dx * cfg.dy * cfg.dz * cfg.cells
    assert abs(d1["mass"] - d0["mass"]) <= tol * scale, (d0, d1, scale)
    assert d1["nonfinite"] == 0 and d1["max_u"] > 5.0
    m.close()


@pytest.mark.parametrize("roles", [1, 2])
def test_fp32_error_against_oracle(cc, oracle_mod, roles):
    """FP32 perturbation form, with either warp-role form of the stencil:
    per-field relative L2 / Linf against the oracle."""
    cfg = W.C1_BELL
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(100)
    m = gpu_model(cc, cfg, cc.CC_FP32)
    m.set_warp_roles(0, roles)
    m.init_state()
    m.step(100)
    errs = _compare(cc, oracle_mod, m, om, report=True)
    for key, (l2, li) in errs.items():
        assert l2 <= 1e-3 and li <= 1e-2, (key, l2, li)
    m.close()


def test_long_run_against_oracle(cc, oracle_mod):
    """5,000 steps (the step count of the 512 x 512 x 128 precision case) on
    the 32 x 32 x 24 bell, against the oracle run for as long: the FP64 form
    stays at rounding level, and the FP32 perturbation form's error stays at
    the level that FP32 rounding accumulated over 5,000 steps gives (relative
    L2 1e-3 at most on the large domain against the FP64 GPU form)."""
    cfg = W.C1_BELL
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(5000)
    for prec, l2tol, litol in ((cc.CC_FP64, 1e-9, 1e-7), (cc.CC_FP32, 5e-3, 5e-2)):
        m = gpu_model(cc, cfg, prec)
        m.init_state()
        m.step(5000)
        errs = _compare(cc, oracle_mod, m, om, report=True)
        print("5000 steps", "FP64" if prec == cc.CC_FP64 else "FP32",
              {f"{k[0]}/{k[1]}": (float(f"{l2:.2e}"), float(f"{li:.2e}")) for k, (l2, li) in errs.items()})
        for key, (l2, li) in errs.items():
            assert l2 <= l2tol and li <= litol, (prec, key, l2, li)
        assert m.diagnostics(0)["steps"] == 5000
        m.close()


def test_ensemble_equals_single_domain_runs(cc):
    """Domains of uneven sizes advanced in one launch give the same bits as
    each domain advanced alone."""
    a = W.SMALL_HEMI
    b = W.C1_BELL.replace(nx=48, ny=40, nz=20, U=7.0, N=0.012, dt=0.12)
    both = gpu_model(cc, [a, b])
    both.init_state()
    both.step(12)
    for d, c in enumerate((a, b)):
        one = gpu_model(cc, c)
        one.init_state()
        one.step(12)
        for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ):
            assert np.array_equal(both.download(d, f), one.download(0, f)), (d, f)
        one.close()
    both.close()


def test_error_paths(cc):
    m = cc.Model(W.C1_BELL)
    with pytest.raises(cc.CutcellError) as e:
        m.step(1)
    assert e.value.status == cc.CC_ESTATE
    with pytest.raises(cc.CutcellError) as e:
        m.build_geometry()
    assert e.value.status == cc.CC_ESTATE
    bad = np.full((W.C1_BELL.ny, W.C1_BELL.nx), -1.0)
    with pytest.raises(cc.CutcellError) as e:
        m.set_terrain(0, bad)
    assert e.value.status == cc.CC_EINVAL
    m.close()


def test_v_shaped_valley_is_a_geometry_error(cc, oracle_mod):
    """Two steep slopes facing each other make two cells merge into each other
    (the excluded 'v-shaped valley' of Sec 2.3): both sides report it."""
    cfg = W.RunConfig("valley", 16, 8, 8, 50.0, 50.0, 50.0, 0.05, 1, "flat", 0.0, 1.0)
    h = np.zeros((8, 16))
    h[:, 7] = 120.0
    h[:, 8] = 20.0
    h[:, 9] = 120.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Model(cfg, h)
    m = cc.Model(cfg)
    m.set_terrain(0, h)
    with pytest.raises(cc.CutcellError) as e:
        m.build_geometry()
    assert e.value.status == cc.CC_EGEOM
    m.close()


def test_schedules_give_identical_bits_and_autotune_keeps_state(cc):
    """Every full-cell schedule (tile height, items per launch) and, in FP32,
    both warp-role forms (one thread updating scalars and momenta, or the two
    updates on separate warpgroups) distribute the same arithmetic: the states
    agree bit for bit; timing the schedules leaves the state unchanged."""
    a = W.SMALL_HEMI
    b = W.C1_BELL.replace(nx=48, ny=40, nz=20, U=7.0, N=0.012, dt=0.12)
    for prec, tys, roles in ((cc.CC_FP32, (16, 8), (1, 2)), (cc.CC_FP64, (8, 4), (1,))):
        ref = None
        for ty in tys:
            for items in (304, 912):
                for nr in roles:
                    m = gpu_model(cc, [a, b], prec)
                    m.init_state()
                    m.set_schedule(0, ty, items)
                    m.set_warp_roles(0, nr)
                    assert m.schedule(0) == (ty, items) and m.warp_roles(0) == nr
                    m.step(7)
                    out = [m.download(d, f) for d in range(2)
                           for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ)]
                    if ref is None:
                        ref = out
                    else:
                        for x, y in zip(out, ref):
                            assert np.array_equal(x, y), (prec, ty, items, nr)
                    m.close()
        m = gpu_model(cc, [a, b], prec)
        m.init_state()
        m.step(3)
        m.autotune(2)
        assert m.schedule(0)[0] in tys
        assert m.warp_roles(0) in roles
        m.step(4)
        out = [m.download(d, f) for d in range(2) for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ)]
        for x, y in zip(out, ref):
            assert np.array_equal(x, y), (prec, "autotuned")
        with pytest.raises(cc.CutcellError):
            m.set_schedule(0, 5, 304)
        for bad in (0, 3) if prec == cc.CC_FP32 else (0, 2):
            with pytest.raises(cc.CutcellError):
                m.set_warp_roles(0, bad)
        m.close()


def test_graph_replay_equals_direct_launches(cc):
    """Steps replayed from captured CUDA graphs give the same bits as the
    kernels launched one by one, across all four arrangements of the time
    levels."""
    a = W.SMALL_HEMI
    b = W.C1_BELL.replace(nx=48, ny=40, nz=20, U=7.0, N=0.012, dt=0.12)
    outs = []
    for on in (False, True):
        m = gpu_model(cc, [a, b], cc.CC_FP32)
        m.graphs(on)
        m.init_state()
        m.step(8)
        m.step(1)
        assert m.last_launch_count == 3  # one step: stencil, cut cells, diagnosis
        outs.append([m.download(d, f, lev) for d in range(2) for lev in (0, 1)
                     for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ, cc.CC_UB)
                     if not (f == cc.CC_UB and lev == 0)])
        m.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_full_size_hemisphere_rest_state_2000_steps(cc):
    """The 128x128x64 hemisphere (71 degree slopes, vertical and horizontal
    merges) at rest for 2000 FP64 steps: no spurious velocity and no mass
    change at all (the hydrostatic base state is exactly balanced)."""
    cfg = W.C2_HEMI.replace(U=0.0)
    m = gpu_model(cc, cfg, cc.CC_FP64)
    m.init_state()
    d0 = m.diagnostics()
    m.step(2000)
    d1 = m.diagnostics()
    assert d1["steps"] == 2000 and d1["nonfinite"] == 0
    assert d1["max_u"] == 0.0 and d1["max_w"] == 0.0
    assert d1["mass"] == d0["mass"] == 0.0
    for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ):
        assert np.abs(m.download(0, f)).max() == 0.0
    m.close()


def test_async_transfers_match_synchronous(cc, oracle_mod):
    """Queued uploads and downloads (one wait at the end) give the same
    state as the waiting ones."""
    torch = pytest.importorskip("torch")
    cfg = W.SMALL_HEMI
    om = oracle_mod.Model(cfg)
    om.init_state()
    om.step(5)
    pairs = [(cc.CC_RHOP, oracle_mod.F_RHOP), (cc.CC_PP, oracle_mod.F_PP), (cc.CC_MX, oracle_mod.F_MX),
             (cc.CC_MY, oracle_mod.F_MY), (cc.CC_MZ, oracle_mod.F_MZ)]
    outs = []
    for wait in (True, False):
        m = gpu_model(cc, cfg)
        m.init_state()
        m.step(1)
        host = {(f, lev): torch.from_numpy(om.field(fo, lev)).pin_memory() for f, fo in pairs for lev in (0, 1)}
        for (f, lev), a in host.items():
            m.upload_ptr(0, f, lev, a.data_ptr(), wait=wait)
        m.step(3)
        res = {f: torch.empty(tuple(m._shape(0, f)), dtype=torch.float64).pin_memory() for f, _ in pairs}
        for f, r in res.items():
            m.download_ptr(0, f, 1, r.data_ptr(), wait=wait)
        m.synchronize()
        outs.append([res[f].numpy().copy() for f, _ in pairs])
        m.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
