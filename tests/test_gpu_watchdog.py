"""Step watchdog (no counterpart in the paper).  A non-finite value or a corner
whose advective Courant number sum_d |u_d| dt / d_d exceeds 1 raises a flag in
the full-cell stencil; cc_synchronize, and a later cc_step, report it as
CC_ENUMERIC instead of stepping on silently, and cc_init_state clears it.  A
bounded wait for TMA copies that runs out raises a third flag, reported as
CC_ETIMEOUT.  The faults are planted on the host, in the uploaded state, or
by a barrier that expects bytes which never come: nothing faults on the GPU."""
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


def _model(cc, prec):
    cfg = W.SMALL_HEMI
    m = cc.Model(cfg, prec)
    m.set_terrain(0, cfg.heights())
    m.build_geometry()
    m.init_state()
    return cfg, m


@pytest.mark.parametrize("prec_name,roles", [("fp64", 1), ("fp32", 1), ("fp32", 2)])
def test_watchdog_reports_a_planted_nan(cc, prec_name, roles):
    prec = cc.CC_FP64 if prec_name == "fp64" else cc.CC_FP32
    cfg, m = _model(cc, prec)
    m.set_warp_roles(0, roles)
    m.step(3)
    m.synchronize()  # a healthy run raises nothing
    p = m.download(0, cc.CC_PP)
    p[cfg.nz // 2, cfg.ny // 3, cfg.nx // 4] = np.nan
    m.upload(0, cc.CC_PP, 1, p)
    m.step(2)
    with pytest.raises(cc.CutcellError) as e:
        m.synchronize()
    assert e.value.status == cc.CC_ENUMERIC and "non-finite" in str(e.value)
    # the flags have reached the host: the next call refuses to step on
    with pytest.raises(cc.CutcellError) as e:
        m.step(1)
    assert e.value.status == cc.CC_ENUMERIC
    # a new state clears the watchdog
    m.init_state()
    m.step(3)
    m.synchronize()
    m.close()


def test_watchdog_reports_an_excessive_courant_number(cc):
    cfg, m = _model(cc, cc.CC_FP64)
    m.step(2)
    m.synchronize()
    mx = m.download(0, cc.CC_MX)
    gz = 2  # corner levels below the floor in host arrays
    # a corner high above the hill: rho u with |u| dt / dx = 1.5
    K, J, I = cfg.nz - 3, cfg.ny // 2, cfg.nx // 2
    rho = mx[K + gz, J, I] / cfg.U
    mx[K + gz, J, I] = rho * 1.5 * cfg.dx / cfg.dt
    m.upload(0, cc.CC_MX, 1, mx)
    m.step(1)
    with pytest.raises(cc.CutcellError) as e:
        m.synchronize()
    assert e.value.status == cc.CC_ENUMERIC and "Courant" in str(e.value)
    m.close()


def _refined(cc, prec):
    rc = W.SMALL_REFINED
    m = cc.RefinedModel(rc.base, rc.boxes, prec)
    for lev, c in enumerate(m.cfgs):
        m.set_terrain(lev, rc.finest_heights() if lev == m.nlev - 1 else np.zeros((c.ny, c.nx)))
    m.build_geometry()
    return m


@pytest.mark.parametrize("roles", [1, 2])
def test_watchdog_reports_a_tma_wait_that_runs_out(cc, roles):
    """The refined boxes' FP32 stencil stages its planes with TMA copies and
    waits for each plane's barrier at most a second.  With every barrier made
    to expect 16 bytes more than its copies bring, each block's wait runs out:
    the block stops, drains its copies (bounded) and returns, and the host
    reads CC_ETIMEOUT, with one or two warp roles per block.  The context
    stays usable: the same model, restarted, matches a fresh one bit for
    bit."""
    m = _refined(cc, cc.CC_FP32)
    for lev in range(m.nlev):
        m.set_warp_roles(lev, roles)
    m.init_state()
    m.step(1)
    m.synchronize()
    m.inject_wait_timeout(True)
    m.step(1)
    with pytest.raises(cc.CutcellError) as e:
        m.synchronize()
    assert e.value.status == cc.CC_ETIMEOUT and "bounded wait" in str(e.value)
    with pytest.raises(cc.CutcellError) as e:
        m.step(1)
    assert e.value.status == cc.CC_ETIMEOUT
    m.inject_wait_timeout(False)
    m.init_state()
    m.step(3)
    m.synchronize()
    fresh = _refined(cc, cc.CC_FP32)
    fresh.init_state()
    fresh.step(3)
    for lev in range(m.nlev):
        for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ):
            assert np.array_equal(m.download(lev, f), fresh.download(lev, f)), (lev, f)
    fresh.close()
    m.close()
