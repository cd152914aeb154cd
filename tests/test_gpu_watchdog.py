"""Step watchdog (no counterpart in the paper).  A non-finite value or a corner
whose advective Courant number sum_d |u_d| dt / d_d exceeds 1 raises a flag in
the full-cell stencil; cc_synchronize, and a later cc_step, report it as
CC_ENUMERIC instead of stepping on silently, and cc_init_state clears it.  The
faults are planted on the host, in the uploaded state: nothing faults on the
GPU."""
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


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_watchdog_reports_a_planted_nan(cc, prec_name):
    prec = cc.CC_FP64 if prec_name == "fp64" else cc.CC_FP32
    cfg, m = _model(cc, prec)
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
