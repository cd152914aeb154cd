"""The allocation-free mass sum, for callers that cannot call cudaMalloc (for
example code that runs inside another framework's memory pool): called
through the C ABI on device buffers the caller owns, it must give the mass
that cc_diagnostics reports, on two calls in a row.  This file is collected
last so that a stop at the first failure has run every other test."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return torch, cutcell


@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_noalloc_mass_matches_diagnostics(env, prec_name, tol):
    torch, cc = env
    prec = cc.CC_FP64 if prec_name == "fp64" else cc.CC_FP32
    cfg = W.SMALL_HEMI
    m = cc.Model(cfg, prec)
    m.set_terrain(0, cfg.heights())
    m.build_geometry()
    m.init_state()
    m.step(30)
    ref = m.diagnostics()["mass"]
    rp = m.download(0, cc.CC_RHOP)
    vol = m.geometry()["vf"] * (cfg.dx * cfg.dy * cfg.dz)
    tdt = torch.float64 if prec == cc.CC_FP64 else torch.float32
    rho_dev = torch.tensor(rp.ravel(), dtype=tdt, device="cuda")
    vol_dev = torch.tensor(vol.ravel(), dtype=torch.float64, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    scale = np.abs(rp).max() * cfg.dx * cfg.dy * cfg.dz * cfg.cells
    # 256 partials is cc_diagnostics' own block count and reduction: the same
    # bits; one partial and the whole scratch array (its two edges) agree
    # within the tolerance, each on two calls in a row
    for nparts in (256, 1, cc.CC_NOALLOC_MAX_PARTS):
        for call in range(2):
            cc.mass_sum_noalloc(rho_dev.data_ptr(), prec, vol_dev.data_ptr(), rp.size, nparts, out.data_ptr())
            torch.cuda.synchronize()
            got = float(out[0].item())
            if nparts == 256:
                assert got == ref, (call, got, ref)
            assert abs(got - ref) <= tol * scale, (nparts, call, got, ref)
    m.close()


def test_noalloc_rejects_too_many_partials(env):
    torch, cc = env
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(cc.CutcellError) as e:
        cc.mass_sum_noalloc(x.data_ptr(), cc.CC_FP64, x.data_ptr(), 8, cc.CC_NOALLOC_MAX_PARTS + 1, out.data_ptr())
    assert e.value.status == cc.CC_EINVAL and "nparts" in str(e.value)
