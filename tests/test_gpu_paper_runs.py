"""The paper's uniform-grid experiments (Sec 3.1) at its own configuration on
the GPU: a 64 x 32 x 16 km domain at 200 m, U = 10 m/s, N = 0.01 1/s,
Theta = 300 K, one hour of flow (FP32). The lee-wave wavelength downstream
of the hill, measured from the vertical velocity along the line through the
hill centre, against the values the paper reports (tests/golden); and the
upstream ascent / leeward descent it describes (needs a GB300)."""
import os

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lee_wavelengths.txt")


def _rows():
    rows = []
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            k, h0, a, z, lam, tol = ln.split()
            rows.append((k, float(h0), float(a), float(z), float(lam), float(tol)))
    return rows


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def downstream_maxima(w, x0, dx, frac=0.02):
    """x positions (km) of the local maxima of w beyond x0 that exceed frac
    of the largest |w| on the segment."""
    i0 = int(round(x0 / dx))
    seg = w[i0:]
    big = frac * np.abs(seg).max()
    return [(i0 + i) * dx / 1000.0 for i in range(1, len(seg) - 1)
            if seg[i] > seg[i - 1] and seg[i] >= seg[i + 1] and seg[i] > big]


@pytest.mark.timeout(900)
@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[0])
def test_lee_wavelength_matches_the_paper(cc, row):
    kind, h0, a, z, lam, tol = row
    d = 200.0
    cfg = W.RunConfig(f"paper-{kind}", 320, 160, 80, d, d, d, 0.15, 1, kind, h0, a, theta0=300.0)
    m = cc.Model([cfg], cc.CC_FP32)
    m.set_terrain(0, cfg.heights())
    m.build_geometry()
    m.init_state()
    m.step(int(round(3600.0 / cfg.dt)))
    assert m.diagnostics(0)["nonfinite"] == 0
    w = m.derived(0, cc.CC_W)[int(round(z / d)), cfg.ny // 2, :]
    m.close()
    xc = cfg.nx * d / 2
    maxima = downstream_maxima(w, xc, d)
    assert len(maxima) >= 3, maxima
    wavelength = (maxima[2] - maxima[0]) / 2.0  # mean of the first two spacings
    assert abs(wavelength - lam) <= tol, (kind, maxima, wavelength)
    # ascent upstream of the hill, descent over its lee side
    assert w[int(round((xc - 1000.0) / d))] > 0 and w[int(round((xc + 1000.0) / d))] < 0
