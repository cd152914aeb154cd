"""Cyclic lateral boundaries (Sec 2.2) with the hill across the seam.  The
lateral boundaries are periodic, so moving the terrain by half the domain in x
and y moves the solution by the same amount.  The corner heights are rolled as
numbers, so the geometry is the same column by column; what differs is where
the periodic seam falls: through the hill, where the cut cells and the largest
perturbations are.  The stencils read the cyclic neighbours of the tiles at
the seam through wrapped indices.  The two runs agree to round-off only, since
the merge groups that straddle the seam sum their members in another order
(needs a GB300)."""
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


def _run(cc, cfg, h, prec, steps):
    m = cc.Model([cfg], prec)
    m.set_terrain(0, h)
    m.build_geometry()
    m.init_state()
    m.step(steps)
    out = {}
    for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ, cc.CC_UB):
        for level in ((1,) if f == cc.CC_UB else (0, 1)):
            out[(f, level)] = m.download(0, f, level)
    m.close()
    return out


@pytest.mark.parametrize("prec_name,tol", [("fp32", (1e-5, 1e-4)), ("fp64", (1e-12, 1e-10))])
# the small domains have only tiles whose halo wraps; 128 x 96 also has
# inner tiles
@pytest.mark.parametrize("cfg", [W.SMALL_HEMI, W.C1_BELL.replace(nx=48, ny=40, nz=20, U=7.0, N=0.012, dt=0.12),
                                 W.C1_BELL.replace(nx=128, ny=96, nz=20, U=7.0, N=0.012, dt=0.12, a=2500.0)],
                         ids=["hemisphere-40x36", "bell-48x40", "bell-128x96"])
def test_hill_across_the_periodic_seam(cc, cfg, prec_name, tol):
    prec = cc.CC_FP32 if prec_name == "fp32" else cc.CC_FP64
    h = cfg.heights()
    sy, sx = cfg.ny // 2, cfg.nx // 2
    a = _run(cc, cfg, h, prec, 20)
    b = _run(cc, cfg, np.roll(h, (sy, sx), axis=(0, 1)), prec, 20)
    for key, va in a.items():
        # host layouts: (levels, ny, nx), boundary-point velocity (ny, nx, 3)
        ax = (0, 1) if key[0] == cc.CC_UB else (-2, -1)
        ra = np.roll(va, (sy, sx), axis=ax)
        vb = b[key]
        scale = np.abs(ra).max()
        assert scale > 0.0, key
        l2 = np.sqrt(np.sum((vb - ra) ** 2) / np.sum(ra ** 2))
        li = np.abs(vb - ra).max() / scale
        assert l2 <= tol[0] and li <= tol[1], (key, l2, li)
