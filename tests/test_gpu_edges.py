"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI
(needs a GB300): a domain smaller than one tile, odd extents that leave
ragged tiles, terrain with no cut cells (a flat floor at zero height, a flat
floor exactly on a face level) and so no merge groups, and a zero-step call."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("RHOP", "PP", "MX", "MY", "MZ", "UB")


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def _cfg(name, nx, ny, nz, terrain, h0, a, **kw):
    return W.RunConfig(name, nx, ny, nz, 50.0, 50.0, 50.0, 0.0375, 1, terrain, h0, a, **kw)


CASES = [
    (_cfg("tiny-4x4x4-bump", 4, 4, 4, "bell", 20.0, 40.0), None),
    (_cfg("odd-6x5x7-bell", 6, 5, 7, "bell", 30.0, 60.0), None),
    (_cfg("ragged-33x17x9-hemisphere", 33, 17, 9, "hemisphere", 200.0, 200.0), None),
    (_cfg("flat-24x20x12", 24, 20, 12, "flat", 0.0, 1.0), None),
    (_cfg("face-level-floor-24x20x12", 24, 20, 12, "flat", 0.0, 1.0), 50.0),
]


def _compare(cc, oracle_mod, m, om, l2tol, inftol):
    for name in FIELDS:
        fg, fo = getattr(cc, "CC_" + name), getattr(oracle_mod, "F_" + name)
        for level in ((1,) if name == "UB" else (0, 1)):
            a, b = m.download(0, fg, level), om.field(fo, level)
            scale = np.abs(b).max()
            if scale == 0.0:
                assert np.abs(a).max() == 0.0, (name, level)
                continue
            l2 = np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
            li = np.abs(a - b).max() / scale
            assert l2 <= l2tol and li <= inftol, (name, level, l2, li)


@pytest.mark.parametrize("cfg,floor", CASES, ids=[c.name for c, _ in CASES])
def test_edge_domains_match_oracle(cc, oracle_mod, cfg, floor):
    h = cfg.heights() if floor is None else np.full((cfg.ny, cfg.nx), floor)
    om = oracle_mod.Model(cfg, h)
    m = cc.Model([cfg], cc.CC_FP64)
    m.set_terrain(0, h)
    m.build_geometry()
    og, g = om.geometry(), m.geometry(0)
    assert np.array_equal(g["cls"], og["cls"]) and np.array_equal(g["root"], og["root"])
    hosts, _, _ = m.groups(0)
    if cfg.terrain == "flat":
        assert hosts.size == 0  # no cut cells, so no merge groups
    om.init_state()
    m.init_state()
    if cfg.terrain == "flat":
        # uniform flow over a flat floor stays uniform: seed a pressure bubble
        # in the full cells (the same values on both sides)
        k, j, i = np.meshgrid(np.arange(cfg.nz), np.arange(cfg.ny), np.arange(cfg.nx), indexing="ij")
        r2 = ((i - cfg.nx / 2) ** 2 + (j - cfg.ny / 2) ** 2 + (k - cfg.nz / 2) ** 2) / 9.0
        pp = np.where(og["cls"] == oracle_mod.C_FULL, 50.0 * np.exp(-r2), 0.0)
        for lev in (0, 1):
            om.set_field(oracle_mod.F_PP, lev, pp)
            m.upload(0, cc.CC_PP, lev, pp)
    _compare(cc, oracle_mod, m, om, 1e-13, 1e-11)
    om.step(1)
    m.step(1)
    _compare(cc, oracle_mod, m, om, 1e-12, 1e-10)
    om.step(9)
    m.step(9)
    _compare(cc, oracle_mod, m, om, 1e-10, 1e-8)
    before = [m.download(0, getattr(cc, "CC_" + f)) for f in FIELDS]
    steps = m.diagnostics(0)["steps"]
    m.step(0)
    assert m.diagnostics(0)["steps"] == steps
    for x, f in zip(before, FIELDS):
        assert np.array_equal(x, m.download(0, getattr(cc, "CC_" + f))), f
    m.close()
    # the FP32 form on the same domain
    m = cc.Model([cfg], cc.CC_FP32)
    m.set_terrain(0, h)
    m.build_geometry()
    m.init_state()
    if cfg.terrain == "flat":
        for lev in (0, 1):
            m.upload(0, cc.CC_PP, lev, pp)
    m.step(10)
    for name in FIELDS:
        a = m.download(0, getattr(cc, "CC_" + name))
        b = om.field(getattr(oracle_mod, "F_" + name))
        nb = np.linalg.norm(b)
        if nb > 0:
            assert np.linalg.norm(a - b) <= 1e-3 * nb, name
    m.close()


def test_ensemble_of_edge_domains_equals_single_runs(cc):
    """The edge domains advanced together in one ensemble launch give the same
    bits as each alone."""
    cfgs = [c for c, floor in CASES if floor is None]
    m = cc.Model(cfgs, cc.CC_FP32)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    m.init_state()
    m.step(6)
    together = [m.download(d, cc.CC_PP) for d in range(len(cfgs))]
    m.close()
    for d, c in enumerate(cfgs):
        s = cc.Model([c], cc.CC_FP32)
        s.set_terrain(0, c.heights())
        s.build_geometry()
        s.init_state()
        s.step(6)
        assert np.array_equal(s.download(0, cc.CC_PP), together[d]), c.name
        s.close()
