"""Sibling blocks of the finest level (Sec 2.2: a level made of blocks, each with
its own ghost shell, filled by copies from the blocks next to it on the same
level and by injection from the coarser level elsewhere) through the C ABI
(needs a GB300).

The same-level copy puts into every block's ghost shell the values its
neighbours hold, at the time levels the next step reads, so each cell is
updated from the same values in the same operations as in the undivided box:
the blocked run must equal the undivided run bit for bit, and so the oracle of
the undivided level is the oracle of the blocked one."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RC = W.SMALL_BLOCKED
FIELDS = ("CC_RHOP", "CC_PP", "CC_MX", "CC_MY", "CC_MZ", "CC_UB")


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def _model(cc, prec, blocks, **kw):
    base = RC.base.replace(**kw) if kw else RC.base
    m = cc.RefinedModel(base, RC.boxes, prec, xcuts=RC.xcuts if blocks else (), ycuts=RC.ycuts if blocks else ())
    for lev in range(m.nlev):
        c = m.cfgs[m.level_domains(lev)[0]]
        if lev == m.nlev - 1:
            m.set_level_terrain(lev, RC.finest_heights())
        else:
            m.set_terrain(lev, np.zeros((c.ny, c.nx)))
    m.build_geometry()
    return m


def _state(cc, m):
    """Every field of every level at both time levels (the finest level
    stitched from its blocks)."""
    out = {}
    for lev in range(m.nlev):
        for name in FIELDS:
            f = getattr(cc, name)
            for tl in ((1,) if name == "CC_UB" else (0, 1)):
                out[(lev, name, tl)] = m.download_level(lev, f, tl)
    return out


def test_blocked_layout(cc):
    m = _model(cc, cc.CC_FP64, True)
    assert m.ndom == 2 + 6 and m.nlev == 3
    assert [b for b in m.blocks[2:]] == [(2, 0, 0), (2, 18, 0), (2, 46, 0), (2, 0, 46), (2, 18, 46), (2, 46, 46)]
    assert [(c.nx, c.ny) for c in m.cfgs[2:]] == [(18, 46), (28, 46), (18, 46), (18, 18), (28, 18), (18, 18)]
    m.close()


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_blocks_equal_the_undivided_box_bit_for_bit(cc, prec_name):
    prec = cc.CC_FP64 if prec_name == "fp64" else cc.CC_FP32
    runs = []
    for blocks in (False, True):
        m = _model(cc, prec, blocks)
        m.init_state()
        m.step(1)   # forward-Euler start
        m.step(4)
        runs.append(_state(cc, m))
        m.close()
    for key, a in runs[0].items():
        b = runs[1][key]
        assert a.shape == b.shape, key
        assert np.array_equal(a, b), (key, np.abs(a - b).max())


def test_warp_roles_give_the_same_bits_on_every_level(cc):
    """FP32: the stencil with the scalar and momentum updates on separate
    warpgroups gives the same bits as one thread per pair updating both, on
    the periodic level 0 (cyclic gather) and the refined levels (TMA-staged
    boxes and blocks) alike, after the start and four cycles."""
    runs = []
    for nr in (1, 2):
        m = _model(cc, cc.CC_FP32, True)
        for lev in range(m.nlev):
            m.set_warp_roles(m.level_domains(lev)[0], nr)
        assert all(m.warp_roles(d) == nr for d in range(m.ndom))
        m.init_state()
        m.step(1)
        m.step(4)
        runs.append(_state(cc, m))
        m.close()
    for key, a in runs[0].items():
        assert np.array_equal(a, runs[1][key]), (key, np.abs(a - runs[1][key]).max())


def test_blocks_against_the_oracle(cc, oracle_mod):
    """FP64: every level, field and time level against the oracle of the
    undivided levels, after the start and after five cycles."""
    R = oracle_mod.Refine(RC.base, RC.boxes, RC.finest_heights(pad=4))
    R.init_state()
    m = _model(cc, cc.CC_FP64, True)
    m.init_state()
    pairs = [(n, getattr(oracle_mod, "F_" + n[3:])) for n in FIELDS]
    for steps, (tl2, tli) in ((1, (1e-12, 1e-10)), (4, (1e-10, 1e-8))):
        R.step(steps)
        m.step(steps)
        for name, fo in pairs:
            f = getattr(cc, name)
            for tl in ((1,) if name == "CC_UB" else (0, 1)):
                a = [m.download_level(lev, f, tl) for lev in range(m.nlev)]
                b = [lev.field(fo, tl) for lev in R.levels]
                scale = max(np.abs(x).max() for x in b)
                norm = np.sqrt(sum(np.sum(x ** 2) for x in b))
                for lev in range(m.nlev):
                    if scale == 0.0:
                        assert np.abs(a[lev]).max() == 0.0
                        continue
                    l2 = np.sqrt(np.sum((a[lev] - b[lev]) ** 2)) / norm
                    li = np.abs(a[lev] - b[lev]).max() / scale
                    assert l2 <= tl2 and li <= tli, (steps, lev, name, tl, l2, li)
    m.close()


def test_blocks_conserve_mass_with_the_filter_off(cc):
    """FP64, Robert-Asselin filter off: the two-time-level perturbation mass
    over the active cells of all levels (the finest level summed over its
    blocks) is conserved to round-off."""
    m = _model(cc, cc.CC_FP64, True, ra_nu=0.0)
    whole = _model(cc, cc.CC_FP64, False, ra_nu=0.0)
    for x in (m, whole):
        x.init_state()
        x.step(1)  # the forward-Euler start (not part of the two-time-level invariant)
    q0 = m.mass()
    b = RC.base
    nx, ny, nz, ox, oy = RC.boxes[0]
    # the mass one step moves through the coarse-fine interface
    scale = 1.2 * b.U * (ny * b.dy / 2) * (nz * b.dz / 2) * 2 * b.dt
    for _ in range(3):
        m.step(2)
        whole.step(2)
        assert abs(m.mass() - q0) <= 1e-13 * scale, (m.mass(), q0)
        # the same state, summed over the blocks in another order
        assert abs(m.mass() - whole.mass()) <= 1e-13 * scale
    assert np.abs(m.download_level(2, cc.CC_RHOP)).max() > 0.0
    whole.close()
    m.close()


def test_block_cuts_are_checked(cc):
    with pytest.raises(cc.CutcellError) as e:
        cc.RefinedModel(RC.base, RC.boxes, cc.CC_FP64, xcuts=(17,))
    assert e.value.status == cc.CC_EINVAL
    with pytest.raises(cc.CutcellError):
        cc.RefinedModel(RC.base, RC.boxes, cc.CC_FP64, xcuts=(10,))
    with pytest.raises(cc.CutcellError):
        cc.RefinedModel(RC.base, RC.boxes, cc.CC_FP64, ycuts=(30, 40))
    # terrain within 8 corners of a cut
    m = cc.RefinedModel(RC.base, RC.boxes, cc.CC_FP64, xcuts=(30,))
    with pytest.raises(cc.CutcellError) as e:
        m.set_level_terrain(2, RC.finest_heights())
    assert e.value.status == cc.CC_EINVAL
    m.close()
