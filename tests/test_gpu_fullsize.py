"""The benchmark's full-size single-level configurations, launched as the
benchmark launches them (FP32 perturbation form, autotuned schedule, CUDA
graphs), against the FP64 oracle (needs a GB300):
  * the 512 x 512 x 128 bell (100 m / 50 m cells): geometry bit for bit, then
    the first steps element by element in FP64 and FP32 over the whole domain;
  * the 64-instance ensemble of uneven sizes: instances sampled from the one
    ensemble launch against the oracle run of each sampled instance alone."""
import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAIRS = ("RHOP", "PP", "MX", "MY", "MZ", "UB")


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


def bench_model(cc, cfgs, prec):
    """A model made as the benchmark makes it (terrain, geometry, state, then
    the autotuner; graphs are on by default)."""
    m = cc.Model(cfgs, prec)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    m.init_state()
    m.autotune(2)
    return m


def errors(cc, oracle_mod, m, d, om):
    out = {}
    for name in PAIRS:
        fg, fo = getattr(cc, "CC_" + name), getattr(oracle_mod, "F_" + name)
        for level in ((1,) if name == "UB" else (0, 1)):
            a, b = m.download(d, fg, level), om.field(fo, level)
            scale = np.abs(b).max()
            if scale == 0.0:
                out[(name, level)] = (float(np.abs(a).max()), float(np.abs(a).max()))
                continue
            out[(name, level)] = (float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))),
                                  float(np.abs(a - b).max() / scale))
    return out


@pytest.mark.timeout(1800)
def test_c3_bell_full_size_against_oracle(cc, oracle_mod):
    cfg = W.C3_BELL
    om = oracle_mod.Model(cfg)
    og = om.geometry()
    m64 = cc.Model([cfg], cc.CC_FP64)
    m64.set_terrain(0, cfg.heights())
    m64.build_geometry()
    g = m64.geometry(0)
    assert np.array_equal(g["cls"], og["cls"]) and np.array_equal(g["root"], og["root"])
    assert np.max(np.abs(g["vf"] - og["vf"])) <= 1e-14
    del g, og
    om.init_state()
    om.step(2)
    m64.init_state()
    m64.autotune(2)
    m64.step(2)
    for key, (l2, li) in errors(cc, oracle_mod, m64, 0, om).items():
        assert l2 <= 1e-10 and li <= 1e-8, (key, l2, li)
    m64.close()
    m32 = bench_model(cc, [cfg], cc.CC_FP32)
    m32.step(2)
    for key, (l2, li) in errors(cc, oracle_mod, m32, 0, om).items():
        assert l2 <= 1e-4 and li <= 1e-3, (key, l2, li)
    m32.close()


@pytest.mark.timeout(1800)
def test_full_ensemble_sampled_instances_against_oracle(cc, oracle_mod):
    cfgs = W.ensemble_configs(64)
    m = bench_model(cc, cfgs, cc.CC_FP32)
    steps = 10
    m.step(steps)
    for d in range(len(cfgs)):
        assert m.diagnostics(d)["nonfinite"] == 0
    # the three smallest instances, one of each hill kind where possible
    order = sorted(range(len(cfgs)), key=lambda d: (cfgs[d].cells, d))
    picked, kinds = [], set()
    for d in order:
        if cfgs[d].terrain not in kinds or len(picked) >= 2:
            picked.append(d)
            kinds.add(cfgs[d].terrain)
        if len(picked) == 3:
            break
    for d in picked:
        om = oracle_mod.Model(cfgs[d])
        om.init_state()
        om.step(steps)
        for key, (l2, li) in errors(cc, oracle_mod, m, d, om).items():
            assert l2 <= 1e-3 and li <= 1e-2, (d, key, l2, li)
    m.close()
