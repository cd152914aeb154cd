"""Checkpoint and resume through the C ABI (cc_save / cc_load): a model that
loads a checkpoint continues bit for bit as the saved one does, for an
ensemble and for a refined model; files that do not match the model are
rejected (needs a GB300)."""
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


ENS = W.ensemble_configs(3, seed=7)


def ensemble(cc, prec, cfgs=ENS):
    m = cc.Model(cfgs, prec)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    return m


def refined(cc, prec, rc=W.SMALL_REFINED):
    m = cc.RefinedModel(rc.base, rc.boxes, prec)
    for l, c in enumerate(m.cfgs):
        m.set_terrain(l, rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx)))
    m.build_geometry()
    return m


def state(cc, m, ndom):
    out = []
    for d in range(ndom):
        for f in (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ, cc.CC_UB):
            for tl in (0, 1):
                out.append(m.download(d, f, tl))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ensemble_resume_is_bit_exact(cc, tmp_path, prec):
    p = cc.CC_FP32 if prec == "fp32" else cc.CC_FP64
    path = str(tmp_path / "ens.ckpt")
    a = ensemble(cc, p)
    a.init_state()
    a.step(5)
    a.save(path)
    a.step(7)
    ref = state(cc, a, len(ENS))
    a.close()
    b = ensemble(cc, p)
    b.load(path)
    b.step(7)
    out = state(cc, b, len(ENS))
    b.close()
    for x, y in zip(out, ref):
        assert np.array_equal(x, y)


def test_refined_resume_is_bit_exact(cc, tmp_path):
    path = str(tmp_path / "ref.ckpt")
    a = refined(cc, cc.CC_FP32)
    a.init_state()
    a.step(3)
    a.save(path)
    q = a.mass()
    a.step(4)
    ref = state(cc, a, a.nlev)
    a.close()
    b = refined(cc, cc.CC_FP32)
    b.load(path)
    assert b.mass() == q
    b.step(4)
    out = state(cc, b, b.nlev)
    b.close()
    for x, y in zip(out, ref):
        assert np.array_equal(x, y)


def test_checkpoint_mismatch_is_rejected(cc, tmp_path):
    path = str(tmp_path / "ens.ckpt")
    a = ensemble(cc, cc.CC_FP32)
    with pytest.raises(cc.CutcellError) as e:
        a.save(path)  # no state yet
    assert e.value.status == cc.CC_ESTATE
    a.init_state()
    a.step(2)
    a.save(path)
    a.close()
    for other in (lambda: ensemble(cc, cc.CC_FP64),            # precision
                  lambda: ensemble(cc, cc.CC_FP32, ENS[:2]),   # domain count
                  lambda: ensemble(cc, cc.CC_FP32, [ENS[1], ENS[0], ENS[2]]),  # sizes
                  lambda: refined(cc, cc.CC_FP32),              # refinement
                  # the same sizes, another hill or another flow: the fingerprint
                  lambda: ensemble(cc, cc.CC_FP32, [ENS[0].replace(h0=ENS[0].h0 * 0.5), ENS[1], ENS[2]]),
                  lambda: ensemble(cc, cc.CC_FP32, [ENS[0], ENS[1].replace(U=ENS[1].U + 1.0), ENS[2]])):
        m = other()
        with pytest.raises(cc.CutcellError) as e:
            m.load(path)
        assert e.value.status == cc.CC_EINVAL
        m.close()
    raw = open(path, "rb").read()
    bad = tmp_path / "bad.ckpt"
    m = ensemble(cc, cc.CC_FP32)
    # header: magic (8 bytes), 4 int32, then per domain 10 int32 (sizes, the
    # four time-level roles at bytes 24 .. 39), int64 steps, uint64 fingerprint
    roles = bytearray(raw)
    roles[8 + 16 + 28:8 + 16 + 32] = roles[8 + 16 + 24:8 + 16 + 28]  # role 1 := role 0
    for blob in (b"not a checkpoint", raw[: len(raw) // 2], bytes(roles)):
        bad.write_bytes(blob)
        with pytest.raises(cc.CutcellError) as e:
            m.load(str(bad))
        assert e.value.status == cc.CC_EINVAL
    with pytest.raises(cc.CutcellError) as e:
        m.step(1)  # the truncated load left no valid state
    assert e.value.status == cc.CC_ESTATE
    with pytest.raises(cc.CutcellError) as e:
        m.load(str(tmp_path / "missing.ckpt"))
    assert e.value.status == cc.CC_EINVAL
    m.load(path)  # the intact file still loads into a matching model
    m.step(1)
    assert all(m.diagnostics(d)["nonfinite"] == 0 for d in range(len(ENS)))
    m.close()
