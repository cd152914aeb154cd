"""FP32 host transfers through the C ABI (cc_upload_state_f32,
cc_download_state_f32 and their _async forms): for an FP32 model the values
travel unchanged, a step from FP32-uploaded values equals the step from the
same values uploaded through the FP64 calls, and an FP64 model refuses them
(needs a GB300)."""
import ctypes as ct

import numpy as np
import pytest

from paper_1509_02572_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = (0, 1, 2, 3, 4, 5)  # rho', p', rho u, rho v, rho w, boundary-point velocity


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_02572_gb300 import build, cutcell
    build.build()
    cutcell.load()
    return cutcell


CFGS = W.ensemble_configs(3, seed=11)


def model(cc, prec):
    m = cc.Model(CFGS, prec)
    for d, c in enumerate(CFGS):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    m.init_state()
    return m


def test_f32_download_equals_f64_download(cc):
    m = model(cc, cc.CC_FP32)
    m.step(5)
    for d in range(len(CFGS)):
        for f in FIELDS:
            for lev in (0, 1):
                a64 = m.download(d, f, lev)
                a32 = m.download(d, f, lev, dtype=np.float32)
                assert a32.dtype == np.float32
                # the state is FP32, so its FP64 copy converts back exactly
                assert np.array_equal(a64.astype(np.float32), a32), (d, f, lev)
                assert np.array_equal(a32.astype(np.float64), a64), (d, f, lev)
    m.close()


def test_f32_upload_steps_like_f64_upload(cc):
    rng = np.random.default_rng(1509)
    a = model(cc, cc.CC_FP32)
    b = model(cc, cc.CC_FP32)
    a.step(3)
    b.step(3)  # the same history (the first step of a run is a forward step)
    for d in range(len(CFGS)):
        for f in (0, 1):  # seeded perturbations of rho' and p' on top of the stepped state
            for lev in (0, 1):
                x = a.download(d, f, lev, dtype=np.float32)
                x = x + (rng.standard_normal(x.shape) * 1e-3 * (np.abs(x).max() + 1.0)).astype(np.float32)
                a.upload(d, f, lev, x)
                b.upload(d, f, lev, x.astype(np.float64))
                assert np.array_equal(a.download(d, f, lev, dtype=np.float32), x)
    a.step(4)
    b.step(4)
    for d in range(len(CFGS)):
        for f in FIELDS:
            assert np.array_equal(a.download(d, f), b.download(d, f)), (d, f)
    a.close()
    b.close()


def test_f32_async_round_trip_through_pinned_buffers(cc):
    torch = pytest.importorskip("torch")
    m = model(cc, cc.CC_FP32)
    m.step(2)
    want = {(d, f): m.download(d, f, 1, dtype=np.float32) for d in range(len(CFGS)) for f in FIELDS}
    bufs = {k: torch.from_numpy(v.copy()).pin_memory() for k, v in want.items()}
    outs = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in want.items()}
    for (d, f), t in bufs.items():
        m.upload_ptr(d, f, 1, t.data_ptr(), wait=False, f32=True)
    for (d, f), t in outs.items():
        m.download_ptr(d, f, 1, t.data_ptr(), wait=False, f32=True)
    m.synchronize()
    for k in want:
        assert np.array_equal(outs[k].numpy(), want[k]), k
    m.close()


def test_fp64_model_refuses_f32_buffers(cc):
    m = model(cc, cc.CC_FP64)
    x = np.zeros(m._shape(0, 0), np.float32)
    for fn in (m.L.cc_upload_state_f32, m.L.cc_download_state_f32, m.L.cc_upload_state_f32_async,
               m.L.cc_download_state_f32_async):
        assert fn(m.h, 0, 0, 1, x.ctypes.data_as(ct.c_void_p)) == 1  # CC_EINVAL
    # the model is unharmed
    m.step(1)
    assert np.isfinite(m.download(0, 1)).all()
    m.close()


@pytest.mark.parametrize("prec_name,f32", [("fp32", True), ("fp32", False), ("fp64", False)])
def test_whole_state_upload_equals_per_array_uploads(cc, prec_name, f32):
    """cc_upload_all_*: one host buffer with every domain's five fields at
    both levels lands where the per-array uploads put them, and the next
    steps are the same bit for bit."""
    torch = pytest.importorskip("torch")
    prec = cc.CC_FP32 if prec_name == "fp32" else cc.CC_FP64
    np_dt, t_dt = (np.float32, torch.float32) if f32 else (np.float64, torch.float64)
    src = model(cc, prec)
    src.step(4)
    parts = [src.download(d, f, lev, dtype=np_dt).ravel()
             for d in range(len(CFGS)) for f in range(5) for lev in (0, 1)]
    flat = np.concatenate(parts)
    src.step(1)  # the source moves on: the uploads must not read it
    a = model(cc, prec)
    b = model(cc, prec)
    assert a.state_elems() == flat.size == b.state_elems()
    host = torch.from_numpy(flat).pin_memory()
    a.upload_all_ptr(host.data_ptr(), f32=f32)
    a.synchronize()
    k = 0
    for d in range(len(CFGS)):
        for f in range(5):
            for lev in (0, 1):
                arr = np.ascontiguousarray(parts[k].reshape(src._shape(d, f)))
                b.upload(d, f, lev, arr.astype(np.float64))
                k += 1
    for m in (a, b):
        m.step(3)
    for d in range(len(CFGS)):
        for f in FIELDS:
            for lev in (0, 1):
                assert np.array_equal(a.download(d, f, lev), b.download(d, f, lev)), (d, f, lev)
    for m in (src, a, b):
        m.close()


def test_whole_state_upload_refusals(cc):
    m = model(cc, cc.CC_FP64)
    buf = (ct.c_float * 4)()
    with pytest.raises(cc.CutcellError) as e:
        m.upload_all_ptr(ct.addressof(buf), f32=True)
    assert e.value.status == cc.CC_EINVAL
    with pytest.raises(cc.CutcellError) as e:
        m.upload_all_ptr(0)
    assert e.value.status == cc.CC_EINVAL
    m.close()
