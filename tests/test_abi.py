"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/cutcell.h declares (no compute call here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1509_02572_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    assert "cc_create" in names and "cc_step" in names and len(names) >= 14


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1509_02572_gb300 import cutcell
    assert set(_declared()) <= set(cutcell.EXPORTS)


def test_create_rejects_bad_config_without_touching_the_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_1509_02572_gb300 import cutcell, workloads as W
    L = cutcell.load()
    bad = cutcell.config_from(W.C1_BELL.replace(nx=2))
    h = ctypes.c_void_p()
    st = L.cc_create(ctypes.byref(bad), 1, cutcell.CC_FP64, None, ctypes.byref(h))
    assert st == cutcell.CC_EINVAL and not h.value
    assert b"nx" in L.cc_last_error(None)
    st = L.cc_create(ctypes.byref(cutcell.config_from(W.C1_BELL)), 1, 7, None, ctypes.byref(h))
    assert st == cutcell.CC_EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1509_02572_gb300 import cutcell
    saved = cutcell._lib
    cutcell._lib = None
    try:
        with pytest.raises(RuntimeError):
            cutcell.load(str(tmp_path / "missing.so"))
    finally:
        cutcell._lib = saved


def test_create_rejects_empty_and_inconsistent_inputs(lib):
    """Empty and inconsistent inputs fail in the argument checks, before any
    CUDA call: no domains, domains that disagree on R / cp / p0, refined
    models with too few levels or odd box extents, a NULL result pointer."""
    from paper_1509_02572_gb300 import cutcell, workloads as W
    L = cutcell.load()
    h = ctypes.c_void_p()
    one = cutcell.config_from(W.C1_BELL)
    assert L.cc_create(ctypes.byref(one), 0, cutcell.CC_FP64, None, ctypes.byref(h)) == cutcell.CC_EINVAL
    assert b"at least one domain" in L.cc_last_error(None) and not h.value
    two = (cutcell.CCConfig * 2)(cutcell.config_from(W.C1_BELL), cutcell.config_from(W.C1_BELL.replace(R=288.0)))
    assert L.cc_create(two, 2, cutcell.CC_FP32, None, ctypes.byref(h)) == cutcell.CC_EINVAL
    assert b"share R" in L.cc_last_error(None)
    assert L.cc_create(ctypes.byref(one), 1, cutcell.CC_FP64, None, None) == cutcell.CC_EINVAL
    base = cutcell.config_from(W.SMALL_REFINED.base)
    boxes = (cutcell.CCBox * 1)(cutcell.CCBox(32, 32, 16, 16, 16))
    assert L.cc_create_refined(ctypes.byref(base), 1, boxes, cutcell.CC_FP32, None,
                               ctypes.byref(h)) == cutcell.CC_EINVAL
    odd = (cutcell.CCBox * 1)(cutcell.CCBox(31, 32, 16, 16, 16))
    assert L.cc_create_refined(ctypes.byref(base), 2, odd, cutcell.CC_FP32, None,
                               ctypes.byref(h)) == cutcell.CC_EINVAL
    assert b"even" in L.cc_last_error(None) and not h.value


def test_cube_layout_is_host_code_equal_to_the_oracle(lib):
    """The library's cube layout (host code, no GPU) equals the oracle's on
    the paper's hemisphere grids, a ridge that needs the balance pass and a
    plateau that drops cubes."""
    import numpy as np
    from paper_1509_02572_gb300 import cutcell, workloads as W
    from oracle import cbcm
    cases = []
    for nlev in (1, 2, 3):
        d = 400.0 / (1 << (nlev - 1))
        h = W.corner_heights("hemisphere", int(64000 / d), int(32000 / d), d, d, 1000.0, 1000.0)
        cases.append((160, 80, 40, 20, 400.0, nlev, h))
    nf = 8 * 8 * 8
    ridge = np.zeros((nf // 2, nf))
    ridge[:, nf // 2] = 50.0
    cases.append((64, 32, 16, 8, 100.0, 4, ridge))
    plateau = np.full((64, 128), 900.0)
    plateau[10, 10] = 950.0
    cases.append((64, 32, 32, 8, 100.0, 2, plateau))
    bell = W.corner_heights("bell", 256, 128, 50.0, 50.0, 600.0, 1500.0)
    cases.append((64, 32, 32, 16, 200.0, 3, bell))
    for args in cases:
        assert cutcell.cbcm_cubes(*args) == cbcm.cube_layout(*args), args[:6]
    assert [len(cutcell.cbcm_cubes(*c)) for c in cases[:3]] == [64, 148, 232]
    with pytest.raises(cutcell.CutcellError):
        cutcell.cbcm_cubes(30, 20, 20, 20, 400.0, 1, np.zeros((20, 30)))  # 30 is not a multiple of 20
