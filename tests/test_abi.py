"""The C-ABI library builds, loads and exports every entry point declared in
include/pmh.h; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pmh.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmh_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_00675_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    # the calls of the hot path's boundary: handle, batch sketch, estimator counts (all pairs and
    # listed pairs), merge of partial signatures, status reduction and the resource caps
    names = _declared()
    for n in ("pmh_create", "pmh_destroy", "pmh_last_error", "pmh_sketch_batch", "pmh_estimate_jp",
              "pmh_estimate_allpairs", "pmh_estimate_pairs", "pmh_merge", "pmh_sync_status", "pmh_set_limits",
              "pmh_sketch_batch_host", "pmh_sketch_batch_noalloc"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1911_00675_gb300 import pmh
    assert sorted(pmh.EXPORTS) == _declared()


def test_null_handle_and_bad_arguments_rejected_on_host(lib):
    lib.pmh_sketch_batch.restype = ctypes.c_int32
    lib.pmh_estimate_allpairs.restype = ctypes.c_int32
    lib.pmh_merge.restype = ctypes.c_int32
    vp = ctypes.c_void_p
    variants = (ctypes.c_int32 * 1)(0)
    rc = lib.pmh_sketch_batch(vp(0), vp(0), vp(0), vp(0), ctypes.c_int64(1), ctypes.c_uint32(8), variants,
                              ctypes.c_int32(1), ctypes.c_int32(1), ctypes.c_uint64(0), vp(0), vp(0), vp(0), vp(0),
                              vp(0))
    assert rc == 1   # PMH_ERR_INVALID_ARG
    assert lib.pmh_estimate_allpairs(vp(0), vp(0), ctypes.c_int64(1), ctypes.c_uint32(8), 0, vp(0), vp(0)) == 1
    assert lib.pmh_merge(vp(0), vp(0), vp(0), ctypes.c_int64(1), ctypes.c_uint32(8), vp(0), vp(0), vp(0)) == 1
    lib.pmh_estimate_jp.restype = ctypes.c_int32
    assert lib.pmh_estimate_jp(vp(0), vp(0), ctypes.c_int64(1), ctypes.c_uint32(8), 0, vp(0), vp(0)) == 1
    lib.pmh_sync_status.restype = ctypes.c_int32
    assert lib.pmh_sync_status(vp(0), vp(0), ctypes.c_int64(1), vp(0), vp(0), vp(0)) == 1
    lib.pmh_set_limits.restype = ctypes.c_int32
    assert lib.pmh_set_limits(vp(0), ctypes.c_uint32(0), ctypes.c_int32(-1)) == 1


def test_create_without_device_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.pmh_create.restype = ctypes.c_int32
    lib.pmh_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    rc = lib.pmh_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value
    assert lib.pmh_last_error(None)


def test_binding_counters_match_header():
    """The binding's counter names follow the header's PMH_CNT_* indices, and cover all of them."""
    from paper_1911_00675_gb300 import pmh
    with open(os.path.join(ROOT, "include", "pmh.h")) as f:
        src = f.read()
    idx = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"PMH_CNT_([A-Z0-9_]+)\s*=\s*(\d+)", src)}
    total = int(re.search(r"PMH_NUM_COUNTERS\s*=\s*(\d+)", src).group(1))
    assert len(pmh.COUNTERS) == total == len(idx)
    for name, i in idx.items():
        assert pmh.COUNTERS[i] == name, (name, i)


def test_prefilter_setter_checks_its_arguments(lib):
    lib.pmh_set_prefilter.restype = ctypes.c_int32
    lib.pmh_set_prefilter.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.pmh_set_prefilter(None, 2.0) == 1   # PMH_ERR_INVALID_ARG: no handle
