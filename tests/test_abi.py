"""The C ABI library loads and exports every function include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for mt in re.finditer(r"\b(cc_[A-Za-z0-9_]+)\s*\(", text):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("cc_init", "cc_run", "cc_free", "cc_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in _declared() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_strerror_without_gpu(built_lib):
    import paper_2311_02811_gb300 as cc
    assert cc.cc_strerror(cc.CC_OK) == "success"
    assert cc.cc_strerror(cc.CC_EIDRANGE) == "vertex id out of range"
    assert cc.cc_strerror(99) == "unknown status"


def test_argument_errors_need_no_gpu(built_lib):
    """Host-side argument checks run before any CUDA call."""
    import paper_2311_02811_gb300 as cc
    g = ctypes.c_void_p()
    assert cc.lib.cc_init(None, 4, 32, 0, None, None, 0, 0, None) == cc.CC_EINVAL
    assert cc.lib.cc_init(ctypes.byref(g), -1, 32, 0, None, None, 0, 0, None) == cc.CC_EINVAL
    assert cc.lib.cc_init(ctypes.byref(g), 4, 16, 0, None, None, 0, 0, None) == cc.CC_EINVAL
    assert cc.lib.cc_init(ctypes.byref(g), 1 << 31, 32, 0, None, None, 0, 0, None) == cc.CC_EINVAL
    assert cc.lib.cc_init(ctypes.byref(g), 4, 32, 7, None, None, 0, 0, None) == cc.CC_EINVAL
    assert cc.lib.cc_init(ctypes.byref(g), 4, 32, 0, None, None, 3, 0, None) == cc.CC_EINVAL
    assert "NULL" in cc.cc_last_error()
    assert cc.lib.cc_run(None, 2, 1, 1, 10, None, None, 0, None) == cc.CC_EINVAL


def test_scheduler_host_side_without_gpu(built_lib):
    """Class decoding and blob validation happen on the host."""
    import paper_2311_02811_gb300 as cc
    seen = set()
    for k in range(cc.CC_SCHED_CLASSES):
        o, m, c = cc.cc_sched_decode(k)
        assert o == (2, 4, cc.CC_ORDER_FULL)[k // 6] and m == (k // 3) % 2 and c == (1, 2, 4)[k % 3]
        seen.add((o, m, c))
    assert len(seen) == 18
    with pytest.raises(cc.CCError):
        cc.cc_sched_decode(18)
    assert cc.lib.cc_sched_load(b"not a blob", 10) == cc.CC_EINVAL
    assert cc.cc_sched_blob_bytes() == 120 + 2 * (64 * 12 + 64 * 64 * 2 + 18 * 64) + 4 * (64 * 3 + 18)


def test_release_memory_without_pools(built_lib):
    import paper_2311_02811_gb300 as cc
    cc.cc_release_memory()  # nothing allocated yet: no CUDA call is made
