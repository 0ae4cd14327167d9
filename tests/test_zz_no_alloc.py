"""cc_run_noalloc: the entry point for callers that cannot allocate device memory.

Some callers own no device memory of their own -- for example a plugin or
serving loop inside a framework that has reserved the GPU's memory in its own
pool and forbids cudaMalloc during a step, or a latency-critical loop that
cannot pay for cudaMalloc/cudaFree synchronising the device.  For them the
library keeps its scratch (control words and the synchronous update array)
in one fixed device array, and the caller passes only edges and labels.

These tests call it through the C ABI and check that it returns exactly the
labels (and, for the deterministic synchronous mode, the sweep count) that the
handle-based cc_run returns, on two calls in a row so that the shared scratch
left behind by the first call cannot leak into the second.  The file is named
to be collected last.
"""
import ctypes

import pytest
import torch

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_2311_02811_gb300 as lib
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return lib


def _reference(cc, n, s, d, order, mode, c):
    g = cc.cc_init(n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = cc.cc_run(g, out, order, mode, c)
    cc.cc_free(g)
    return out, st.sweeps


def _noalloc(cc, n, s, d, order, mode, c):
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sweeps = ctypes.c_int32(-1)
    stream = torch.cuda.current_stream().cuda_stream
    rc = cc.lib.cc_run_noalloc(n, s.data_ptr(), d.data_ptr(), s.numel(), order, mode, c, 1 << 20,
                               out.data_ptr(), ctypes.byref(sweeps), stream)
    assert rc == cc.CC_OK, cc.cc_last_error()
    return out, sweeps.value


@pytest.mark.parametrize("case", ["components64-sync-o2", "components64-async-o2",
                                  "rmat16-async-o2", "rmat16-sync-o4", "grid-async-full-c2"])
def test_noalloc_matches_cc_run_twice(cc, case):
    if case.startswith("components64"):
        n, s, d = gg.components64(device="cuda")
    elif case.startswith("rmat16"):
        n = 1 << 16
        s, d = gg.rmat(16, device="cuda")
    else:
        n = 300 * 301
        s, d = gg.grid(300, 301, device="cuda")
    mode = cc.CC_SYNC if "-sync-" in case else cc.CC_ASYNC
    order = {"o2": 2, "o4": 4, "full": cc.CC_ORDER_FULL}[case.split("-")[2]]
    c = 2 if case.endswith("c2") else 1
    want, want_sweeps = _reference(cc, n, s, d, order, mode, c)
    for call in range(2):
        got, sweeps = _noalloc(cc, n, s, d, order, mode, c)
        assert torch.equal(got, want), (case, call)
        assert sweeps >= 1 and sweeps % c == 0
        if mode == cc.CC_SYNC:
            assert sweeps == want_sweeps, (case, call)


def test_noalloc_rejects_sizes_beyond_its_scratch(cc):
    n = cc.CC_NOALLOC_MAX_N
    e = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(n + 4, dtype=torch.int32, device="cuda")
    sweeps = ctypes.c_int32(0)
    rc = cc.lib.cc_run_noalloc(n + 1, e.data_ptr(), e.data_ptr(), 4, 2, cc.CC_SYNC, 1, 100,
                               out.data_ptr(), ctypes.byref(sweeps), None)
    assert rc == cc.CC_EINVAL
    assert "scratch" in cc.cc_last_error()
    # misaligned buffers are refused rather than copied
    rc = cc.lib.cc_run_noalloc(8, e.data_ptr() + 4, e.data_ptr(), 3, 2, cc.CC_ASYNC, 1, 100,
                               out.data_ptr(), ctypes.byref(sweeps), None)
    assert rc == cc.CC_EINVAL
    # out-of-range ids are found on the device and reported
    bad = torch.tensor([0, 1, 2, 99], dtype=torch.int32, device="cuda")
    rc = cc.lib.cc_run_noalloc(8, bad.data_ptr(), e.data_ptr(), 4, 2, cc.CC_ASYNC, 1, 100,
                               out.data_ptr(), ctypes.byref(sweeps), None)
    assert rc == cc.CC_EIDRANGE
