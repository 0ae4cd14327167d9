"""cc_run_noalloc: the entry point for callers that cannot allocate device memory.

Some callers own no device memory of their own -- for example a plugin or
serving loop inside a framework that has reserved the GPU's memory in its own
pool and forbids cudaMalloc during a step, or a latency-critical loop that
cannot pay for cudaMalloc/cudaFree synchronising the device.  For them the
library keeps its scratch (control words and the synchronous update array)
in one fixed device array, and the caller passes only edges and labels.

These tests call it through the C ABI and check it against the CPU oracle:
final labels against union-find (the smallest id of each component), and, in
the deterministic synchronous mode, the state after every sweep against the
Alg. 1 simulator.  Each case runs twice in a row, so that scratch left behind
by the first call cannot leak into the second, and the second call must leave
the device's free memory and torch's allocator untouched.  The existing
handle-based cc_run is run beside it as a second check.  The file is named to
be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_2311_02811_gb300 as lib
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return lib


def _noalloc(cc, n, s, d, order, mode, c, max_sweeps=1 << 20):
    """One call through the C ABI; returns (status, labels on the host, sweeps)."""
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sweeps = ctypes.c_int32(-1)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    rc = cc.lib.cc_run_noalloc(n, s.data_ptr(), d.data_ptr(), s.numel(), order, mode, c, max_sweeps,
                               out.data_ptr(), ctypes.byref(sweeps), stream)
    torch.cuda.synchronize()
    grew = (free0 - torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated() - alloc0)
    return rc, out.cpu().numpy(), sweeps.value, grew


def _graph(name):
    if name == "components64":
        return gg.components64()
    if name == "rmat16":
        return (1 << 16, *gg.rmat(16))
    if name == "grid":
        return (300 * 301, *gg.grid(300, 301))
    return (5001, *gg.path(5001))


@pytest.mark.parametrize("case", ["components64-sync-o2", "components64-async-o2", "rmat16-async-o2",
                                  "rmat16-sync-o4", "grid-async-full-c2", "path-sync-o2"])
def test_noalloc_matches_oracle_twice(cc, case):
    name, mode_s, order_s = case.split("-")[:3]
    n, s, d = _graph(name)
    mode = cc.CC_SYNC if mode_s == "sync" else cc.CC_ASYNC
    order = {"o2": 2, "o4": 4, "full": cc.CC_ORDER_FULL}[order_s]
    c = 2 if case.endswith("c2") else 1
    want = oracle.uf_labels(n, s, d)
    sim_iters = None
    if mode == cc.CC_SYNC:
        _, sim_iters, conv, _ = oracle.contour_sync(n, s, d, order)
        assert conv
    sd, dd = s.cuda(), d.cuda()
    for call in range(2):
        rc, got, sweeps, grew = _noalloc(cc, n, sd, dd, order, mode, c)
        assert rc == cc.CC_OK, (case, call, cc.cc_last_error())
        assert np.array_equal(got, want), (case, call)
        assert sweeps >= 1 and sweeps % c == 0
        if sim_iters is not None:
            assert sweeps == sim_iters, (case, call, sweeps, sim_iters)
        if call == 1:  # the defining property: nothing allocated on the device
            assert grew == (0, 0), (case, grew)
    # the handle-based entry point returns the same labels
    g = cc.cc_init(n, sd, dd)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = cc.cc_run(g, out, order, mode, c)
    cc.cc_free(g)
    assert np.array_equal(out.cpu().numpy(), want)
    if sim_iters is not None:
        assert st.sweeps == sim_iters


@pytest.mark.parametrize("order", [2, 4])
def test_noalloc_sync_every_sweep_matches_simulator(cc, order):
    """Stopped after k sweeps, the call returns CC_ENOTCONVERGED and the raw
    state of Alg. 1 after iteration k (Def. 3 with h = order)."""
    n, s, d = _graph("components64")
    _, it, conv, states = oracle.contour_sync(n, s, d, order, record=True)
    assert conv
    sd, dd = s.cuda(), d.cuda()
    for k in range(1, it + 1):
        for call in range(2):
            rc, got, sweeps, _ = _noalloc(cc, n, sd, dd, order, cc.CC_SYNC, 1, max_sweeps=k)
            assert sweeps == k, (k, call)
            assert np.array_equal(got, states[k - 1]), (k, call)
            assert rc == (cc.CC_OK if k == it else cc.CC_ENOTCONVERGED), (k, call, rc)


def test_noalloc_rejects_bad_arguments(cc):
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
    # host memory is refused before any launch
    h = torch.zeros(8, dtype=torch.int32).pin_memory()
    hn = np.zeros(8, dtype=np.int32)
    for a, b, o in [(h.data_ptr(), e.data_ptr(), out.data_ptr()), (e.data_ptr(), e.data_ptr(), hn.ctypes.data)]:
        rc = cc.lib.cc_run_noalloc(8, a, b, 4, 2, cc.CC_ASYNC, 1, 100, o, ctypes.byref(sweeps), None)
        msg = cc.cc_last_error()
        assert rc == cc.CC_EINVAL and ("device memory" in msg or "CUDA pointer" in msg), (rc, msg)
    with pytest.raises(ValueError):
        cc.cc_run_noalloc(8, e.cpu(), e, out)
    with pytest.raises(ValueError):
        cc.cc_run_noalloc(8, e.long(), e.long(), out)
    # out-of-range ids are found on the device and reported
    bad = torch.tensor([0, 1, 2, 99], dtype=torch.int32, device="cuda")
    rc = cc.lib.cc_run_noalloc(8, bad.data_ptr(), e.data_ptr(), 4, 2, cc.CC_ASYNC, 1, 100,
                               out.data_ptr(), ctypes.byref(sweeps), None)
    assert rc == cc.CC_EIDRANGE
    # and the entry point still works afterwards
    n2, s2, d2 = _graph("components64")
    rc, got, _, _ = _noalloc(cc, n2, s2.cuda(), d2.cuda(), 2, cc.CC_ASYNC, 1)
    assert rc == cc.CC_OK and np.array_equal(got, oracle.uf_labels(n2, s2, d2))
