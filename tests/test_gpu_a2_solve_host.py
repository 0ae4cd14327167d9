"""GPU parity of cc_solve_host (one solve of host edges, the upload overlapped
with sweeps) against the CPU oracle.

Asynchronous solves: final labels equal the union-find labels (the unique
fixed point), for every order, with edge lists of one chunk and of several
chunks with a ragged tail.  Synchronous solves: labels equal the oracle's and
the sweep count equals the Alg. 1 simulator's (the streamed part only checks
ids there).  Errors: out-of-range ids, device pointers, bad arguments.
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


def _pinned(x):
    return x.cpu().contiguous().pin_memory()


FAMILIES = {
    "rmat14": lambda: ((1 << 14),) + gg.rmat(14, seed=31),
    "path": lambda: (20_000,) + gg.path(20_000, seed=32),
    "grid": lambda: (128 * 96,) + gg.grid(128, 96, seed=33),
    "components64": lambda: gg.components64(seed=34),
    "er-sparse": lambda: (50_000,) + gg.er(50_000, 30_000, seed=35),
}


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("order", [1, 2, 4, 0, 3])
def test_async_labels_match_oracle(cc, family, order):
    n, s, d = FAMILIES[family]()
    want = oracle.uf_labels(n, s, d)
    out = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    st = cc.cc_solve_host(n, _pinned(s), _pinned(d), out, order, cc.CC_ASYNC, 1)
    assert np.array_equal(out.numpy(), want)
    assert st.sweeps >= 2 and st.solve_ms > 0
    # device output, check interval 2
    outd = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = cc.cc_solve_host(n, _pinned(s), _pinned(d), outd, order, cc.CC_ASYNC, 2)
    assert np.array_equal(outd.cpu().numpy(), want)


@pytest.mark.parametrize("family", ["path", "components64", "grid", "rmat14"])
def test_sync_sweeps_match_simulator(cc, family):
    """c = 1: Alg. 1's first iteration is streamed with the upload; c = 2:
    the chunks are only checked.  Every sweep count equals the simulator's,
    and a run stopped after k sweeps returns the simulator's k-th state."""
    n, s, d = FAMILIES[family]()
    want, iters, conv, _ = oracle.contour_sync(n, s.numpy(), d.numpy(), 2)
    assert conv
    out = torch.empty(n, dtype=torch.int32).pin_memory()
    st = cc.cc_solve_host(n, _pinned(s), _pinned(d), out, 2, cc.CC_SYNC, 1)
    assert st.sweeps == iters
    assert np.array_equal(out.numpy(), want)
    st = cc.cc_solve_host(n, _pinned(s), _pinned(d), out, 2, cc.CC_SYNC, 2)
    assert st.sweeps == iters + (iters % 2)
    assert np.array_equal(out.numpy(), want)
    for k in sorted({2, 3, iters - 1}):
        if not 2 <= k < iters:
            continue
        state_k = oracle.contour_sync(n, s.numpy(), d.numpy(), 2, max_iters=k)[0]
        rc, st = cc.cc_solve_host(n, _pinned(s), _pinned(d), out, 2, cc.CC_SYNC, 1, max_sweeps=k,
                                  raise_on_error=False)
        assert rc == cc.CC_ENOTCONVERGED and st.sweeps == k
        assert np.array_equal(out.numpy(), state_k), k


@pytest.mark.parametrize("n,m", [(1 << 21, (1 << 24) + (1 << 23) + 3), (1 << 23, (1 << 24) + (1 << 22) + 1)],
                         ids=["dense-sorted-chunks", "sparse-chunks-in-place"])
def test_several_chunks_with_ragged_tail(cc, n, m):
    """More than 2^24 edges: several chunks of the streamed upload (the tail
    halving), the last one ragged (not a multiple of 4 edges); average degree
    12 (chunks sorted) and 2.5 (chunks left in place)."""
    s, d = gg.er(n, m, seed=36)
    want = oracle.uf_labels(n, s, d)
    sp, dp = _pinned(s), _pinned(d)
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    for order in (2, 0):
        out.fill_(-1)
        cc.cc_solve_host(n, sp, dp, out, order, cc.CC_ASYNC, 1)
        assert np.array_equal(out.cpu().numpy(), want), order
    # the same graph through cc_init + cc_run: identical labels and, in sync
    # mode, identical sweep counts
    g = cc.cc_init(n, s.cuda(), d.cuda())
    ref = torch.empty(n, dtype=torch.int32, device="cuda")
    st_ref = cc.cc_run(g, ref, 2, cc.CC_SYNC, 1)
    cc.cc_free(g)
    out.fill_(-1)
    st = cc.cc_solve_host(n, sp, dp, out, 2, cc.CC_SYNC, 1)
    assert st.sweeps == st_ref.sweeps
    assert torch.equal(out, ref)


def test_pageable_host_edges(cc):
    n, s, d = FAMILIES["rmat14"]()
    out = np.full(n, -1, dtype=np.int32)
    cc.cc_solve_host(n, s.numpy(), d.numpy(), out, 2, cc.CC_ASYNC, 1)
    assert np.array_equal(out, oracle.uf_labels(n, s, d))


def test_edge_cases(cc):
    # no edges: identity labels; no vertices and no edges: nothing to do
    out = torch.full((7,), -1, dtype=torch.int32).pin_memory()
    e = torch.empty(0, dtype=torch.int32)
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        out.fill_(-1)
        cc.cc_solve_host(7, e, e, out, 2, mode, 1)
        assert out.tolist() == list(range(7))
    cc.cc_solve_host(0, e, e, torch.empty(0, dtype=torch.int32), 2, cc.CC_ASYNC, 1)
    # self-loops only: Alg. 1 stops after its first iteration
    s = torch.tensor([3, 3, 0], dtype=torch.int32)
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        out.fill_(-1)
        st = cc.cc_solve_host(7, s, s.clone(), out, 2, mode, 1)
        assert out.tolist() == list(range(7))
        if mode == cc.CC_SYNC:
            assert st.sweeps == 1


def test_not_converged_leaves_a_resumable_state(cc):
    n, s, d = FAMILIES["path"]()
    want = oracle.uf_labels(n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    rc, st = cc.cc_solve_host(n, _pinned(s), _pinned(d), out, 1, cc.CC_ASYNC, 1, max_sweeps=2,
                              raise_on_error=False)
    assert rc == cc.CC_ENOTCONVERGED and st.sweeps == 2
    snap = out.clone()
    lab = snap.cpu().numpy()
    assert (lab >= 0).all() and (lab <= np.arange(n)).all()
    g = cc.cc_init(n, s.cuda(), d.cuda())
    cc.cc_run(g, out, 2, cc.CC_ASYNC, 1, init_labels=snap)
    cc.cc_free(g)
    assert np.array_equal(out.cpu().numpy(), want)


def test_errors(cc):
    n = 100
    s = torch.tensor([0, 5, 100, 7], dtype=torch.int32)  # 100 is outside [0, 100)
    d = torch.tensor([1, 6, 2, -1], dtype=torch.int32)   # so is -1
    out = torch.empty(n, dtype=torch.int32).pin_memory()
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        rc, _ = cc.cc_solve_host(n, s, d, out, 2, mode, 1, raise_on_error=False)
        assert rc == cc.CC_EIDRANGE
        assert "first at edge 2" in cc.cc_last_error()
    # no vertices but edges
    rc, _ = cc.cc_solve_host(0, s, d, torch.empty(0, dtype=torch.int32), 2, cc.CC_ASYNC, 1,
                             raise_on_error=False)
    assert rc == cc.CC_EIDRANGE
    ok = torch.tensor([0, 1], dtype=torch.int32)
    # arguments
    for order, mode, c, ms in [(cc.CC_ORDER_AUTO, cc.CC_ASYNC, 1, 10), (2, cc.CC_ASYNC_COMPACT, 1, 10),
                               (2, cc.CC_ASYNC, 0, 10), (2, cc.CC_ASYNC, 1, 1), (cc.CC_ORDER_11MM, cc.CC_ASYNC, 1, 10)]:
        rc, _ = cc.cc_solve_host(n, ok, ok, out, order, mode, c, max_sweeps=ms, raise_on_error=False)
        assert rc == cc.CC_EINVAL, (order, mode, c, ms)
    # device edges: refused by the binding, and by the library itself
    dev = ok.cuda()
    with pytest.raises(ValueError):
        cc.cc_solve_host(n, dev, dev, out, 2, cc.CC_ASYNC, 1)
    st = cc.cc_stats()
    rc = cc.lib.cc_solve_host(n, dev.data_ptr(), dev.data_ptr(), 2, 2, cc.CC_ASYNC, 1, 10,
                              out.data_ptr(), 0, ctypes.byref(st), torch.cuda.current_stream().cuda_stream)
    assert rc == cc.CC_EINVAL
