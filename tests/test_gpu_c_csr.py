"""GPU parity of the native CSR sweep (CC_CSR_NATIVE, CC_CSR_NATIVE_SYM).

The rows are walked in place of an expanded edge list, so the edge set a
sweep applies is
* CC_CSR_NATIVE: every stored entry (r, cols[k]);
* CC_CSR_NATIVE_SYM: the entries with cols[k] < r (one per undirected edge of
  a symmetric input; self-loops dropped).
Synchronous runs are compared with the Alg. 1 simulator on exactly that edge
set after every sweep; asynchronous runs end at the union-find labels.
"""
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


def applied_edges(off, cols, symmetric):
    """The (row, col) pairs a native CSR sweep applies, from the CSR arrays."""
    off, cols = off.cpu().numpy(), cols.cpu().numpy()
    rows = np.repeat(np.arange(off.size - 1, dtype=np.int64), np.diff(off)).astype(np.int32)
    if symmetric:
        keep = cols < rows
        return rows[keep], cols[keep]
    return rows, cols


def csr_solve(cc, n, off, cols, layout, order=2, mode=1, c=1, max_sweeps=1 << 20, on_device=True,
              expect_ok=True):
    if on_device:
        off, cols = off.cuda(), cols.cuda()
    g = cc.cc_init(n, off, cols, m=cols.numel(), id_bits=32, layout=layout, on_device=on_device)
    try:
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc, st = cc.cc_run(g, out, order, mode, c, max_sweeps, raise_on_error=False)
    finally:
        cc.cc_free(g)
    if expect_ok:
        assert rc == cc.CC_OK, (rc, cc.cc_last_error())
    return out.cpu().numpy(), st, rc


GRAPHS = {
    "components64": lambda seed: gg.components64(seed=seed),
    "rmat12": lambda seed: (1 << 12, *gg.rmat(12, seed=seed)),
    "grid64": lambda seed: (64 * 64, *gg.grid(64, 64, seed=seed)),
    "path3001": lambda seed: (3001, *gg.path(3001, seed=seed)),
    "er": lambda seed: (5000, *gg.er(5000, 3000, seed=seed)),  # isolated vertices = empty rows
}
LAYOUTS = [(2, False), (3, True)]  # (layout, symmetric input)


@pytest.mark.parametrize("layout,sym", LAYOUTS, ids=["native", "native-sym"])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 0])
@pytest.mark.parametrize("name", ["rmat12", "grid64", "path3001", "er"])
def test_csr_sync_matches_simulator(cc, name, order, layout, sym):
    n, s, d = GRAPHS[name](1)
    off, cols = gg.to_csr(n, s, d, symmetric=sym)
    es, ed = applied_edges(off, cols, sym)
    h = 1024 if order == 0 else order
    want, it, conv, _ = oracle.contour_sync(n, es, ed, h)
    assert conv
    got, st, _ = csr_solve(cc, n, off, cols, layout, order, cc.CC_SYNC)
    assert st.sweeps == it
    assert (got == want).all()
    assert (got == oracle.uf_labels(n, s, d)).all()


@pytest.mark.parametrize("layout,sym", LAYOUTS, ids=["native", "native-sym"])
def test_csr_sync_every_sweep(cc, layout, sym):
    n, s, d = gg.components64()
    off, cols = gg.to_csr(n, s, d, symmetric=sym)
    es, ed = applied_edges(off, cols, sym)
    _, it, conv, states = oracle.contour_sync(n, es, ed, 2, record=True)
    assert conv
    for k in range(1, it + 1):
        got, st, rc = csr_solve(cc, n, off, cols, layout, 2, cc.CC_SYNC, 1, max_sweeps=k, expect_ok=False)
        assert st.sweeps == k and (got == states[k - 1]).all(), k
        assert rc == (cc.CC_OK if k == it else cc.CC_ENOTCONVERGED)


@pytest.mark.parametrize("layout,sym", LAYOUTS, ids=["native", "native-sym"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_csr_async_many_seeds(cc, name, layout, sym):
    for seed in range(6):
        n, s, d = GRAPHS[name](seed)
        off, cols = gg.to_csr(n, s, d, symmetric=sym)
        want = oracle.uf_labels(n, s, d)
        for order in (1, 2, 3, 4, 0):
            for c in (1, 2):
                got, st, _ = csr_solve(cc, n, off, cols, layout, order, cc.CC_ASYNC, c)
                assert (got == want).all(), (name, seed, order, c)


@pytest.mark.parametrize("layout,sym", LAYOUTS, ids=["native", "native-sym"])
def test_csr_host_input_and_ragged_tails(cc, layout, sym):
    """Host arrays (copied), and nnz % 4 = 0..3 so the last group is ragged."""
    for m in (1, 2, 3, 4, 5, 6, 7, 33, 1001):
        n = 97
        s, d = gg.er(n, m, seed=m)
        off, cols = gg.to_csr(n, s, d, symmetric=sym)
        want = oracle.uf_labels(n, s, d)
        for on_dev in (False, True):
            for mode in (cc.CC_SYNC, cc.CC_ASYNC):
                got, _, _ = csr_solve(cc, n, off, cols, layout, 2, mode, on_device=on_dev)
                assert (got == want).all(), (m, on_dev, mode)


def test_csr_edge_cases(cc):
    e64 = torch.zeros(1, dtype=torch.int64)
    e32 = torch.empty(0, dtype=torch.int32)
    for layout in (cc.CC_CSR_NATIVE, cc.CC_CSR_NATIVE_SYM):
        # n = 0, no entries
        g = cc.cc_init(0, e64.cuda(), e32.cuda(), m=0, id_bits=32, layout=layout, on_device=True)
        cc.cc_run(g, torch.empty(0, dtype=torch.int32, device="cuda"), 2, cc.CC_ASYNC, 1)
        cc.cc_free(g)
        # vertices without entries
        off = torch.zeros(9, dtype=torch.int64)
        got, st, _ = csr_solve(cc, 8, off, e32, layout, 2, cc.CC_SYNC)
        assert (got == np.arange(8)).all() and st.sweeps == 1
    # self-loops only, empty rows in between, one real edge stored both ways
    off = torch.tensor([0, 1, 1, 3, 3, 4, 5], dtype=torch.int64)
    cols = torch.tensor([0, 2, 4, 4, 2], dtype=torch.int32)  # rows: 0:[0] 2:[2,4] 4:[4] 5:[2]
    want = oracle.uf_labels(6, [0, 2, 2, 4, 5], [0, 2, 4, 4, 2])
    for layout in (cc.CC_CSR_NATIVE, cc.CC_CSR_NATIVE_SYM):
        for mode in (cc.CC_SYNC, cc.CC_ASYNC):
            got, _, _ = csr_solve(cc, 6, off, cols, layout, 2, mode)
            if layout == cc.CC_CSR_NATIVE:
                assert (got == want).all()
            else:  # only (5, 2) has col < row; (2, 4) is not mirrored, so it is dropped
                assert got.tolist() == [0, 1, 2, 3, 4, 2]


def test_csr_errors(cc):
    off = torch.tensor([0, 2, 1, 3], dtype=torch.int64)  # decreasing
    cols = torch.tensor([1, 2, 0], dtype=torch.int32)
    for layout in (cc.CC_CSR_NATIVE, cc.CC_CSR_NATIVE_SYM):
        with pytest.raises(cc.CCError) as ei:
            cc.cc_init(3, off, cols, m=3, id_bits=32, layout=layout, on_device=False)
        assert ei.value.status == cc.CC_EINVAL
        good = torch.tensor([0, 1, 2, 3], dtype=torch.int64)
        with pytest.raises(cc.CCError) as ei:
            cc.cc_init(3, good, torch.tensor([1, 5, 0], dtype=torch.int32), m=3, id_bits=32, layout=layout,
                       on_device=False)
        assert ei.value.status == cc.CC_EIDRANGE
        with pytest.raises(cc.CCError) as ei:
            cc.cc_init(3, good, cols.to(torch.int64), m=3, id_bits=64, layout=layout, on_device=False)
        assert ei.value.status == cc.CC_EINVAL
        g = cc.cc_init(3, good, cols, m=3, id_bits=32, layout=layout, on_device=False)
        with pytest.raises(cc.CCError) as ei:
            cc.cc_graph_reorder(g, cc.CC_REORDER_LOWDEG)
        assert ei.value.status == cc.CC_EINVAL
        assert cc.cc_graph_info(g) == (3, 3)
        cc.cc_free(g)


def test_csr_borrowed_arrays_and_edges_pointers(cc):
    n, s, d = GRAPHS["rmat12"](3)
    off, cols = gg.to_csr(n, s, d, symmetric=True)
    off, cols = off.cuda(), cols.cuda()
    g = cc.cc_init(n, off, cols, m=cols.numel(), id_bits=32, layout=cc.CC_CSR_NATIVE_SYM, on_device=True)
    a, b = cc.cc_graph_edges(g)
    assert a == off.data_ptr() and b == cols.data_ptr()  # borrowed, not copied
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = cc.cc_run(g, out, 2, cc.CC_ASYNC, 1)
    cc.cc_free(g)
    assert (out.cpu().numpy() == oracle.uf_labels(n, s, d)).all()
    assert st.alg_bytes > 0


def test_csr_auto_schedule_and_features(cc):
    """CC_ORDER_AUTO on a native CSR handle samples (row, col) pairs for the
    feature pass; n and m features equal those of the edge-list handle."""
    cc.load_default_scheduler()
    n, s, d = GRAPHS["grid64"](4)
    off, cols = gg.to_csr(n, s, d, symmetric=True)
    gc = cc.cc_init(n, off.cuda(), cols.cuda(), m=cols.numel(), id_bits=32, layout=cc.CC_CSR_NATIVE_SYM,
                    on_device=True)
    go = cc.cc_init(n, s.cuda(), d.cuda())
    fc, fo = cc.cc_graph_features(gc), cc.cc_graph_features(go)
    assert np.isfinite(fc).all()
    assert fc[0] == fo[0] and fc[1] == fo[1]  # log2(1 + n), log2(1 + m)
    assert abs(fc[3] - fo[3]) < 1.0  # max degree estimate, from another sample
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cc.cc_run(gc, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
    assert (out.cpu().numpy() == oracle.uf_labels(n, s, d)).all()
    cc.cc_free(gc)
    cc.cc_free(go)


def test_csr_rmat24_symmetric_full_size(cc):
    """R-MAT scale 24 stored symmetrically (nnz = 2^29 entries)."""
    n = 1 << 24
    s, d = gg.rmat(24, device="cuda")
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    off, cols = gg.to_csr(n, s, d, symmetric=True)
    del s, d
    torch.cuda.empty_cache()
    assert cols.numel() == 1 << 29
    g = cc.cc_init(n, off, cols, m=cols.numel(), id_bits=32, layout=cc.CC_CSR_NATIVE_SYM, on_device=True)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for order, mode in [(2, cc.CC_ASYNC), (0, cc.CC_ASYNC), (2, cc.CC_SYNC)]:
        out.fill_(-1)
        st = cc.cc_run(g, out, order, mode, 1)
        assert (out.cpu().numpy() == want).all(), (order, mode)
        assert st.sweeps < 40
    cc.cc_free(g)
