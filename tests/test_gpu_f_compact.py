"""GPU parity of CC_ASYNC_COMPACT: asynchronous full-chain sweeps that drop
the edges whose two chain walks ended at the same root.

The labels must still be the union-find labels (the unique fixed point), for
every graph family, seed and check interval, through both launch modes, and
after a run stopped at max_sweeps.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

FULL, COMPACT = 0, 2


@pytest.fixture(scope="module")
def cc():
    import paper_2311_02811_gb300 as lib
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return lib


GRAPHS = {
    "components64": lambda seed: gg.components64(seed=seed),
    "rmat12": lambda seed: (1 << 12, *gg.rmat(12, seed=seed)),
    "grid64": lambda seed: (64 * 64, *gg.grid(64, 64, seed=seed)),
    "path3001": lambda seed: (3001, *gg.path(3001, seed=seed)),
    "er": lambda seed: (5000, *gg.er(5000, 3000, seed=seed)),
    "caterpillar": lambda seed: (200 * 16, *gg.caterpillar(200, seed=seed)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_compact_matches_union_find(cc, name):
    for seed in range(10):
        n, s, d = GRAPHS[name](seed)
        want = oracle.uf_labels(n, s, d)
        g = cc.cc_init(n, s.cuda(), d.cuda())
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        for c in (1, 2, 4):
            out.fill_(-1)
            st = cc.cc_run(g, out, FULL, COMPACT, c)
            assert (out.cpu().numpy() == want).all(), (name, seed, c)
            assert st.check_interval == 1 and st.mode == COMPACT  # compaction checks every sweep
        cc.cc_free(g)


def test_compact_launch_modes_reorder_and_resume(cc):
    n, s, d = GRAPHS["rmat12"](5)
    want = oracle.uf_labels(n, s, d)
    g = cc.cc_init(n, s.cuda(), d.cuda())
    cc.cc_graph_reorder(g, cc.CC_REORDER_LOWDEG)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for launch in (cc.CC_LAUNCH_HOST, cc.CC_LAUNCH_GRAPH):
        cc.cc_graph_set_launch(g, launch)
        cc.cc_run(g, out, FULL, COMPACT, 1)
        assert (out.cpu().numpy() == want).all(), launch
    # stopped after one sweep: a valid partial state; a new run restarts the lists
    rc, st = cc.cc_run(g, out, FULL, COMPACT, 1, max_sweeps=1, raise_on_error=False)
    assert rc == cc.CC_ENOTCONVERGED and st.sweeps == 1
    lab = out.cpu().numpy()
    assert (lab <= np.arange(n)).all() and (lab >= 0).all()
    cc.cc_run(g, out, FULL, COMPACT, 1, init_labels=out.clone())
    assert (out.cpu().numpy() == want).all()
    cc.cc_free(g)


def test_compact_rejects_other_orders_and_layouts(cc):
    n, s, d = GRAPHS["grid64"](1)
    g = cc.cc_init(n, s.cuda(), d.cuda())
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for order in (1, 2, 4, cc.CC_ORDER_11MM):
        rc, _ = cc.cc_run(g, out, order, COMPACT, 1, raise_on_error=False)
        assert rc == cc.CC_EINVAL, order
    cc.cc_free(g)
    g = cc.cc_init(n, s.cuda().long(), d.cuda().long())
    out64 = torch.empty(n, dtype=torch.int64, device="cuda")
    rc, _ = cc.cc_run(g, out64, FULL, COMPACT, 1, raise_on_error=False)
    assert rc == cc.CC_EINVAL
    cc.cc_free(g)
    off, cols = gg.to_csr(n, s, d)
    g = cc.cc_init(n, off.cuda(), cols.cuda(), m=cols.numel(), id_bits=32, layout=cc.CC_CSR_NATIVE,
                   on_device=True)
    rc, _ = cc.cc_run(g, out, FULL, COMPACT, 1, raise_on_error=False)
    assert rc == cc.CC_EINVAL
    cc.cc_free(g)


def test_compact_edgeless_and_loops(cc):
    for s, d, n in (([], [], 9), ([3, 3, 5], [3, 3, 5], 7), ([1], [0], 2)):
        st_ = torch.tensor(s, dtype=torch.int32, device="cuda")
        dt_ = torch.tensor(d, dtype=torch.int32, device="cuda")
        g = cc.cc_init(n, st_, dt_)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        cc.cc_run(g, out, FULL, COMPACT, 1)
        assert (out.cpu().numpy() == oracle.uf_labels(n, s, d)).all()
        cc.cc_free(g)


@pytest.mark.parametrize("name", ["rmat24", "grid4096"])
def test_compact_full_size(cc, name):
    if name == "rmat24":
        n = 1 << 24
        s, d = gg.rmat(24, device="cuda")
    else:
        n = 4096 * 4096
        s, d = gg.grid(4096, 4096, device="cuda")
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    g = cc.cc_init(n, s, d)
    cc.cc_graph_reorder(g, cc.CC_REORDER_LOWDEG)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    # labels only: asynchronous sweep counts (and so the bytes a run moves)
    # depend on thread timing; bench.py reports compaction's bytes and time
    for mode in (cc.CC_ASYNC, COMPACT):
        out.fill_(-1)
        cc.cc_run(g, out, FULL, mode, 1)
        assert (out.cpu().numpy() == want).all(), mode
    cc.cc_free(g)
