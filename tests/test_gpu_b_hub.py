"""GPU parity of the hub-table sweep (edge lists reordered with CC_REORDER_HUB).

The labels of the highest-degree vertices are read from a shared-memory
table that is loaded from L at every sweep; synchronous sweeps must still
equal the Alg. 1 simulator after every sweep, asynchronous runs must end at
the union-find labels.
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


GRAPHS = {
    "rmat12": lambda seed: (1 << 12, *gg.rmat(12, seed=seed)),
    "rmat16": lambda seed: (1 << 16, *gg.rmat(16, seed=seed)),
    "caterpillar": lambda seed: (300 * 16, *gg.caterpillar(300, seed=seed)),  # backbone degree 17
    "dense_er": lambda seed: (200, *gg.er(200, 4000, seed=seed)),  # every vertex a hub
    "components64": lambda seed: gg.components64(seed=seed),
}


def hub_handle(cc, n, s, d):
    g = cc.cc_init(n, s.cuda(), d.cuda())
    cc.cc_graph_reorder(g, cc.CC_REORDER_HUB)
    return g


@pytest.mark.parametrize("name", ["rmat12", "rmat16", "caterpillar", "dense_er"])
def test_hub_table_present(cc, name):
    n, s, d = GRAPHS[name](0)
    g = hub_handle(cc, n, s, d)
    ptr, k = cc.cc_graph_hubs(g)
    deg = np.bincount(np.concatenate([s.numpy(), d.numpy()]), minlength=n)
    assert k == min(int((deg >= 16).sum()), 24576) and k > 0 and ptr != 0
    cc.cc_free(g)


@pytest.mark.parametrize("order", [1, 2, 4, 0])
@pytest.mark.parametrize("name", ["rmat12", "caterpillar", "dense_er", "components64"])
def test_hub_sync_every_sweep(cc, name, order):
    n, s, d = GRAPHS[name](1)
    h = 1024 if order == 0 else order
    _, it, conv, states = oracle.contour_sync(n, s, d, h, record=True)
    assert conv
    g = hub_handle(cc, n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for k in range(1, it + 1):
        rc, st = cc.cc_run(g, out, order, cc.CC_SYNC, 1, max_sweeps=k, raise_on_error=False)
        assert st.sweeps == k and (out.cpu().numpy() == states[k - 1]).all(), (name, order, k)
        assert rc == (cc.CC_OK if k == it else cc.CC_ENOTCONVERGED)
    cc.cc_free(g)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_hub_async_many_seeds(cc, name):
    for seed in range(8):
        n, s, d = GRAPHS[name](seed)
        want = oracle.uf_labels(n, s, d)
        g = hub_handle(cc, n, s, d)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        for order in (1, 2, 3, 4, 0, cc.CC_ORDER_11MM, cc.CC_ORDER_1M1M):
            for c in (1, 2):
                out.fill_(-1)
                cc.cc_run(g, out, order, cc.CC_ASYNC, c)
                assert (out.cpu().numpy() == want).all(), (name, seed, order, c)
        cc.cc_free(g)


def test_hub_features_equal_lowdeg_features(cc):
    """The feature pass decodes hub entries: a hub handle and a lowdeg handle
    of the same graph hold the same edges at the same positions."""
    n, s, d = GRAPHS["rmat16"](2)
    gh = hub_handle(cc, n, s, d)
    gl = cc.cc_init(n, s.cuda(), d.cuda())
    cc.cc_graph_reorder(gl, cc.CC_REORDER_LOWDEG)
    assert cc.cc_graph_hubs(gh)[1] > 0 and cc.cc_graph_hubs(gl)[1] == 0
    assert np.array_equal(cc.cc_graph_features(gh), cc.cc_graph_features(gl))
    cc.load_default_scheduler()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cc.cc_run(gh, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
    assert (out.cpu().numpy() == oracle.uf_labels(n, s, d)).all()
    cc.cc_free(gh)
    cc.cc_free(gl)


def test_hub_reorder_twice_rejected_and_no_hub_graphs(cc):
    n, s, d = GRAPHS["rmat12"](3)
    g = hub_handle(cc, n, s, d)
    with pytest.raises(cc.CCError) as ei:
        cc.cc_graph_reorder(g, cc.CC_REORDER_LOWDEG)
    assert ei.value.status == cc.CC_EINVAL
    cc.cc_free(g)
    # a grid has no vertex of degree >= 16: plain ids, plain sweep kernel
    n, s, d = 64 * 64, *gg.grid(64, 64, seed=4)
    g = hub_handle(cc, n, s, d)
    assert cc.cc_graph_hubs(g) == (0, 0) or cc.cc_graph_hubs(g)[1] == 0
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cc.cc_run(g, out, 2, cc.CC_ASYNC, 1)
    assert (out.cpu().numpy() == oracle.uf_labels(n, s, d)).all()
    cc.cc_free(g)


def test_hub_rmat24_full_size(cc):
    n = 1 << 24
    s, d = gg.rmat(24, device="cuda")
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    g = cc.cc_init(n, s, d)
    cc.cc_graph_reorder(g, cc.CC_REORDER_HUB)
    assert cc.cc_graph_hubs(g)[1] == 24576
    del s, d
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for order, mode in [(2, cc.CC_ASYNC), (4, cc.CC_ASYNC), (0, cc.CC_ASYNC), (2, cc.CC_SYNC)]:
        out.fill_(-1)
        st = cc.cc_run(g, out, order, mode, 1)
        assert (out.cpu().numpy() == want).all(), (order, mode)
        assert st.sweeps < 40
    cc.cc_free(g)
