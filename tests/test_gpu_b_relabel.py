"""GPU parity of the renumbered layout (cc_graph_reorder with CC_REORDER_DEGREE).

The handle renumbers the vertices in order of decreasing degree, runs the
sweeps on the renumbered graph and maps the labels back.  Checked here:
- the renumbering is the one the header defines (a stable sort by degree);
- asynchronous runs of every order end at the union-find labels;
- synchronous runs equal, after every sweep, the Alg. 1 simulator run on the
  renumbered graph, mapped back tree by tree (each tree labelled by its
  smallest original id; at convergence that is the component minimum);
- resume from snapshots of either layout, host output, full-size R-MAT 24.
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
    "caterpillar": lambda seed: (300 * 16, *gg.caterpillar(300, seed=seed)),
    "dense_er": lambda seed: (200, *gg.er(200, 4000, seed=seed)),  # every vertex in the shared-memory prefix
    "components64": lambda seed: gg.components64(seed=seed),
    "grid64": lambda seed: (64 * 64, *gg.grid(64, 64, seed=seed)),  # no vertex of degree >= 16
    "path3001": lambda seed: (3001, *gg.path(3001, seed=seed)),
}


class _Dev:
    """A device int32 array given by pointer, for torch.as_tensor."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 3}


def renumbering(n, s, d):
    """perm[x] = new id of x: decreasing degree, equal degrees by increasing id."""
    deg = np.bincount(s, minlength=n) + np.bincount(d, minlength=n)
    inv = np.argsort(-deg, kind="stable")
    perm = np.empty(n, dtype=np.int64)
    perm[inv] = np.arange(n)
    return perm, inv


def to_caller_ids(state, perm, inv):
    """A label state on the new ids -> caller ids: every tree labelled by the
    smallest original id among its members."""
    r = state.astype(np.int64)
    while True:
        nxt = r[r]
        if np.array_equal(nxt, r):
            break
        r = nxt
    tree_min = np.full(len(r), np.iinfo(np.int64).max)
    np.minimum.at(tree_min, r, inv)
    return tree_min[r[perm]].astype(np.int32)


def relabelled(cc, n, s, d):
    g = cc.cc_init(n, s.cuda(), d.cuda())
    cc.cc_graph_reorder(g, cc.CC_REORDER_DEGREE)
    return g


@pytest.mark.parametrize("name", ["rmat12", "rmat16", "caterpillar", "dense_er", "grid64"])
def test_renumbering_is_the_degree_order(cc, name):
    n, s, d = GRAPHS[name](0)
    g = relabelled(cc, n, s, d)
    pp, ip = cc.cc_graph_perm(g)
    perm = torch.as_tensor(_Dev(pp, n), device="cuda").cpu().numpy()
    inv = torch.as_tensor(_Dev(ip, n), device="cuda").cpu().numpy()
    want_perm, want_inv = renumbering(n, s.numpy(), d.numpy())
    assert np.array_equal(perm, want_perm) and np.array_equal(inv, want_inv)
    deg = np.bincount(s.numpy(), minlength=n) + np.bincount(d.numpy(), minlength=n)
    ptr, k = cc.cc_graph_hubs(g)
    assert ptr is None and k == min(int((deg >= 16).sum()), 24576)
    # stored edges: new ids, larger first, sorted by the larger
    a, b = cc.cc_graph_edges(g)
    m = s.numel()
    w = torch.as_tensor(_Dev(a, m), device="cuda").cpu().numpy()
    v = torch.as_tensor(_Dev(b, m), device="cuda").cpu().numpy()
    ps, pd = want_perm[s.numpy()], want_perm[d.numpy()]
    assert (w >= v).all() and (np.diff(w) >= 0).all()
    got = np.sort(w.astype(np.int64) * n + v)
    exp = np.sort(np.maximum(ps, pd) * n + np.minimum(ps, pd))
    assert np.array_equal(got, exp)
    # the caller's edge arrays are untouched, the handle keeps its own
    g2 = cc.cc_init(n, s.cuda(), d.cuda())
    assert cc.cc_graph_perm(g2) == (None, None)
    cc.cc_free(g2)
    cc.cc_free(g)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 0, -2, -3])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_relabel_async_matches_union_find(cc, name, order):
    for seed in range(3):
        n, s, d = GRAPHS[name](seed)
        want = oracle.uf_labels(n, s, d)
        g = relabelled(cc, n, s, d)
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        for c in (1, 2):
            if order < 0 and c > 1:
                continue
            out.fill_(-1)
            cc.cc_run(g, out, order, cc.CC_ASYNC, c)
            assert np.array_equal(out.cpu().numpy(), want), (name, order, seed, c)
        cc.cc_free(g)


@pytest.mark.parametrize("order", [1, 2, 4, 0])
@pytest.mark.parametrize("name", ["rmat12", "caterpillar", "dense_er", "components64", "grid64"])
def test_relabel_sync_every_sweep(cc, name, order):
    n, s, d = GRAPHS[name](1)
    h = 1024 if order == 0 else order
    perm, inv = renumbering(n, s.numpy(), d.numpy())
    ps = torch.from_numpy(perm[s.numpy()].astype(np.int32))
    pd = torch.from_numpy(perm[d.numpy()].astype(np.int32))
    _, it, conv, states = oracle.contour_sync(n, ps, pd, h, record=True)
    assert conv
    g = relabelled(cc, n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for k in range(1, it + 1):
        rc, st = cc.cc_run(g, out, order, cc.CC_SYNC, 1, max_sweeps=k, raise_on_error=False)
        assert st.sweeps == k
        assert np.array_equal(out.cpu().numpy(), to_caller_ids(states[k - 1], perm, inv)), (name, order, k)
        assert rc == (cc.CC_OK if k == it else cc.CC_ENOTCONVERGED)
    assert np.array_equal(out.cpu().numpy(), oracle.uf_labels(n, s, d))
    cc.cc_free(g)


def test_relabel_resume_and_host_output(cc):
    n, s, d = GRAPHS["rmat16"](2)
    want = oracle.uf_labels(n, s, d)
    g = relabelled(cc, n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        rc, st = cc.cc_run(g, out, 2, mode, 1, max_sweeps=1, raise_on_error=False)
        assert rc == cc.CC_ENOTCONVERGED
        snap = out.cpu().numpy()
        assert (snap >= 0).all() and (snap <= np.arange(n)).all()
        cc.cc_run(g, out, 2, mode, 1, init_labels=out.clone())
        assert np.array_equal(out.cpu().numpy(), want), mode
    # a snapshot of the plain layout (Alg. 1 after 2 iterations) resumes too
    _, _, _, states = oracle.contour_sync(n, s, d, 2, max_iters=2, record=True)
    snap = torch.from_numpy(states[-1].copy())
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        cc.cc_run(g, out, 2, mode, 1, init_labels=snap)
        assert np.array_equal(out.cpu().numpy(), want), mode
    # host output and host snapshot
    host = np.full(n, -1, dtype=np.int32)
    cc.cc_run(g, host, 0, cc.CC_ASYNC, 1, init_labels=snap.numpy())
    assert np.array_equal(host, want)
    # an invalid snapshot is refused before any gather
    bad = snap.clone()
    bad[5] = n - 1
    with pytest.raises(cc.CCError) as ei:
        cc.cc_run(g, out, 2, cc.CC_ASYNC, 1, init_labels=bad)
    assert ei.value.status == cc.CC_EINVAL
    cc.cc_free(g)


def test_relabel_rejections_and_auto(cc):
    n, s, d = GRAPHS["rmat12"](3)
    g = relabelled(cc, n, s, d)
    for method in (cc.CC_REORDER_HUB, cc.CC_REORDER_DEGREE, cc.CC_REORDER_LOWDEG):
        with pytest.raises(cc.CCError) as ei:
            cc.cc_graph_reorder(g, method)
        assert ei.value.status == cc.CC_EINVAL
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as ei:
        cc.cc_run(g, out, cc.CC_ORDER_FULL, cc.CC_ASYNC_COMPACT, 1)
    assert ei.value.status == cc.CC_EINVAL
    cc.load_default_scheduler()
    try:
        cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
    finally:
        cc.unload_scheduler()
    assert np.array_equal(out.cpu().numpy(), oracle.uf_labels(n, s, d))
    for launch in (cc.CC_LAUNCH_HOST, cc.CC_LAUNCH_GRAPH):
        cc.cc_graph_set_launch(g, launch)
        out.fill_(-1)
        cc.cc_run(g, out, 2, cc.CC_SYNC, 1)
        assert np.array_equal(out.cpu().numpy(), oracle.uf_labels(n, s, d))
    cc.cc_free(g)
    # a graph without edges is left as it is
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    g = cc.cc_init(10, e, e)
    cc.cc_graph_reorder(g, cc.CC_REORDER_DEGREE)
    o = torch.empty(10, dtype=torch.int32, device="cuda")
    cc.cc_run(g, o, 2, cc.CC_ASYNC, 1)
    assert np.array_equal(o.cpu().numpy(), np.arange(10))
    cc.cc_free(g)


def test_relabel_rmat24_full_size(cc):
    n = 1 << 24
    s, d = gg.rmat(24, device="cuda")
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    g = cc.cc_init(n, s, d)
    cc.cc_graph_reorder(g, cc.CC_REORDER_DEGREE)
    del s, d
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for order, mode in [(2, cc.CC_ASYNC), (4, cc.CC_ASYNC), (0, cc.CC_ASYNC), (2, cc.CC_SYNC)]:
        out.fill_(-1)
        st = cc.cc_run(g, out, order, mode, 1)
        assert np.array_equal(out.cpu().numpy(), want), (order, mode)
        assert st.sweeps < 40
    cc.cc_free(g)
