"""GPU parity of the CUDA path against the CPU oracle (needs a GB300).

Labels are integers, so every comparison is bit-exact:
* synchronous runs equal the Alg. 1 simulator state after every sweep and in
  their sweep count;
* asynchronous runs (whose intermediate states depend on thread timing) end
  at the unique fixed point, the union-find labels;
* the full-size R-MAT scale-24 and 4096 x 4096 grid graphs run in the launch
  configuration that bench.py times and are compared entry by entry.
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


def _gpu(x):
    return x.cuda() if x.device.type != "cuda" else x


def solve(cc, n, s, d, order=2, mode=1, c=1, max_sweeps=1 << 20, init=None, expect_ok=True):
    s, d = _gpu(s), _gpu(d)
    g = cc.cc_init(n, s, d)
    try:
        out = torch.empty(n, dtype=s.dtype, device="cuda")
        ini = None if init is None else torch.as_tensor(init, dtype=s.dtype).cuda()
        rc, st = cc.cc_run(g, out, order, mode, c, max_sweeps, init_labels=ini, raise_on_error=False)
    finally:
        cc.cc_free(g)
    if expect_ok:
        assert rc == cc.CC_OK, (rc, cc.cc_last_error())
    return out.cpu().numpy(), st, rc


SMALL = {
    "components64": lambda seed: gg.components64(seed=seed),
    "rmat12": lambda seed: (1 << 12, *gg.rmat(12, seed=seed)),
    "grid64": lambda seed: (64 * 64, *gg.grid(64, 64, seed=seed)),
    "path3001": lambda seed: (3001, *gg.path(3001, seed=seed)),
    "er": lambda seed: (5000, *gg.er(5000, 3000, seed=seed)),
    "caterpillar": lambda seed: (200 * 16, *gg.caterpillar(200, seed=seed)),
}


# ---------------------------------------------------------------------------
# synchronous mode: bit-exact per sweep against the Alg. 1 simulator
# ---------------------------------------------------------------------------

def test_components64_sync_order2_every_sweep(cc):
    """The 65,536-vertex, 64-component graph: order 2, synchronous, c = 1."""
    n, s, d = gg.components64()
    _, it, conv, states = oracle.contour_sync(n, s, d, 2, record=True)
    assert conv
    for k in range(1, it + 1):
        got, st, rc = solve(cc, n, s, d, 2, cc.CC_SYNC, 1, max_sweeps=k, expect_ok=False)
        assert st.sweeps == k
        assert (got == states[k - 1]).all(), k
        assert rc == (cc.CC_OK if k == it else cc.CC_ENOTCONVERGED)
    assert len(np.unique(got)) == 64


@pytest.mark.parametrize("order", [1, 2, 3, 4, 0])
@pytest.mark.parametrize("name", ["rmat12", "grid64", "path3001", "caterpillar"])
def test_sync_matches_simulator(cc, order, name):
    n, s, d = SMALL[name](1)
    h = 1024 if order == 0 else order
    want, it, conv, _ = oracle.contour_sync(n, s, d, h)
    got, st, _ = solve(cc, n, s, d, order, cc.CC_SYNC, 1)
    assert st.sweeps == it
    assert (got == want).all()


def test_sync_check_interval_blocks(cc):
    n, s, d = SMALL["grid64"](2)
    want, it, _, states = oracle.contour_sync(n, s, d, 2, record=True)
    for c in (2, 3, 4):
        got, st, _ = solve(cc, n, s, d, 2, cc.CC_SYNC, c)
        blocks = -(-it // c)
        assert st.sweeps == blocks * c
        assert (got == want).all()


# ---------------------------------------------------------------------------
# asynchronous mode: the unique fixed point
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(SMALL))
def test_async_all_orders_intervals_many_seeds(cc, name):
    seeds = range(20) if name not in ("components64",) else range(4)
    for seed in seeds:
        n, s, d = SMALL[name](seed)
        want = oracle.uf_labels(n, s, d)
        for order in (1, 2, 3, 4, 0):
            for c in (1, 2, 4):
                got, st, _ = solve(cc, n, s, d, order, cc.CC_ASYNC, c)
                assert (got == want).all(), (name, seed, order, c)
                assert st.sweeps % c == 0 and st.sweeps >= 1


def test_int64_ids(cc):
    for name in ("rmat12", "grid64", "components64"):
        n, s, d = SMALL[name](3)
        want = oracle.uf_labels(n, s, d)
        s64, d64 = s.to(torch.int64), d.to(torch.int64)
        for mode in (cc.CC_SYNC, cc.CC_ASYNC):
            for order in (2, 4, 0):
                got, st, _ = solve(cc, n, s64, d64, order, mode, 1)
                assert got.dtype == np.int64 and (got == want).all()
        sim, it, _, _ = oracle.contour_sync(n, s, d, 2)
        got, st, _ = solve(cc, n, s64, d64, 2, cc.CC_SYNC, 1)
        assert st.sweeps == it and (got == sim).all()


# ---------------------------------------------------------------------------
# input forms and error paths
# ---------------------------------------------------------------------------

def test_host_buffers_and_host_output(cc):
    n, s, d = SMALL["rmat12"](4)
    want = oracle.uf_labels(n, s, d)
    sn, dn = s.numpy(), d.numpy()
    g = cc.cc_init(n, sn, dn, on_device=False)
    out = np.empty(n, dtype=np.int32)
    st = cc.cc_run(g, out, 2, cc.CC_ASYNC, 1)
    cc.cc_free(g)
    assert (out == want).all() and st.sweeps >= 1 and st.solve_ms > 0


def test_unaligned_borrowed_edges_are_copied(cc):
    n, s, d = SMALL["grid64"](5)
    want = oracle.uf_labels(n, s[1:], d[1:])
    sg, dg = s.cuda(), d.cuda()
    got, _, _ = solve(cc, n, sg[1:], dg[1:], 2, cc.CC_ASYNC, 1)
    assert (got == want).all()


def test_csr_input(cc):
    n, s, d = SMALL["er"](6)
    sn, dn = s.numpy().astype(np.int64), d.numpy().astype(np.int64)
    rows = np.concatenate([sn, dn])
    cols = np.concatenate([dn, sn])
    order = np.argsort(rows, kind="stable")
    rows, cols = rows[order], cols[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, rows + 1, 1)
    off = np.cumsum(off)
    want = oracle.uf_labels(n, s, d)
    for on_dev in (False, True):
        offs = torch.from_numpy(off)
        col = torch.from_numpy(cols.astype(np.int32))
        if on_dev:
            offs, col = offs.cuda(), col.cuda()
        g = cc.cc_init(n, offs, col, m=len(cols), id_bits=32, layout=cc.CC_CSR, on_device=on_dev)
        assert cc.cc_graph_info(g) == (n, len(cols))
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        cc.cc_run(g, out, 2, cc.CC_ASYNC, 1)
        cc.cc_free(g)
        assert (out.cpu().numpy() == want).all()
    bad = off.copy()
    bad[3] = bad[4] + 1
    with pytest.raises(cc.CCError) as ei:
        cc.cc_init(n, torch.from_numpy(bad), torch.from_numpy(cols.astype(np.int32)),
                   m=len(cols), layout=cc.CC_CSR, on_device=False)
    assert ei.value.status == cc.CC_EINVAL


def test_out_of_range_ids_rejected(cc):
    s = torch.tensor([0, 1, 2, 7], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 2, 3, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as ei:
        cc.cc_init(5, s, d)
    assert ei.value.status == cc.CC_EIDRANGE
    with pytest.raises(cc.CCError) as ei:
        cc.cc_init(8, s, d - 1)
    assert ei.value.status == cc.CC_EIDRANGE


def test_empty_and_edgeless(cc):
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    g = cc.cc_init(0, e, e)
    cc.cc_run(g, e, 2, cc.CC_ASYNC, 1)
    cc.cc_free(g)
    for mode in (cc.CC_SYNC, cc.CC_ASYNC):
        got, st, _ = solve(cc, 1000, e, e, 2, mode, 1)
        assert (got == np.arange(1000)).all() and st.sweeps == 1
    s = torch.tensor([3, 3, 5], dtype=torch.int32)
    d = torch.tensor([3, 3, 5], dtype=torch.int32)  # self-loops only
    got, _, _ = solve(cc, 7, s, d, 2, cc.CC_ASYNC, 1)
    assert (got == np.arange(7)).all()


def test_max_sweeps_then_resume(cc):
    n, s, d = SMALL["path3001"](7)
    want = oracle.uf_labels(n, s, d)
    # synchronous: resuming from a stopped state continues the same sequence
    full, it, _, states = oracle.contour_sync(n, s, d, 2, record=True)
    part, st, rc = solve(cc, n, s, d, 2, cc.CC_SYNC, 1, max_sweeps=3, expect_ok=False)
    assert rc == cc.CC_ENOTCONVERGED and (part == states[2]).all()
    got, st, _ = solve(cc, n, s, d, 2, cc.CC_SYNC, 1, init=part)
    assert st.sweeps == it - 3 and (got == want).all()
    # asynchronous: any valid snapshot converges to the same fixed point
    part, st, rc = solve(cc, n, s, d, 2, cc.CC_ASYNC, 1, max_sweeps=2, expect_ok=False)
    assert rc == cc.CC_ENOTCONVERGED
    got, _, _ = solve(cc, n, s, d, 2, cc.CC_ASYNC, 1, init=part)
    assert (got == want).all()
    # a snapshot with L[x] > x is refused before any sweep
    bad = np.arange(n, dtype=np.int32)
    bad[5] = 9
    _, _, rc = solve(cc, n, s, d, 2, cc.CC_ASYNC, 1, init=bad, expect_ok=False)
    assert rc == cc.CC_EINVAL


def test_bad_arguments(cc):
    n, s, d = SMALL["rmat12"](8)
    s, d = s.cuda(), d.cuda()
    g = cc.cc_init(n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for args in [(2000, 1, 1), (2, 5, 1), (2, 1, 0), (2, 1, 65)]:
        rc, _ = cc.cc_run(g, out, *args, raise_on_error=False)
        assert rc == cc.CC_EINVAL, args
    rc, _ = cc.cc_run(g, out, 2, 1, 1, max_sweeps=0, raise_on_error=False)
    assert rc == cc.CC_EINVAL
    cc.cc_free(g)


def test_repeated_runs_reuse_handle(cc):
    n, s, d = SMALL["grid64"](9)
    want = oracle.uf_labels(n, s, d)
    g = cc.cc_init(n, s.cuda(), d.cuda())  # the handle keeps the borrowed device copies alive
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]
    for rep in range(4):
        for o in outs:
            for mode in (cc.CC_SYNC, cc.CC_ASYNC):
                o.fill_(-1)
                cc.cc_run(g, o, 2, mode, 1)
                assert (o.cpu().numpy() == want).all()
    cc.cc_free(g)


# ---------------------------------------------------------------------------
# full sizes (the bench workload)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def rmat24():
    s, d = gg.rmat(24, device="cuda")
    return 1 << 24, s, d


def test_rmat24_full_size(cc, rmat24):
    n, s, d = rmat24
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    for order, mode in [(2, cc.CC_ASYNC), (4, cc.CC_ASYNC), (2, cc.CC_SYNC), (4, cc.CC_SYNC)]:
        got, st, _ = solve(cc, n, s, d, order, mode, 1)
        assert (got == want).all(), (order, mode)
        assert st.sweeps < 40


def test_grid4096_full_size(cc):
    n = 4096 * 4096
    s, d = gg.grid(4096, 4096, device="cuda")
    assert abs(s.numel() - 0.95 * 33546240) < 20000
    want = oracle.uf_labels(n, s.cpu(), d.cpu())
    for order, mode in [(2, cc.CC_ASYNC), (4, cc.CC_ASYNC), (2, cc.CC_SYNC), (4, cc.CC_SYNC)]:
        got, st, _ = solve(cc, n, s, d, order, mode, 1)
        assert (got == want).all(), (order, mode)


@pytest.mark.parametrize("method", [1, 2, 3], ids=["src", "lowdeg", "hub"])
def test_reorder_keeps_labels_and_sync_sequence(cc, method):
    """Edge order is a layout choice: labels (and, in sync mode, every state
    and the sweep count) are those of the original edge list."""
    for name in ("rmat12", "grid64", "components64", "path3001", "caterpillar"):
        n, s, d = SMALL[name](2)
        want = oracle.uf_labels(n, s, d)
        sim, it, _, _ = oracle.contour_sync(n, s, d, 2)
        sg, dg = s.cuda(), d.cuda()
        g = cc.cc_init(n, sg, dg)
        cc.cc_graph_reorder(g, method)
        del sg, dg  # the handle owns its reordered copy
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        for order in (2, 4, 0):
            for c in (1, 2):
                cc.cc_run(g, out, order, cc.CC_ASYNC, c)
                assert (out.cpu().numpy() == want).all(), (name, order, c)
        st = cc.cc_run(g, out, 2, cc.CC_SYNC, 1)
        assert st.sweeps == it and (out.cpu().numpy() == sim).all()
        cc.cc_free(g)


@pytest.mark.parametrize("sched", ["11mm", "1m1m"])
def test_per_iteration_order_schedules(cc, sched):
    """C-11mm and C-1m1m (Section III-B4): in sync mode every sweep equals the
    Alg. 1 simulator run one iteration at a time with the scheduled order."""
    code = cc.CC_ORDER_11MM if sched == "11mm" else cc.CC_ORDER_1M1M
    for name in ("rmat12", "grid64", "path3001", "components64", "caterpillar"):
        n, s, d = SMALL[name](3)
        want = oracle.uf_labels(n, s, d)
        L, k = None, 0
        while True:
            one = (k < 2) if sched == "11mm" else (k % 2 == 0)
            L, _, conv, _ = oracle.contour_sync(n, s, d, 1 if one else 1024, max_iters=1, init=L)
            k += 1
            if conv:
                break
        got, st, _ = solve(cc, n, s, d, code, cc.CC_SYNC, 1)
        assert st.sweeps == k and (got == L).all(), (name, st.sweeps, k)
        for c in (1, 4):  # the interval is ignored: schedules check every sweep
            got, st, _ = solve(cc, n, s, d, code, cc.CC_ASYNC, c)
            assert (got == want).all() and st.check_interval == 1


def test_generators_bit_identical_on_gpu():
    """The seeded generators produce the same graphs on the GPU as on the CPU."""
    makers = [lambda dev: gg.rmat(14, device=dev), lambda dev: gg.grid(90, 110, device=dev),
              lambda dev: gg.delaunay_like(13, device=dev)[1:], lambda dev: gg.er(9000, 30000, device=dev),
              lambda dev: gg.caterpillar(500, device=dev), lambda dev: gg.components64(device=dev)[1:]]
    for make in makers:
        a, b = make("cpu")
        c, d = make("cuda")
        assert torch.equal(a, c.cpu()) and torch.equal(b, d.cpu())
    v1, e1, s1, d1, _ = gg.batch_mix(16, device="cpu", n_hi=2e4)
    v2, e2, s2, d2, _ = gg.batch_mix(16, device="cuda", n_hi=2e4)
    assert torch.equal(v1, v2) and torch.equal(e1, e2)
    assert torch.equal(s1, s2.cpu()) and torch.equal(d1, d2.cpu())


def test_non_default_streams_and_concurrent_handles(cc):
    """Handles enqueue on the stream they were created with (or set later);
    two handles on two streams run concurrently and stay correct."""
    graphs = [SMALL["rmat12"](11), SMALL["grid64"](12)]
    wants = [oracle.uf_labels(n, s, d) for n, s, d in graphs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    handles, outs, keep = [], [], []
    for (n, s, d), st in zip(graphs, streams):
        with torch.cuda.stream(st):
            sg, dg = s.cuda(), d.cuda()
            keep.append((sg, dg))
            handles.append(cc.cc_init(n, sg, dg, stream=st.cuda_stream))
            outs.append(torch.empty(n, dtype=torch.int32, device="cuda"))
    for rep in range(3):
        for h, o, st in zip(handles, outs, streams):
            with torch.cuda.stream(st):
                cc.cc_run(h, o, 0 if rep % 2 else 2, cc.CC_ASYNC, 1)
    torch.cuda.synchronize()
    for o, want in zip(outs, wants):
        assert (o.cpu().numpy() == want).all()
    cc.cc_graph_set_stream(handles[0], streams[1].cuda_stream)
    with torch.cuda.stream(streams[1]):
        cc.cc_run(handles[0], outs[0], 2, cc.CC_SYNC, 1)
    torch.cuda.synchronize()
    assert (outs[0].cpu().numpy() == wants[0]).all()
    for h in handles:
        cc.cc_free(h)


@pytest.mark.parametrize("layout", ["coo", "hub", "csr"])
def test_host_polled_launch_matches_graph_launch(cc, layout):
    """CC_LAUNCH_HOST runs the same blocks from the host: identical labels,
    sweep counts and (sync, stopped early) intermediate states."""
    n, s, d = SMALL["rmat12"](7)
    if layout == "csr":
        off, cols = gg.to_csr(n, s, d, symmetric=True)
        g = cc.cc_init(n, off.cuda(), cols.cuda(), m=cols.numel(), id_bits=32,
                       layout=cc.CC_CSR_NATIVE_SYM, on_device=True)
    else:
        g = cc.cc_init(n, s.cuda(), d.cuda())
        if layout == "hub":
            cc.cc_graph_reorder(g, cc.CC_REORDER_HUB)
    want = oracle.uf_labels(n, s, d)
    _, it, _, states = oracle.contour_sync(n, s, d, 2, record=True)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for launch in (cc.CC_LAUNCH_HOST, cc.CC_LAUNCH_GRAPH, cc.CC_LAUNCH_HOST):
        cc.cc_graph_set_launch(g, launch)
        for order, mode, c in [(2, cc.CC_ASYNC, 1), (0, cc.CC_ASYNC, 2), (cc.CC_ORDER_1M1M, cc.CC_ASYNC, 1)]:
            cc.cc_run(g, out, order, mode, c)
            assert (out.cpu().numpy() == want).all(), (launch, order, mode, c)
        for k in (1, 2, it):
            rc, st = cc.cc_run(g, out, 2, cc.CC_SYNC, 1, max_sweeps=k, raise_on_error=False)
            assert st.sweeps == k and (out.cpu().numpy() == states[k - 1]).all(), (launch, k)
    with pytest.raises(cc.CCError):
        cc.cc_graph_set_launch(g, 7)
    cc.cc_free(g)
