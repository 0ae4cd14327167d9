"""GPU parity of the batched path (cc_batch_*) against the CPU oracle.

Every graph of a batch is checked on its own: labels (local ids) equal the
union-find labels of that graph; in synchronous mode the per-graph sweep count
equals the Alg. 1 simulator's iteration count as well.  Both execution paths
are covered: graphs solved whole in shared memory and graphs advanced round
by round through global memory (forced with the tuning override).
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


@pytest.fixture(scope="module")
def mix():
    """32 graphs of the batch mix (ER, path, grid, R-MAT), n in [300, 2e5]."""
    vo, eo, s, d, params = gg.batch_mix(32, seed=77, device="cuda", n_lo=300, n_hi=2e5)
    sh, dh = s.cpu().numpy(), d.cpu().numpy()
    truth = []
    for g in range(32):
        a, b = int(eo[g]), int(eo[g + 1])
        truth.append(oracle.uf_labels(int(vo[g + 1] - vo[g]), sh[a:b], dh[a:b]))
    return vo.numpy(), eo.numpy(), s, d, sh, dh, truth


def _check_labels(vo, labels, truth):
    lab = labels.cpu().numpy()
    for g, want in enumerate(truth):
        got = lab[vo[g]:vo[g + 1]]
        assert np.array_equal(got, want), f"graph {g}"


# (smem budget in bytes, threads, edges per thread): default split, all
# large, nearly all small
TUNINGS = [None, (0, 512, 4), (200 * 1024, 1024, 2)]


@pytest.mark.parametrize("tuning", TUNINGS, ids=["default", "all-large", "mostly-small"])
@pytest.mark.parametrize("order,mode,c", [(2, 1, 1), (2, 0, 1), (4, 1, 2), (0, 1, 1), (1, 1, 1),
                                          (3, 0, 2), (4, 0, 1)])
def test_batch_labels_match_oracle(cc, mix, tuning, order, mode, c):
    vo, eo, s, d, _, _, truth = mix
    b = cc.cc_batch_init(vo, eo, s, d)
    if tuning is not None:
        cc.cc_batch_set_tuning(b, *tuning)
    out = torch.full((int(vo[-1]),), -1, dtype=torch.int32, device="cuda")
    sweeps, ms = cc.cc_batch_run(b, out, order, mode, c)
    cc.cc_batch_free(b)
    _check_labels(vo, out, truth)
    assert (sweeps >= 1).all() and (sweeps % c == 0).all() and ms > 0


@pytest.mark.parametrize("tuning", TUNINGS, ids=["default", "all-large", "mostly-small"])
def test_batch_sync_sweeps_match_simulator(cc, mix, tuning):
    vo, eo, s, d, sh, dh, truth = mix
    want_sweeps = []
    for g in range(len(truth)):
        a, bnd = int(eo[g]), int(eo[g + 1])
        _, it, conv, _ = oracle.contour_sync(int(vo[g + 1] - vo[g]), sh[a:bnd], dh[a:bnd], 2)
        want_sweeps.append(it)
    b = cc.cc_batch_init(vo, eo, s, d)
    if tuning is not None:
        cc.cc_batch_set_tuning(b, *tuning)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    for rep in range(2):
        sweeps, _ = cc.cc_batch_run(b, out, 2, cc.CC_SYNC, 1)
        _check_labels(vo, out, truth)
        assert sweeps.tolist() == want_sweeps
    cc.cc_batch_free(b)


def test_batch_per_graph_schedules(cc, mix):
    vo, eo, s, d, _, _, truth = mix
    G = len(truth)
    rng = np.random.default_rng(5)
    order = rng.choice([1, 2, 3, 4, 0], G)
    mode = rng.integers(0, 2, G)
    c = rng.choice([1, 2, 4], G)
    b = cc.cc_batch_init(vo, eo, s, d)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    for tuning in TUNINGS[1:]:
        cc.cc_batch_set_tuning(b, *tuning)
        cc.cc_batch_set_schedule(b, order, mode, c)
        out.fill_(-1)
        sweeps, _ = cc.cc_batch_run_scheduled(b, out)
        _check_labels(vo, out, truth)
        assert (sweeps % c == 0).all()
    cc.cc_batch_free(b)


def test_batch_edge_cases(cc):
    # graphs: empty (n=0), isolated vertices (m=0), self-loops only, a path,
    # a single edge -- concatenated with local ids
    parts = [(0, [], []), (5, [], []), (4, [1, 3, 3], [1, 3, 3]), (6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5]),
             (2, [1], [0])]
    vo = np.cumsum([0] + [p[0] for p in parts])
    eo = np.cumsum([0] + [len(p[1]) for p in parts])
    s = torch.tensor(sum((p[1] for p in parts), []), dtype=torch.int32, device="cuda")
    d = torch.tensor(sum((p[2] for p in parts), []), dtype=torch.int32, device="cuda")
    truth = [oracle.uf_labels(p[0], p[1], p[2]) for p in parts]
    for tuning in TUNINGS:
        for mode in (0, 1):
            b = cc.cc_batch_init(vo, eo, s, d)
            if tuning is not None:
                cc.cc_batch_set_tuning(b, *tuning)
            out = torch.full((int(vo[-1]),), -1, dtype=torch.int32, device="cuda")
            sweeps, _ = cc.cc_batch_run(b, out, 2, mode, 1)
            cc.cc_batch_free(b)
            _check_labels(vo, out, truth)
            assert sweeps[1] == 1 and sweeps[2] == 1  # no edge lowers a label
    # one-shot form
    out = torch.full((int(vo[-1]),), -1, dtype=torch.int32, device="cuda")
    cc.cc_batch(vo, eo, s, d, out, 2, cc.CC_ASYNC, 1)
    _check_labels(vo, out, truth)


def test_batch_errors(cc):
    vo = np.array([0, 3, 6])
    eo = np.array([0, 2, 4])
    s = torch.tensor([0, 1, 0, 3], dtype=torch.int32, device="cuda")  # 3 is outside graph 1's [0, 3)
    d = torch.tensor([1, 2, 1, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as ei:
        cc.cc_batch_init(vo, eo, s, d)
    assert ei.value.status == cc.CC_EIDRANGE
    with pytest.raises(cc.CCError) as ei:
        cc.cc_batch_init(np.array([0, 3, 2]), eo, s, d)
    assert ei.value.status == cc.CC_EINVAL
    # max_sweeps: a long path cannot converge in 2 sweeps
    n = 5000
    ps, pd = gg.path(n, seed=3, device="cuda")
    b = cc.cc_batch_init(np.array([0, n]), np.array([0, n - 1]), ps, pd)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for tuning in TUNINGS[1:]:
        cc.cc_batch_set_tuning(b, *tuning)
        rc, sweeps, _ = cc.cc_batch_run(b, out, 2, cc.CC_ASYNC, 1, max_sweeps=2, raise_on_error=False)
        assert rc == cc.CC_ENOTCONVERGED and sweeps[0] == 2
    cc.cc_batch_free(b)


def test_batch_autotune_picks_valid_tuning(cc, mix):
    vo, eo, s, d, _, _, truth = mix
    b = cc.cc_batch_init(vo, eo, s, d, autotune=2)
    budget, threads, ept = cc.cc_batch_tuning(b)
    assert 0 <= budget <= 232448 and threads in (256, 512, 1024) and 1 <= ept <= 4
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    cc.cc_batch_run(b, out, 2, cc.CC_ASYNC, 1)
    cc.cc_batch_free(b)
    _check_labels(vo, out, truth)
    # a second plan of the same size mix reuses the cached tuning
    b2 = cc.cc_batch_init(vo, eo, s, d, autotune=1)
    assert cc.cc_batch_tuning(b2) == (budget, threads, ept)
    cc.cc_batch_free(b2)


def test_batch_reorder_keeps_every_graph(cc, mix):
    """cc_batch_reorder groups each graph's edges by its lower-degree endpoint;
    labels, and in sync mode every sweep count, are unchanged."""
    vo, eo, s, d, sh, dh, truth = mix
    want_sweeps = []
    for g in range(len(truth)):
        a, bnd = int(eo[g]), int(eo[g + 1])
        want_sweeps.append(oracle.contour_sync(int(vo[g + 1] - vo[g]), sh[a:bnd], dh[a:bnd], 2)[1])
    # tune and solve first: the reorder must not depend on the plan's history
    b = cc.cc_batch_init(vo, eo, s.clone(), d.clone(), autotune=1)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    cc.cc_batch_run(b, out, 2, cc.CC_ASYNC, 1)
    cc.cc_batch_reorder(b)
    for tuning in TUNINGS:
        if tuning is not None:
            cc.cc_batch_set_tuning(b, *tuning)
        for order, mode in [(2, 1), (0, 1), (4, 1)]:
            out.fill_(-1)
            cc.cc_batch_run(b, out, order, mode, 1)
            _check_labels(vo, out, truth)
        sweeps, _ = cc.cc_batch_run(b, out, 2, cc.CC_SYNC, 1)
        assert sweeps.tolist() == want_sweeps
        _check_labels(vo, out, truth)
    cc.cc_batch_free(b)


def test_batch_waves_keep_per_graph_sweeps(cc):
    """Twenty 10^6-vertex graphs: 80 MB of labels, more than one wave of the
    large-graph path (a wave holds at most 64 MB of labels).  Each graph's
    synchronous sweep count is counted from its own first sweep, so it must
    still equal the Alg. 1 simulator's, and every label the oracle's."""
    G, n = 20, 1_000_000
    graphs = [gg.er(n, 2 * n, seed=900 + g) for g in range(G)]
    vo = np.arange(G + 1, dtype=np.int64) * n
    eo = np.concatenate([[0], np.cumsum([s.numel() for s, _ in graphs])]).astype(np.int64)
    s = torch.cat([x for x, _ in graphs]).cuda()
    d = torch.cat([y for _, y in graphs]).cuda()
    b = cc.cc_batch_init(vo, eo, s, d)
    cc.cc_batch_set_tuning(b, 0, 512, 4)  # every graph on the large-graph path
    out = torch.empty(G * n, dtype=torch.int32, device="cuda")
    sweeps, _ = cc.cc_batch_run(b, out, 2, cc.CC_SYNC, 1)
    lab = out.cpu().numpy()
    for g, (gs, gd) in enumerate(graphs):
        want, it, conv, _ = oracle.contour_sync(n, gs, gd, 2)
        assert conv and sweeps[g] == it, (g, sweeps[g], it)
        assert np.array_equal(lab[g * n:(g + 1) * n], want), g
    for order in (2, 0):
        out.fill_(-1)
        cc.cc_batch_run(b, out, order, cc.CC_ASYNC, 1)
        lab = out.cpu().numpy()
        for g, (gs, gd) in enumerate(graphs):
            assert np.array_equal(lab[g * n:(g + 1) * n], oracle.uf_labels(n, gs, gd)), (order, g)
    cc.cc_batch_free(b)
