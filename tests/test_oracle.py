"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: brute-force
reachability, closed forms derived from Def. 1-3 and Alg. 1, the iteration
bounds of Lemma 2 and the Theorem, invariants stated in Section II, and
constructed graphs whose components are known in advance.
"""
import itertools
import math
import os

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# brute force on every graph with n <= 6
# ---------------------------------------------------------------------------

def _closure_labels(n, edges):
    """label[v] = min reachable id, by boolean transitive closure."""
    R = np.eye(n, dtype=bool)
    for a, b in edges:
        R[a, b] = R[b, a] = True
    for k in range(n):  # Warshall
        R = R | (R[:, [k]] & R[[k], :])
    return np.array([np.flatnonzero(R[v]).min() for v in range(n)], dtype=np.int64)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_all_small_graphs_against_closure(oracle_lib, n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        want = _closure_labels(n, edges)
        src = np.array([e[0] for e in edges], dtype=np.int32)
        dst = np.array([e[1] for e in edges], dtype=np.int32)
        # random orientation so the operator sees both directions
        flip = (mask * 2654435761 >> 7) & ((1 << len(edges)) - 1) if edges else 0
        for i in range(len(edges)):
            if flip >> i & 1:
                src[i], dst[i] = dst[i], src[i]
        assert (oracle.uf_labels(n, src, dst) == want).all(), (n, edges)
        if mask % 17 == 0 or n <= 4:
            assert (oracle.bfs_labels(n, src, dst) == want).all(), (n, edges)
        if mask % 7 == 0 or n <= 4:
            for h in (1, 2, 4):
                L, it, conv, _ = oracle.contour_sync(n, src, dst, h)
                assert conv and (L == want).all(), (n, edges, h)


def test_self_loops_and_duplicates_brute_force(oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 14))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        want = _closure_labels(n, list(zip(src.tolist(), dst.tolist())))
        assert (oracle.uf_labels(n, src, dst) == want).all()
        assert (oracle.bfs_labels(n, src, dst) == want).all()
        for h in (1, 2, 3, 1024):
            L, it, conv, _ = oracle.contour_sync(n, src, dst, h)
            assert conv and (L == want).all()


# ---------------------------------------------------------------------------
# union-find against BFS on the generator families
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("family", ["rmat", "grid", "er", "path", "caterpillar"])
def test_uf_equals_bfs(oracle_lib, family):
    for seed in range(3):
        if family == "rmat":
            n, (s, d) = 1 << 11, gg.rmat(11, seed=seed)
        elif family == "grid":
            n, (s, d) = 40 * 50, gg.grid(40, 50, seed=seed)
        elif family == "er":
            n, (s, d) = 3000, gg.er(3000, 2500, seed=seed)
        elif family == "path":
            n, (s, d) = 777, gg.path(777, seed=seed)
        else:
            n, (s, d) = 64 * 16, gg.caterpillar(64, seed=seed)
        a = oracle.uf_labels(n, s, d)
        b = oracle.bfs_labels(n, s, d)
        assert (a == b).all()
        a64 = oracle.uf_labels(n, s.to(torch.int64), d.to(torch.int64), id_bits=64)
        assert (a64 == a).all()


def test_oracle_rejects_out_of_range_ids(oracle_lib):
    with pytest.raises(oracle.OracleIdError) as ei:
        oracle.uf_labels(4, [0, 1, 4], [1, 2, 3])
    assert ei.value.edge == 2
    with pytest.raises(oracle.OracleIdError):
        oracle.uf_labels(4, [0, -1], [1, 2])


def test_empty_graphs(oracle_lib):
    assert oracle.uf_labels(0, [], []).size == 0
    assert (oracle.uf_labels(5, [], []) == np.arange(5)).all()
    L, it, conv, _ = oracle.contour_sync(5, [], [], 2)
    assert conv and it == 1 and (L == np.arange(5)).all()


# ---------------------------------------------------------------------------
# constructed graphs with known components
# ---------------------------------------------------------------------------

def test_components64_labels_known_from_permutation(oracle_lib):
    n, s, d = gg.components64()
    assert n == 65536 and s.numel() == 294880
    # the generator's vertex relabelling, reproduced from its seed
    perm = gg._random_rank(gg.stream_key(gg.BASE_SEED, 101), n, "cpu").numpy()
    comp = np.arange(n) // 1024
    new_ids = perm.reshape(64, 1024)
    comp_min = new_ids.min(axis=1)
    want = np.empty(n, dtype=np.int64)
    want[perm] = comp_min[comp]
    got = oracle.uf_labels(n, s, d)
    assert (got == want).all()
    assert len(np.unique(got)) == 64


@pytest.mark.parametrize("maker", ["path", "caterpillar", "grid_full"])
def test_connected_families_label_zero(oracle_lib, maker):
    if maker == "path":
        n, (s, d) = 5000, gg.path(5000)
    elif maker == "caterpillar":
        n, (s, d) = 300 * 16, gg.caterpillar(300)
    else:
        n, (s, d) = 30 * 31, gg.grid(30, 31, p_drop=0)
    assert (oracle.uf_labels(n, s, d) == 0).all()
    L, it, conv, _ = oracle.contour_sync(n, s, d, 2)
    assert conv and (L == 0).all()


# ---------------------------------------------------------------------------
# Alg. 1 simulator: closed forms, worked example, bounds, invariants
# ---------------------------------------------------------------------------

def test_golden_hand_worked_path5(oracle_lib):
    with open(os.path.join(GOLDEN, "path5_mm2_sync.txt")) as f:
        lines = [ln.split("#")[0].strip() for ln in f]
    lines = [ln for ln in lines if ln]
    head = lines[0].split("|")
    n = int(head[0].split()[1])
    src = [int(x) for x in head[1].split()]
    dst = [int(x) for x in head[2].split()]
    want = np.array([[int(x) for x in ln.split()] for ln in lines[1:]])
    L, it, conv, states = oracle.contour_sync(n, src, dst, 2, record=True)
    assert conv and it == len(want)
    assert (states == want).all()


@pytest.mark.parametrize("h", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [2, 3, 17, 100, 1000])
def test_sorted_path_closed_form(oracle_lib, h, n):
    """On the path 0-1-..-(n-1) every state is L_k[x] = max(0, x - d_k).

    From Def. 3: vertex x is lowered through the edge <x-1, x> to
    L^h_{k-1}[x-1] = x-1-h*d_{k-1}, and no other edge reaches lower, so
    d_k = h*d_{k-1} + 1, d_0 = 0.  The do-while of Alg. 1 ends one iteration
    after d_k first reaches n-1.
    """
    src, dst = gg.path(n, permute=False)
    L, it, conv, states = oracle.contour_sync(n, src, dst, h, record=True)
    x = np.arange(n)
    dk = 0
    for k in range(1, it + 1):
        dk = h * dk + 1
        assert (states[k - 1] == np.maximum(0, x - dk)).all(), (k, h, n)
    dk, k_conv = 0, 0
    while dk < n - 1:
        dk = h * dk + 1
        k_conv += 1
    assert conv and it == k_conv + 1


def _lemma2_bound(d):
    """ceil(log_1.5 d) + 1 (Lemma 2 / Theorem), d >= 1."""
    if d <= 1:
        return 1
    return math.ceil(math.log(d) / math.log(1.5) - 1e-12) + 1


@pytest.mark.parametrize("n", [2, 3, 5, 9, 33, 100, 257, 1024, 4097])
def test_lemma2_path_bound_sync_mm2(oracle_lib, n):
    """Lemma 2: a path needs at most ceil(log_1.5(n-1))+1 changing iterations.

    The simulator counts the final no-change iteration of Alg. 1's do-while
    as well, hence the +1.
    """
    for seed in range(12):
        src, dst = gg.path(n, seed=seed)
        L, it, conv, _ = oracle.contour_sync(n, src, dst, 2)
        assert conv and (L == 0).all()
        assert it <= _lemma2_bound(n - 1) + 1, (n, seed, it)


def test_theorem_bound_on_grids_sync_mm2(oracle_lib):
    """Theorem (Graph Convergence): at most ceil(log_1.5 d_max)+1 iterations."""
    for rows, cols in [(2, 40), (7, 9), (20, 20), (3, 300)]:
        for seed in range(4):
            s, d = gg.grid(rows, cols, p_drop=0, seed=seed)
            L, it, conv, _ = oracle.contour_sync(rows * cols, s, d, 2)
            assert conv and (L == 0).all()
            assert it <= _lemma2_bound(rows + cols - 2) + 1


def test_sync_invariants_per_iteration(oracle_lib):
    """Per-iteration facts that follow from Def. 1-3 and Section II-C.

    * labels never increase (Def. 1 only lowers);
    * L[x] <= x and L[x] lies in x's component;
    * MMS(k)^1 >= MMS(k)^2 >= MMS(k+1)^1 (Def. 5 and the remark after it);
    * the final state is the union-find answer.
    """
    for maker in range(4):
        if maker == 0:
            n, s, d = gg.components64()
        elif maker == 1:
            n, (s, d) = 1 << 12, gg.rmat(12, seed=3)
        elif maker == 2:
            n, (s, d) = 60 * 70, gg.grid(60, 70, seed=5)
        else:
            n, (s, d) = 2000, gg.er(2000, 1100, seed=9)
        truth = oracle.uf_labels(n, s, d)
        for h in (2, 4):
            L, it, conv, states = oracle.contour_sync(n, s, d, h, record=True)
            assert conv and (L == truth).all()
            prev = np.arange(n)
            for k in range(it):
                cur = states[k]
                assert (cur <= prev).all()
                assert (cur <= np.arange(n)).all()
                assert (truth[cur] == truth).all()
                mms1_prev = set(np.unique(prev).tolist())
                mms2_prev = set(np.unique(prev[prev]).tolist())
                mms1_cur = set(np.unique(cur).tolist())
                assert mms2_prev <= mms1_prev and mms1_cur <= mms2_prev
                prev = cur


def test_order_one_is_label_propagation(oracle_lib):
    """Section II-C: MM^1 is label propagation -- each vertex takes the minimum
    of its own and its neighbours' labels every iteration."""
    n, (s, d) = 500, gg.er(500, 700, seed=2)
    _, it, conv, states = oracle.contour_sync(n, s, d, 1, record=True)
    s_np, d_np = s.numpy().astype(np.int64), d.numpy().astype(np.int64)
    L = np.arange(n)
    for k in range(it):
        nxt = L.copy()
        np.minimum.at(nxt, s_np, L[d_np])
        np.minimum.at(nxt, d_np, L[s_np])
        assert (states[k] == nxt).all()
        L = nxt


def test_iteration_order_relation(oracle_lib):
    """Section IV-C: iterations(C-m) <= iterations(C-2) <= iterations(C-1).

    The paper observes this on its graphs; here it is checked on the
    long-diameter families, summed over seeds.
    """
    tot = {1: 0, 2: 0, 1024: 0}
    for seed in range(5):
        for n, (s, d) in [(400, gg.path(400, seed=seed)), (30 * 30, gg.grid(30, 30, seed=seed)),
                          (40 * 16, gg.caterpillar(40, seed=seed))]:
            for h in tot:
                _, it, conv, _ = oracle.contour_sync(n, s, d, h)
                assert conv
                tot[h] += it
    assert tot[1024] <= tot[2] <= tot[1]


def test_resume_from_snapshot_same_fixed_point(oracle_lib):
    """A partial state obeying L[x] <= x, L[x] in x's component converges to the
    same unique fixed point (stars at the component minimum)."""
    n, (s, d) = 3000, gg.er(3000, 2600, seed=11)
    truth = oracle.uf_labels(n, s, d)
    for k in (1, 2, 3):
        part, it, conv, _ = oracle.contour_sync(n, s, d, 2, max_iters=k)
        assert it == k
        L, _, conv, _ = oracle.contour_sync(n, s, d, 2, init=part)
        assert conv and (L == truth).all()


def test_generator_cpu_is_splitmix64():
    key = gg.stream_key(gg.BASE_SEED, 1)
    got = gg.uniform64(key, 5, 50).tolist()
    want = [gg.mix64_int(key + (i + 1) * 0x9E3779B97F4A7C15) for i in range(5, 55)]
    assert [g & ((1 << 64) - 1) for g in got] == want
    # published SplitMix64 first output for seed 0 (state += gamma, then mix)
    assert gg.mix64_int(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_degree_features_plain(oracle_lib):
    f = oracle.degree_features(4, [0, 0, 1, 2], [1, 2, 2, 2])
    # degrees: 0->2, 1->2, 2->4 (self-loop counts twice), 3->0
    assert f["m"] == 4 and f["deg_max"] == 4.0
    assert f["deg_mean"] == 2.0 and f["deg_var"] == 2.0


# ---------------------------------------------------------------------------
# the multicore asynchronous Contour baseline (contour_omp.c)
# ---------------------------------------------------------------------------

def _omp_graphs():
    yield "path", 5000, *gg.path(5000, seed=11)
    yield "grid", 64 * 64, *gg.grid(64, 64, seed=12)
    yield "rmat12", 1 << 12, *gg.rmat(12, seed=13)
    n64, s64, d64 = gg.components64()
    yield "components64", n64, s64, d64
    yield "er", 3000, *gg.er(3000, 2000, seed=14)


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("order", [1, 2, 1024])
def test_omp_contour_matches_union_find(order, threads):
    for name, n, s, d in _omp_graphs():
        got, iters, used = oracle.omp_contour(n, s, d, order=order, threads=threads)
        assert np.array_equal(got, oracle.uf_labels(n, s, d)), (name, order, threads)
        assert used == threads and iters >= 1


def test_omp_contour_in_place_updates():
    """In-place (asynchronous) updates, Section III-B1: one thread over the
    sorted path 0-1, 1-2, ... in increasing order carries label 0 to the end
    within the first iteration (each edge reads the label its predecessor has
    just written), so the second iteration changes nothing.  The synchronous
    Alg. 1 needs about log_1.5(n) iterations on the same input."""
    n = 1000
    s = np.arange(n - 1, dtype=np.int32)
    d = s + 1
    for order in (1, 2, 1024):
        got, iters, _ = oracle.omp_contour(n, s, d, order=order, threads=1)
        assert iters == 2 and not got.any()
    _, sync_iters, _, _ = oracle.contour_sync(n, s, d, 2)
    assert sync_iters > 10
    # reversed order: order 1 moves label 0 one vertex per iteration
    got, iters, _ = oracle.omp_contour(n, s[::-1].copy(), d[::-1].copy(), order=1, threads=1)
    assert not got.any() and iters == n


def test_omp_contour_edge_cases():
    assert oracle.omp_contour(0, [], [], threads=2)[0].size == 0
    got, iters, _ = oracle.omp_contour(5, [], [], threads=2)
    assert got.tolist() == [0, 1, 2, 3, 4] and iters == 1
    got, _, _ = oracle.omp_contour(4, [3, 2, 2], [3, 2, 0], threads=2)
    assert got.tolist() == [0, 1, 0, 3]
    with pytest.raises(oracle.OracleIdError):
        oracle.omp_contour(3, [0], [3])
