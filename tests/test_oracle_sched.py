"""Pins for the scheduler oracle (oracle/sched.py), no GPU.

Features are pinned by closed forms on paths and stars, by the scaling of a
repeated edge, and by scipy's breadth-first distances; the network by a
hand-built model whose logits are known; the gradient by central finite
differences; the first Adam step by its closed form; bfloat16 decoding by
known bit patterns.
"""
import math
import struct

import numpy as np
import pytest

from oracle import sched as so


def test_sample_positions():
    assert so.sample_positions(10).tolist() == list(range(10))
    p = so.sample_positions(2 * so.SAMPLE)
    assert p.size == so.SAMPLE and (p == 2 * np.arange(so.SAMPLE)).all()
    p = so.sample_positions(3 * so.SAMPLE + 1)
    assert p[0] == 0 and p[-1] == ((so.SAMPLE - 1) * (3 * so.SAMPLE + 1)) // so.SAMPLE


@pytest.mark.parametrize("n", [2, 3, 10, 40, 1000])
def test_path_features_closed_form(n):
    s = np.arange(n - 1)
    d = s + 1
    f = so.features(n, s, d)
    m = n - 1
    mean = 2 * m / n
    var = ((2 * 1 + (n - 2) * 4) / n - mean * mean) if n > 2 else 1.0 - mean * mean
    mx = 2 if n > 2 else 1
    want = [n, m, max(var, 0.0), mx]
    for i in range(8):
        src = ((2 * i + 1) * m) // 16
        want.append(min(max(src, n - 1 - src), so.LEVELS))
    assert np.allclose(f, np.log2(1 + np.array(want, dtype=np.float64)), rtol=0, atol=1e-6)


def test_star_features_closed_form():
    k = 50
    s = np.zeros(k, dtype=np.int64)
    d = np.arange(1, k + 1)
    f = so.features(k + 1, s, d)
    n = k + 1
    mean = 2 * k / n
    var = (k * k + k) / n - mean * mean
    want = [n, k, var, k] + [1] * 8  # every source is the centre (src endpoint 0)
    assert np.allclose(f, np.log2(1 + np.array(want)), atol=1e-6)
    # reversed orientation: sources are leaves, eccentricity 2
    f2 = so.features(k + 1, d, s)
    assert np.allclose(f2[4:], np.log2(3.0), atol=1e-6)


def test_sampled_degree_scaling():
    S = so.SAMPLE
    s = np.zeros(2 * S, dtype=np.int64)
    d = np.ones(2 * S, dtype=np.int64)
    f = so.features(2, s, d)
    # sample: S copies of <0,1>; degrees S each (variance 0); scaled maximum 2S
    assert np.allclose(f[:4], np.log2(1 + np.array([2, 2 * S, 0.0, 2 * S])), atol=1e-6)


def test_bfs_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(5, 60))
        m = int(rng.integers(0, 80))
        s = rng.integers(0, n, m)
        d = rng.integers(0, n, m)
        A = sp.coo_matrix((np.ones(m), (s, d)), shape=(n, n)).tocsr()
        dist = csg.shortest_path(A, directed=False, unweighted=True)
        for src in range(0, n, 7):
            row = dist[src]
            want = int(min(row[np.isfinite(row)].max(), so.LEVELS))
            assert so.bfs_eccentricity(n, s, d, src) == want


def test_bf16_decode():
    bits = [0x3F80, 0xC000, 0x0000, 0x7F80, 0x3E80]
    assert so.bf16_to_f32(bits).tolist() == [1.0, -2.0, 0.0, math.inf, 0.25]


def _blob(layers, mean, std):
    out = b"CCMLP01\x00" + struct.pack("<4i", 12, 64, 3, 18)
    out += np.asarray(mean, np.float32).tobytes() + np.asarray(std, np.float32).tobytes()
    for w, b in layers:
        wb = (np.asarray(w, np.float32).view(np.uint32) >> 16).astype(np.uint16)
        out += wb.tobytes() + np.asarray(b, np.float32).tobytes()
    return out


def test_hand_built_network_logits():
    """W1, W2, W3 pass feature 0 through unit 0; W4 row k = k: logits = 2k + b4[k]."""
    layers = []
    for ni, no in zip(so.LAYER_IN, so.LAYER_OUT):
        w = np.zeros((no, ni))
        b = np.zeros(no)
        if no != so.N_OUT:
            w[0, 0] = 1.0
        else:
            w[:, 0] = np.arange(no)
            b = np.full(no, 0.5)
        layers.append((w, b))
    mean, std = np.zeros(12), np.ones(12)
    m2, s2, parsed = so.parse_blob(_blob(layers, mean, std))
    x = np.zeros((1, 12))
    x[0, 0] = 2.0
    assert np.allclose(so.mlp_forward((x - m2) / s2, parsed)[0], 2 * np.arange(18) + 0.5)
    x[0, 0] = -3.0  # the ReLU cuts it off
    assert np.allclose(so.mlp_forward(x, parsed)[0], np.full(18, 0.5))


def test_uniform_logits_loss_is_log_classes():
    p = np.zeros(sum(i * o + o for i, o in zip(so.LAYER_IN, so.LAYER_OUT)))
    x = np.random.default_rng(0).normal(size=(7, 12))
    y = np.arange(7) % 18
    loss, g = so.loss_and_grad(p, x, y)
    assert abs(loss - math.log(18)) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = sum(i * o + o for i, o in zip(so.LAYER_IN, so.LAYER_OUT))
    p = rng.normal(scale=0.3, size=P)
    x = rng.normal(size=(5, 12))
    y = rng.integers(0, 18, 5)
    _, g = so.loss_and_grad(p, x, y)
    idx = rng.choice(P, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(P)
        e[i] = h
        num = (so.loss_and_grad(p + e, x, y)[0] - so.loss_and_grad(p - e, x, y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-4 * abs(num), (i, num, g[i])


def test_first_adam_step_closed_form():
    p = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -1e-3, 0.0, 2.0])
    lr = 0.01
    want = p - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(so.adam_step(p, g, lr), want, rtol=0, atol=1e-12)
