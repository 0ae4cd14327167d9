"""CPU oracle for the learned scheduler -- TEST INFRASTRUCTURE ONLY.

Plain numpy statements (fp64) of what the scheduler computes:

* ``features``      -- the 12 graph features: n, m, degree variance and maximum
                       on an edge sample (scaled), eccentricities of 8 sampled
                       sources by breadth-first search on the sample graph,
                       each as log2(1 + x).  The sample, the sources and the
                       level cap follow the definition in include/contour.h.
* ``bf16_to_f32``   -- decoding of bfloat16 bit patterns (the top 16 bits of an
                       IEEE-754 binary32).
* ``mlp_forward``   -- 12 -> 64 -> 64 -> 64 -> 18 ReLU network on standardised
                       inputs.
* ``adam_step``     -- one Adam step (Kingma & Ba 2015) from zero moments on the
                       mean softmax cross-entropy, gradients by backpropagation
                       written out layer by layer.

The scheduler is not part of the paper (the paper chooses operators by hand,
Section IV-E); these functions are pinned in tests/test_oracle_sched.py by
closed forms, finite differences and scipy's breadth-first distances.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 12
HIDDEN = 64
N_OUT = 18
SAMPLE = 16384
LEVELS = 16
LAYER_IN = (N_FEAT, HIDDEN, HIDDEN, HIDDEN)
LAYER_OUT = (HIDDEN, HIDDEN, HIDDEN, N_OUT)


def sample_positions(m: int, S: int = SAMPLE) -> np.ndarray:
    """Edge positions of the sample: all edges when m <= S, else floor(j*m/S)."""
    if m <= S:
        return np.arange(m, dtype=np.int64)
    j = np.arange(S, dtype=np.int64)
    return (j * m) // S


def bfs_eccentricity(n: int, s: np.ndarray, d: np.ndarray, source: int, cap: int = LEVELS) -> int:
    """Largest BFS distance (at most ``cap``) reached from ``source``."""
    adj = [[] for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    dist = {source: 0}
    frontier = [source]
    level = 0
    while frontier and level < cap:
        level += 1
        nxt = []
        for x in frontier:
            for y in adj[x]:
                if y not in dist:
                    dist[y] = level
                    nxt.append(y)
        frontier = nxt
    return max(dist.values())


def features(n: int, src, dst) -> np.ndarray:
    """The 12 scheduler features of one graph (float32, log2(1 + x))."""
    s_all = np.asarray(src, dtype=np.int64)
    d_all = np.asarray(dst, dtype=np.int64)
    m = s_all.size
    pos = sample_positions(m)
    S = pos.size
    s, d = s_all[pos], d_all[pos]
    deg = np.bincount(np.concatenate([s, d]), minlength=max(n, 1)).astype(np.float64)
    nn = float(n) if n > 0 else 1.0
    mean = 2.0 * S / nn
    var_s = float((deg ** 2).sum()) / nn - mean * mean
    scale = m / S if S > 0 else 0.0
    var_est = max(var_s, 0.0) * scale * scale
    max_est = float(deg.max()) * scale if S > 0 else 0.0
    ecc = []
    for i in range(8):
        if S == 0:
            ecc.append(0)
            continue
        j = ((2 * i + 1) * S) // 16
        ecc.append(bfs_eccentricity(n, s, d, int(s[j])))
    raw = [n, m, var_est, max_est] + ecc
    return np.log2(1.0 + np.array(raw, dtype=np.float64)).astype(np.float32)


def bf16_to_f32(bits) -> np.ndarray:
    """bfloat16 bit patterns (uint16) -> float32 values."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32)


def parse_blob(blob: bytes):
    """(mean, std, [(W, b)] * 4) of a CCMLP01 weight blob, weights decoded."""
    buf = memoryview(blob)
    assert bytes(buf[:7]) == b"CCMLP01"
    hdr = np.frombuffer(buf[8:24], dtype=np.int32)
    assert tuple(hdr) == (N_FEAT, HIDDEN, 3, N_OUT)
    mean = np.frombuffer(buf[24:24 + 48], dtype=np.float32).astype(np.float64)
    std = np.frombuffer(buf[72:72 + 48], dtype=np.float32).astype(np.float64)
    off = 120
    layers = []
    for ni, no in zip(LAYER_IN, LAYER_OUT):
        w = bf16_to_f32(np.frombuffer(buf[off:off + 2 * ni * no], dtype=np.uint16)).astype(np.float64)
        off += 2 * ni * no
        b = np.frombuffer(buf[off:off + 4 * no], dtype=np.float32).astype(np.float64)
        off += 4 * no
        layers.append((w.reshape(no, ni), b))
    assert off == len(blob)
    return mean, std, layers


def mlp_forward(x_std: np.ndarray, layers) -> np.ndarray:
    """Logits of standardised inputs x_std (rows) through ReLU layers."""
    h = np.asarray(x_std, dtype=np.float64)
    for i, (w, b) in enumerate(layers):
        h = h @ w.T + b
        if i < len(layers) - 1:
            h = np.maximum(h, 0.0)
    return h


def unpack_params(p: np.ndarray):
    """Flat [W1 b1 W2 b2 W3 b3 W4 b4] -> [(W, b)] * 4."""
    layers, off = [], 0
    for ni, no in zip(LAYER_IN, LAYER_OUT):
        w = p[off:off + ni * no].reshape(no, ni)
        off += ni * no
        b = p[off:off + no]
        off += no
        layers.append((w, b))
    return layers


def pack_params(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in layers])


def loss_and_grad(p: np.ndarray, x: np.ndarray, y: np.ndarray):
    """Mean softmax cross-entropy and its gradient w.r.t. the flat parameters."""
    layers = unpack_params(np.asarray(p, dtype=np.float64))
    B = x.shape[0]
    acts, pre = [np.asarray(x, dtype=np.float64)], []
    h = acts[0]
    for i, (w, b) in enumerate(layers):
        z = h @ w.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if i < 3 else z
        acts.append(h)
    z = pre[-1]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    prob = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(np.log(e.sum(axis=1)) + zmax[:, 0] - z[np.arange(B), y]))
    dz = prob.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    grads = [None] * 4
    for i in range(3, -1, -1):
        w, _ = layers[i]
        grads[i] = (dz.T @ acts[i], dz.sum(axis=0))
        if i > 0:
            dz = (dz @ w) * (pre[i - 1] > 0)
    return loss, pack_params(grads)


def adam_step(p: np.ndarray, g: np.ndarray, lr: float, b1=0.9, b2=0.999, eps=1e-8) -> np.ndarray:
    """First Adam step (t = 1) from zero moments."""
    m1 = (1 - b1) * g
    m2 = (1 - b2) * g * g
    mh = m1 / (1 - b1)
    vh = m2 / (1 - b2)
    return p - lr * mh / (np.sqrt(vh) + eps)
