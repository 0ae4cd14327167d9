"""Seeded synthetic graph generators.

These produce the inputs for both sides of every comparison: the CPU oracle
tests and the CUDA connected-components path.  The module holds no part of the
Contour method's arithmetic; it only builds edge lists.

Every random draw is a counter-based SplitMix64 value (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw ``i`` of
stream ``key`` is ``mix64(key + (i + 1) * GAMMA)``.  The generators are written
with PyTorch integer tensor operations only, so the same code runs on the CPU
and on a CUDA device and produces bit-identical graphs on both.

Graph families (the paper measures on real SNAP / SuiteSparse / GraphChallenge
graphs and on Delaunay meshes, Table I; none of those datasets is available
here, so these seeded families stand in for them):

* ``path``         -- a path, the long-diameter case of Lemma 2;
* ``grid``         -- an R x C 4-neighbour grid, each edge dropped with
                      probability 0.05 (long diameter, near-uniform degree);
* ``rmat``         -- R-MAT power-law graph with a/b/c/d = .57/.19/.19/.05;
* ``er``           -- G(n, m) with duplicate pairs and self-loops kept;
* ``caterpillar``  -- a path backbone with leaves hung on every backbone vertex;
* ``components64`` -- 32 paths + 32 Erdos-Renyi graphs with a spanning path,
                      each on 1,024 vertices (65,536 vertices, 294,880 edges);
* ``delaunay_like``-- planar triangulation of a jittered grid with Delaunay
                      diagonals (n = 2^k, m ~ 3n, degree ~6);
* ``batch_mix``    -- many independent graphs of log-uniform size drawn from
                      the four families above.

After construction every generator applies a seeded random permutation to the
vertex ids and a seeded shuffle to the edge order, so that neither ids nor edge
order carry the construction's structure.
"""
from __future__ import annotations

import math
from fractions import Fraction

import torch

__all__ = [
    "BASE_SEED", "mix64_int", "stream_key", "uniform64", "uniform_below",
    "path", "grid", "rmat", "er", "caterpillar", "components64", "delaunay_like",
    "batch_mix_params", "batch_graph", "batch_mix", "permute_and_shuffle", "to_csr"]

BASE_SEED = 2311028110
SHUFFLE_BLOCK = 1 << 30

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """Reinterpret an unsigned 64-bit Python int as a signed int64 value."""
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int (reference form)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *stream: int) -> int:
    """Derive the key of an independent stream from a seed and stream ids."""
    k = seed & _MASK64
    for s in stream:
        k = mix64_int(k + (s + 1) * _GAMMA)
    return k


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes viewed as uint64."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    return z ^ _lsr(z, 31)


def uniform64(key: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """Draws ``start .. start+count-1`` of stream ``key`` as int64 bit patterns."""
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _mix64(i * _s64(_GAMMA) + _s64(key))


def _hi32(z: torch.Tensor) -> torch.Tensor:
    return _lsr(z, 32)


def _lo32(z: torch.Tensor) -> torch.Tensor:
    return z & 0xFFFFFFFF


def uniform_below(u32: torch.Tensor, bound: int) -> torch.Tensor:
    """Map 32-bit uniforms to [0, bound) by multiply-shift (bound < 2**31)."""
    assert 0 < bound < (1 << 31)
    return (u32 * bound) >> 32


def _threshold(p: Fraction) -> int:
    return math.floor(p * (1 << 32))


def _chunks(total: int, size: int):
    s = 0
    while s < total:
        yield s, min(total, s + size)
        s += size


def _random_rank(key: int, count: int, device) -> torch.Tensor:
    """A seeded random permutation of range(count): rank of each draw."""
    if count == 0:
        return torch.empty(0, dtype=torch.int64, device=device)
    keys = uniform64(key, 0, count, device)
    order = torch.sort(keys, stable=True).indices
    del keys
    rank = torch.empty_like(order)
    rank[order] = torch.arange(count, dtype=torch.int64, device=device)
    return rank


def permute_and_shuffle(n: int, src: torch.Tensor, dst: torch.Tensor, seed: int,
                        id_dtype=torch.int32):
    """Relabel vertices by a seeded permutation and shuffle the edge order
    (src and dst are shuffled in place)."""
    device = src.device
    perm = _random_rank(stream_key(seed, 101), n, device)
    m = src.numel()
    # edges are shuffled by a stable sort on seeded 64-bit keys, within
    # consecutive blocks of 2^30 edges (the largest sort torch performs)
    key = stream_key(seed, 102)
    for lo, hi in _chunks(m, SHUFFLE_BLOCK):
        order = torch.sort(uniform64(key, lo, hi - lo, device), stable=True).indices + lo
        src[lo:hi] = src[order]
        dst[lo:hi] = dst[order]
        del order
    s = perm[src].to(id_dtype)
    d = perm[dst].to(id_dtype)
    return s, d


# ---------------------------------------------------------------------------
# families
# ---------------------------------------------------------------------------

def _finish(n, s, d, seed, permute, id_dtype):
    if permute:
        return permute_and_shuffle(n, s, d, seed, id_dtype)
    return s.to(id_dtype), d.to(id_dtype)


def path(n: int, seed: int = BASE_SEED, device="cpu", permute=True, id_dtype=torch.int32):
    """Path 0-1-...-(n-1): n vertices, n-1 edges, diameter n-1."""
    i = torch.arange(max(n - 1, 0), dtype=torch.int64, device=device)
    return _finish(n, i, i + 1, seed, permute, id_dtype)


def grid(rows: int, cols: int, p_drop: Fraction = Fraction(5, 100), seed: int = BASE_SEED,
         device="cpu", permute=True, id_dtype=torch.int32):
    """rows x cols 4-neighbour grid; each edge independently dropped with p_drop."""
    n = rows * cols
    nh = rows * (cols - 1)
    nv = (rows - 1) * cols
    e = torch.arange(nh + nv, dtype=torch.int64, device=device)
    keep = _hi32(uniform64(stream_key(seed, 1), 0, nh + nv, device)) >= _threshold(p_drop)
    e = e[keep]
    is_h = e < nh
    eh = e[is_h]
    ev = e[~is_h] - nh
    rh, ch = eh // (cols - 1), eh % (cols - 1)
    u_h = rh * cols + ch
    u_v = ev  # (r, c) -> r*cols + c, neighbour below at + cols
    s = torch.cat([u_h, u_v])
    d = torch.cat([u_h + 1, u_v + cols])
    # restore the original edge-index order so the pre-shuffle list is canonical
    order = torch.sort(torch.cat([eh, ev + nh]), stable=True).indices
    return _finish(n, s[order], d[order], seed, permute, id_dtype)


RMAT_ABCD = (Fraction(57, 100), Fraction(19, 100), Fraction(19, 100), Fraction(5, 100))


def rmat(scale: int, edge_factor: int = 16, seed: int = BASE_SEED, device="cpu",
         permute=True, id_dtype=torch.int32, n: int | None = None, m: int | None = None,
         abcd=RMAT_ABCD, chunk: int = 1 << 26):
    """R-MAT graph: m = edge_factor * 2**scale (u, v) samples, loops and repeats kept.

    Each level picks a quadrant with probabilities a, b, c, d by comparing the
    high (even levels) or low (odd levels) 32 bits of one 64-bit draw with
    integer thresholds.  With ``n`` given (n <= 2**scale), ids >= n are folded
    into range by subtracting n (used for the batch mix).
    """
    a, b, c, _ = abcd
    t1, t2, t3 = _threshold(a), _threshold(a + b), _threshold(a + b + c)
    N = 1 << scale
    if n is None:
        n = N
    assert n <= N
    if m is None:
        m = edge_factor * N
    key = stream_key(seed, 2)
    per_edge = (scale + 1) // 2
    src = torch.empty(m, dtype=torch.int64, device=device)
    dst = torch.empty(m, dtype=torch.int64, device=device)
    for lo, hi in _chunks(m, chunk):
        cnt = hi - lo
        s = torch.zeros(cnt, dtype=torch.int64, device=device)
        d = torch.zeros(cnt, dtype=torch.int64, device=device)
        base = torch.arange(lo, hi, dtype=torch.int64, device=device) * per_edge
        for j in range(per_edge):
            z = _mix64((base + (j + 1)) * _s64(_GAMMA) + _s64(key))
            for half, r in ((0, _hi32(z)), (1, _lo32(z))):
                level = 2 * j + half
                if level >= scale:
                    break
                bit = 1 << (scale - 1 - level)
                sb = r >= t2
                db = ((r >= t1) & (r < t2)) | (r >= t3)
                s += sb.to(torch.int64) * bit
                d += db.to(torch.int64) * bit
            del z
        if n < N:
            s = torch.where(s >= n, s - n, s)
            d = torch.where(d >= n, d - n, d)
        src[lo:hi] = s
        dst[lo:hi] = d
        del s, d, base
    return _finish(n, src, dst, seed, permute, id_dtype)


def er(n: int, m: int, seed: int = BASE_SEED, device="cpu", permute=True, id_dtype=torch.int32):
    """G(n, m) multigraph: m independent uniform (u, v) pairs."""
    z = uniform64(stream_key(seed, 3), 0, m, device)
    s = uniform_below(_hi32(z), n)
    d = uniform_below(_lo32(z), n)
    return _finish(n, s, d, seed, permute, id_dtype)


def caterpillar(backbone: int, leaves: int = 15, seed: int = BASE_SEED, device="cpu",
                permute=True, id_dtype=torch.int32):
    """Path backbone 0..B-1; vertex B + leaves*i + j is leaf j of backbone i.

    n = B * (leaves + 1), m = B - 1 + leaves * B; one component; diameter B + 1.
    """
    B = backbone
    n = B * (leaves + 1)
    i = torch.arange(B - 1, dtype=torch.int64, device=device)
    leaf = torch.arange(B * leaves, dtype=torch.int64, device=device)
    s = torch.cat([i, leaf // leaves])
    d = torch.cat([i + 1, B + leaf])
    return _finish(n, s, d, seed, permute, id_dtype)


def _distinct_pairs(k: int, count: int, key: int, device):
    """The first ``count`` distinct unordered non-loop pairs of [0,k) in draw order."""
    want = count
    cand = 2 * count + 64
    while True:
        z = uniform64(key, 0, cand, device)
        x = uniform_below(_hi32(z), k)
        y = uniform_below(_lo32(z), k)
        lo, hi = torch.minimum(x, y), torch.maximum(x, y)
        valid = lo != hi
        pk = torch.where(valid, lo * k + hi, torch.full_like(lo, -1))
        order = torch.sort(pk, stable=True).indices
        sk = pk[order]
        first = torch.ones_like(sk, dtype=torch.bool)
        first[1:] = sk[1:] != sk[:-1]
        first &= sk >= 0
        idx = torch.sort(order[first]).values
        if idx.numel() >= want:
            idx = idx[:want]
            return lo[idx], hi[idx]
        cand *= 2


def components64(seed: int = BASE_SEED, device="cpu", permute=True, id_dtype=torch.int32,
                 comp: int = 1024, n_path: int = 32, n_er: int = 32, er_extra: int = 7169):
    """32 paths + 32 ER-with-spanning-path components of 1,024 vertices each.

    Component k owns ids [1024k, 1024k+1024) before the global permutation.
    Each ER component is a spanning path 0-1-..-1023 plus ``er_extra`` distinct
    uniform non-loop pairs (mean degree 8: 1023 + 7169 = 8192 edges).
    Totals: n = 65,536, m = 32*1023 + 32*8192 = 294,880.
    """
    parts_s, parts_d = [], []
    i = torch.arange(comp - 1, dtype=torch.int64, device=device)
    for k in range(n_path + n_er):
        base = k * comp
        parts_s.append(base + i)
        parts_d.append(base + i + 1)
        if k >= n_path:
            x, y = _distinct_pairs(comp, er_extra, stream_key(seed, 4, k), device)
            parts_s.append(base + x)
            parts_d.append(base + y)
    n = comp * (n_path + n_er)
    return n, *_finish(n, torch.cat(parts_s), torch.cat(parts_d), seed, permute, id_dtype)


def delaunay_like(k: int, seed: int = BASE_SEED, device="cpu", permute=True, id_dtype=torch.int32,
                  cell: int = 1024, jitter: int = 200):
    """Delaunay-style planar triangulation with n = 2**k vertices, m ~ 3n.

    Stand-in for the delaunay_n* family (Delaunay triangulations of random
    points, near-uniform degree ~6).  Vertex (r, c) of an R x C grid
    (R = 2**(k//2), C = 2**(k - k//2)) sits at integer point
    (c*cell + jx, r*cell + jy) with jx, jy uniform in [-jitter, jitter].  Grid
    edges are kept and every cell is split by the diagonal that satisfies the
    empty-circumcircle (Delaunay) test for its four corners, evaluated exactly
    in 64-bit integers, so the graph is identical on CPU and GPU.
    """
    R, C = 1 << (k // 2), 1 << (k - k // 2)
    n = R * C
    z = uniform64(stream_key(seed, 8), 0, n, device)
    span = 2 * jitter + 1
    jx = uniform_below(_hi32(z), span) - jitter
    jy = uniform_below(_lo32(z), span) - jitter
    idx = torch.arange(n, dtype=torch.int64, device=device)
    r, c = idx // C, idx % C
    px, py = c * cell + jx, r * cell + jy
    # cells (r, c) for r < R-1, c < C-1; corners a=(r,c) b=(r,c+1) cc=(r+1,c+1) d=(r+1,c)
    cr = torch.arange(R - 1, dtype=torch.int64, device=device).repeat_interleave(C - 1)
    ccol = torch.arange(C - 1, dtype=torch.int64, device=device).repeat(R - 1)
    a = cr * C + ccol
    b = a + 1
    cc_ = a + C + 1
    d = a + C
    # d inside the circumcircle of the counter-clockwise triangle (a, b, cc)?
    ax, ay = px[a] - px[d], py[a] - py[d]
    bx, by = px[b] - px[d], py[b] - py[d]
    cx, cy = px[cc_] - px[d], py[cc_] - py[d]
    a2, b2, c2 = ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy
    det = ax * (by * c2 - b2 * cy) - ay * (bx * c2 - b2 * cx) + a2 * (bx * cy - by * cx)
    flip = det > 0  # then the Delaunay diagonal is b-d, else a-cc
    ds = torch.where(flip, b, a)
    dd = torch.where(flip, d, cc_)
    hs = (idx[c < C - 1])
    vs = idx[r < R - 1]
    s = torch.cat([hs, vs, ds])
    t = torch.cat([hs + 1, vs + C, dd])
    return n, *_finish(n, s, t, seed, permute, id_dtype)


# ---------------------------------------------------------------------------
# batch mix
# ---------------------------------------------------------------------------

BATCH_KINDS = ("er", "path", "grid", "rmat")


def batch_mix_params(n_graphs: int, seed: int = BASE_SEED, n_lo: float = 1e3, n_hi: float = 1e6):
    """Host-side, deterministic per-graph parameters of the batch mix.

    Graph i has kind ``BATCH_KINDS[i % 4]`` (equal mix), n log-uniform in
    [n_lo, n_hi], and for ER a mean degree d uniform in [4, 32] (m = n*d/2).
    Grids use rows = floor(sqrt(n)), cols = n // rows (n rounded down to
    rows*cols); R-MAT uses scale ceil(log2 n), edge factor 16, ids folded to n.
    """
    out = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for g in range(n_graphs):
        u1 = mix64_int(stream_key(seed, 5, g)) >> 11
        u2 = mix64_int(stream_key(seed, 6, g)) >> 11
        f1 = u1 / float(1 << 53)
        f2 = u2 / float(1 << 53)
        n = int(math.floor(math.exp(lo + (hi - lo) * f1)))
        n = max(2, min(n, int(n_hi)))
        kind = BATCH_KINDS[g % 4]
        p = {"kind": kind, "seed": stream_key(seed, 7, g)}
        if kind == "er":
            d = 4.0 + 28.0 * f2
            p.update(n=n, m=int(n * d / 2))
        elif kind == "path":
            p.update(n=n, m=n - 1)
        elif kind == "grid":
            r = max(1, int(math.isqrt(n)))
            c = max(2, n // r)
            p.update(n=r * c, rows=r, cols=c)
        else:
            scale = max(1, (n - 1).bit_length())
            p.update(n=n, scale=scale, m=16 * n)
        out.append(p)
    return out


def batch_graph(p: dict, device="cpu", id_dtype=torch.int32):
    """Generate one graph of the batch mix from its parameter dict (local ids)."""
    k = p["kind"]
    if k == "er":
        s, d = er(p["n"], p["m"], seed=p["seed"], device=device, id_dtype=id_dtype)
    elif k == "path":
        s, d = path(p["n"], seed=p["seed"], device=device, id_dtype=id_dtype)
    elif k == "grid":
        s, d = grid(p["rows"], p["cols"], seed=p["seed"], device=device, id_dtype=id_dtype)
    else:
        s, d = rmat(p["scale"], seed=p["seed"], device=device, n=p["n"], m=p["m"],
                    id_dtype=id_dtype)
    return p["n"], s, d


def batch_mix(n_graphs: int, seed: int = BASE_SEED, device="cpu", n_lo=1e3, n_hi=1e6,
              id_dtype=torch.int32):
    """Concatenated batch: returns (vtx_off, edge_off, src, dst, params).

    ``vtx_off``/``edge_off`` are int64 offsets of length n_graphs+1; src/dst
    hold local ids of each graph, concatenated in graph order.
    """
    params = batch_mix_params(n_graphs, seed, n_lo, n_hi)
    vtx = [0]
    eo = [0]
    for p in params:
        vtx.append(vtx[-1] + p["n"])
        eo.append(eo[-1] + _edge_count(p))
    src = torch.empty(eo[-1], dtype=id_dtype, device=device)
    dst = torch.empty(eo[-1], dtype=id_dtype, device=device)
    for g, p in enumerate(params):
        _, s, d = batch_graph(p, device, id_dtype)
        assert s.numel() == eo[g + 1] - eo[g]
        src[eo[g]:eo[g + 1]] = s
        dst[eo[g]:eo[g + 1]] = d
    return (torch.tensor(vtx, dtype=torch.int64), torch.tensor(eo, dtype=torch.int64),
            src, dst, params)


def _edge_count(p: dict) -> int:
    if p["kind"] == "grid":
        # deletions are random: count them from the keep mask (cheap on CPU)
        rows, cols = p["rows"], p["cols"]
        tot = rows * (cols - 1) + (rows - 1) * cols
        keep = _hi32(uniform64(stream_key(p["seed"], 1), 0, tot, "cpu")) >= _threshold(Fraction(5, 100))
        return int(keep.sum())
    return p["m"]


def to_csr(n: int, src: torch.Tensor, dst: torch.Tensor, symmetric: bool = False):
    """CSR form of an edge list: ``(offsets int64[n + 1], cols)``.

    Entry order: rows ascending; within a row the entries keep the order of
    the edge list (stable sort).  ``symmetric=False``: edge e is the entry
    (src[e], dst[e]).  ``symmetric=True``: edge e is stored in both rows,
    (src[e], dst[e]) and (dst[e], src[e]) (a self-loop twice in its row), so
    nnz = 2 * m.  Runs on the tensors' device; no arithmetic of the method.
    """
    if symmetric:
        rows = torch.cat([src, dst])
        cols = torch.cat([dst, src])
    else:
        rows, cols = src, dst
    order = torch.sort(rows.to(torch.int64), stable=True).indices
    cols = cols[order].contiguous()
    counts = torch.bincount(rows.to(torch.int64), minlength=n)
    off = torch.zeros(n + 1, dtype=torch.int64, device=src.device)
    if n:
        off[1:] = torch.cumsum(counts, 0)
    return off, cols
