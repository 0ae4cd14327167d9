"""The seeded input generators (no GPU): sizes, structure and determinism."""
import pytest
import numpy as np
import torch

import graphgen as gg
import oracle


def test_delaunay_like_counts_and_connectivity():
    for k in (4, 7, 10, 12):
        n, s, d = gg.delaunay_like(k)
        R, C = 1 << (k // 2), 1 << (k - k // 2)
        assert n == 1 << k == R * C
        assert s.numel() == R * (C - 1) + (R - 1) * C + (R - 1) * (C - 1)
        assert (oracle.uf_labels(n, s, d) == 0).all()
        deg = np.bincount(np.concatenate([s.numpy(), d.numpy()]), minlength=n)
        assert deg.max() <= 8


def _incircle(a, b, c, d):
    """> 0 iff d lies inside the circle through the counter-clockwise a, b, c."""
    rows = [(p[0] - d[0], p[1] - d[1]) for p in (a, b, c)]
    m = [[x, y, x * x + y * y] for x, y in rows]
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def test_delaunay_like_diagonals_pass_the_empty_circle_test():
    """Each cell's diagonal leaves the opposite corner outside the circumcircle
    of the triangle it forms (checked in exact Python integers)."""
    k, cell, jit = 8, 1024, 200
    n, s, d = gg.delaunay_like(k, permute=False)
    R, C = 1 << (k // 2), 1 << (k - k // 2)
    z = gg.uniform64(gg.stream_key(gg.BASE_SEED, 8), 0, n)
    jx = (gg.uniform_below(gg._hi32(z), 2 * jit + 1) - jit).tolist()
    jy = (gg.uniform_below(gg._lo32(z), 2 * jit + 1) - jit).tolist()
    P = [((i % C) * cell + jx[i], (i // C) * cell + jy[i]) for i in range(n)]
    edges = set(zip(s.tolist(), d.tolist()))
    for r in range(R - 1):
        for c in range(C - 1):
            a, b, cc, dd = r * C + c, r * C + c + 1, (r + 1) * C + c + 1, (r + 1) * C + c
            if (a, cc) in edges:  # triangles (a, b, cc) and (a, cc, dd)
                assert (b, dd) not in edges
                assert _incircle(P[a], P[b], P[cc], P[dd]) <= 0
            else:
                assert (b, dd) in edges
                assert _incircle(P[a], P[b], P[cc], P[dd]) > 0


def test_generators_are_deterministic_and_seeded():
    for make in (lambda sd: gg.rmat(10, seed=sd), lambda sd: gg.grid(20, 30, seed=sd),
                 lambda sd: gg.delaunay_like(9, seed=sd)[1:], lambda sd: gg.er(500, 900, seed=sd),
                 lambda sd: gg.caterpillar(30, seed=sd), lambda sd: gg.path(300, seed=sd)):
        a1, b1 = make(1)
        a2, b2 = make(1)
        a3, _ = make(2)
        assert torch.equal(a1, a2) and torch.equal(b1, b2)
        assert not torch.equal(a1, a3)


def test_family_sizes():
    assert gg.rmat(8)[0].numel() == 16 * 256
    assert gg.path(100)[0].numel() == 99
    assert gg.caterpillar(10)[0].numel() == 10 * 16 - 1
    s, _ = gg.grid(50, 60, p_drop=0)
    assert s.numel() == 50 * 59 + 49 * 60
    vo, eo, s, d, params = gg.batch_mix(12, n_hi=3e4)
    assert len(vo) == 13 and int(eo[-1]) == s.numel()
    for g, p in enumerate(params):
        n = int(vo[g + 1] - vo[g])
        a, b = int(eo[g]), int(eo[g + 1])
        assert n == p["n"]
        if b > a:
            assert int(s[a:b].max()) < n and int(d[a:b].max()) < n


@pytest.mark.parametrize("symmetric", [False, True])
def test_to_csr_matches_sorted_entries(symmetric):
    n, s, d = 300, *gg.er(300, 900, seed=21)
    s = torch.cat([s, torch.tensor([5, 7], dtype=torch.int32)])  # a loop and a repeat
    d = torch.cat([d, torch.tensor([5, int(d[0])], dtype=torch.int32)])
    off, cols = gg.to_csr(n, s, d, symmetric=symmetric)
    sn, dn = s.numpy().astype(np.int64), d.numpy().astype(np.int64)
    rows = np.concatenate([sn, dn]) if symmetric else sn
    want_cols = np.concatenate([dn, sn]) if symmetric else dn
    order = np.argsort(rows, kind="stable")
    assert off.dtype == torch.int64 and off[0] == 0 and off[-1] == rows.size
    assert np.array_equal(np.diff(off.numpy()), np.bincount(rows, minlength=n))
    assert np.array_equal(cols.numpy(), want_cols[order])
