"""CPU oracle for Contour connected components -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and nothing
here uses the product path.

Contents (each function cites the passage of the paper it follows):

* ``uf_labels``      -- serial union-find (``uf.c``); label[v] = smallest id in
                        v's component, the unique fixed point of Alg. 1
                        (Section II-A: the final pointer graph is S stars).
* ``bfs_labels``     -- an independent second labeller: breadth-first search
                        from each not-yet-visited vertex in increasing id order
                        (numpy; the BFS of Section I, used here as a checker).
* ``contour_sync``   -- a serial simulator of Alg. 1 with the order-h operator
                        of Def. 3 (``contour_sim.c``), returning every
                        per-iteration state of L.
* ``degree_features``-- plain-definition graph statistics for the scheduler.
* ``omp_contour``    -- multicore asynchronous Contour (C-1, C-2, C-m) with
                        OpenMP (``contour_omp.c``, Section III-B): not a
                        checker but the timed multicore CPU baseline; pinned
                        against ``uf_labels`` like the GPU path.

All three labellers are pinned in ``tests/test_oracle.py`` against brute-force
reachability, closed forms and the iteration bounds of Lemma 2 / the Theorem.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["uf.c", "contour_sim.c"]
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_OMP_SOURCES = ["contour_omp.c"]
_lib = None
_omp_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` with the host gcc."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, *srcs])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_omp(force: bool = False) -> str:
    """Compile the multicore baseline into ``oracle/liboracle_omp.so``
    (gcc -fopenmp).  Raises ``subprocess.CalledProcessError`` when the host
    compiler has no OpenMP."""
    srcs = [os.path.join(_HERE, s) for s in _OMP_SOURCES]
    if not force and os.path.exists(_OMP_LIB_PATH):
        if os.path.getmtime(_OMP_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs):
            return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, *srcs])
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_uf_labels_i32.argtypes = [i64, i64, p, p, p]
        lib.oracle_uf_labels_i32.restype = i64
        lib.oracle_uf_labels_i64.argtypes = [i64, i64, p, p, p]
        lib.oracle_uf_labels_i64.restype = i64
        lib.oracle_contour_sync_i32.argtypes = [i64, i64, p, p, ctypes.c_int32, i64, p, p, p]
        lib.oracle_contour_sync_i32.restype = i64
        _lib = lib
    return _lib


def _as_np(x, dtype):
    if hasattr(x, "detach"):  # torch tensor (CPU)
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


class OracleIdError(ValueError):
    """An edge endpoint lies outside [0, n)."""

    def __init__(self, edge):
        super().__init__(f"edge {edge} has an endpoint outside [0, n)")
        self.edge = edge


def uf_labels(n: int, src, dst, id_bits: int = 32) -> np.ndarray:
    """label[v] = min id of v's component, by serial union-find (``uf.c``)."""
    lib = _load()
    dt = np.int32 if id_bits == 32 else np.int64
    s, d = _as_np(src, dt), _as_np(dst, dt)
    assert s.shape == d.shape
    out = np.empty(n, dtype=dt)
    fn = lib.oracle_uf_labels_i32 if id_bits == 32 else lib.oracle_uf_labels_i64
    rc = fn(n, s.size, s.ctypes.data, d.ctypes.data, out.ctypes.data)
    if rc < 0:
        raise OracleIdError(-rc - 1)
    return out


def bfs_labels(n: int, src, dst) -> np.ndarray:
    """label[v] = min id of v's component, by BFS from vertices in id order.

    Scanning start vertices in increasing id order, the first vertex of every
    component reached is that component's smallest id; one BFS from it labels
    the whole component.  Frontier expansion uses a CSR adjacency built with
    numpy; the BFS itself is the plain level-by-level traversal.
    """
    s, d = _as_np(src, np.int64), _as_np(dst, np.int64)
    if s.size and (s.min() < 0 or d.min() < 0 or s.max() >= n or d.max() >= n):
        raise OracleIdError(-1)
    u = np.concatenate([s, d])
    w = np.concatenate([d, s])
    order = np.argsort(u, kind="stable")
    nbr = w[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, u + 1, 1)
    off = np.cumsum(off)
    label = np.full(n, -1, dtype=np.int64)
    for start in range(n):
        if label[start] >= 0:
            continue
        label[start] = start
        frontier = np.array([start], dtype=np.int64)
        while frontier.size:
            lo, hi = off[frontier], off[frontier + 1]
            cnt = hi - lo
            if cnt.sum() == 0:
                break
            idx = np.repeat(lo - np.cumsum(np.concatenate([[0], cnt[:-1]])), cnt) + np.arange(cnt.sum())
            nxt = np.unique(nbr[idx])
            nxt = nxt[label[nxt] < 0]
            label[nxt] = start
            frontier = nxt
    return label


def contour_sync(n: int, src, dst, order: int = 2, max_iters: int = 10_000,
                 init=None, record: bool = False):
    """Simulate Alg. 1 with MM^h (Def. 3), h = ``order``.

    Returns ``(labels, iterations, converged, states)``; ``states`` is a
    (iterations, n) int32 array of L after each iteration when ``record``.
    """
    lib = _load()
    s, d = _as_np(src, np.int32), _as_np(dst, np.int32)
    L = np.empty(n, dtype=np.int32)
    ini = None if init is None else _as_np(init, np.int32)
    states = np.empty((max_iters, n), dtype=np.int32) if record else None
    rc = lib.oracle_contour_sync_i32(
        n, s.size, s.ctypes.data, d.ctypes.data, int(order), int(max_iters),
        None if ini is None else ini.ctypes.data, L.ctypes.data,
        None if states is None else states.ctypes.data)
    if rc == -(1 << 62):
        raise MemoryError("oracle_contour_sync: allocation failed")
    iters = abs(rc)
    converged = rc > 0
    if record:
        states = states[:iters].copy()
    return L, iters, converged, states


def omp_contour(n: int, src, dst, order: int = 2, threads: int = 0, max_iters: int = 1 << 20):
    """Asynchronous order-h Contour on the host's cores (``contour_omp.c``).

    Returns ``(labels, iterations, threads_used)``; raises RuntimeError when
    ``max_iters`` iterations do not reach the fixed point.
    """
    global _omp_lib
    if _omp_lib is None:
        build_omp()
        lib = ctypes.CDLL(_OMP_LIB_PATH)
        i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.omp_contour_async_i32.argtypes = [i64, i64, p, p, i32, i64, i32, p, p]
        lib.omp_contour_async_i32.restype = i64
        _omp_lib = lib
    s, d = _as_np(src, np.int32), _as_np(dst, np.int32)
    assert s.shape == d.shape
    if s.size and (min(s.min(), d.min()) < 0 or max(s.max(), d.max()) >= n):
        raise OracleIdError(-1)
    L = np.empty(n, dtype=np.int32)
    used = ctypes.c_int32(0)
    it = _omp_lib.omp_contour_async_i32(n, s.size, s.ctypes.data, d.ctypes.data, int(order), int(max_iters),
                                        int(threads), L.ctypes.data, ctypes.byref(used))
    if it < 0:
        raise RuntimeError(f"omp_contour: no fixed point after {max_iters} iterations")
    return L, int(it), int(used.value)


def degree_features(n: int, src, dst) -> dict:
    """Plain-definition degree statistics of an undirected multigraph.

    deg[v] counts every edge end at v (a self-loop adds 2).  Returns n, m and
    the mean, population variance and maximum of deg.
    """
    s, d = _as_np(src, np.int64), _as_np(dst, np.int64)
    deg = np.bincount(np.concatenate([s, d]), minlength=n).astype(np.float64)
    return {"n": n, "m": int(s.size), "deg_mean": float(deg.mean()) if n else 0.0,
            "deg_var": float(deg.var()) if n else 0.0,
            "deg_max": float(deg.max()) if n else 0.0}
