"""Python binding of libcontour.so (C ABI in include/contour.h).

The functions below carry the C entry points' names and only marshal
arguments: every step of the computation runs in the CUDA library.  Arrays may
be torch tensors (CPU or CUDA) or numpy arrays; device tensors are passed by
pointer, and the stream defaults to torch's current CUDA stream.

The library must have been built (``paper_2311_02811_gb300.build.build()`` or
``__graft_entry__.build()``); importing this module raises ImportError when
libcontour.so is missing, and there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "CC_OK", "CC_EINVAL", "CC_EIDRANGE", "CC_ENOMEM", "CC_ECUDA", "CC_ENOTCONVERGED",
    "CC_ETIMEOUT", "CC_ID32", "CC_ID64", "CC_COO", "CC_CSR", "CC_CSR_NATIVE", "CC_CSR_NATIVE_SYM",
    "CC_SYNC", "CC_ASYNC", "CC_ASYNC_COMPACT",
    "CC_ORDER_FULL", "CC_ORDER_AUTO", "CC_ORDER_11MM", "CC_ORDER_1M1M", "CC_NOALLOC_MAX_N", "CCError", "cc_stats", "cc_graph", "lib", "LIB_PATH",
    "cc_init", "cc_run", "cc_solve_host", "cc_run_noalloc", "cc_free", "cc_release_memory", "cc_batch_plan", "cc_batch_init",
    "cc_batch_run", "cc_batch_set_schedule", "cc_batch_run_scheduled", "cc_batch_tuning",
    "cc_batch_set_tuning", "cc_batch_reorder", "cc_batch_edges", "cc_batch_free", "cc_batch", "cc_sched_load", "cc_sched_blob_bytes",
    "cc_sched_param_count", "cc_sched_decode", "cc_graph_features", "cc_batch_features",
    "cc_sched_predict", "cc_sched_predict_batch", "cc_sched_load_batch", "unload_scheduler", "cc_sched_train", "load_default_scheduler", "SCHED_WEIGHTS_PATH", "SCHED_BATCH_WEIGHTS_PATH", "cc_sched_train_step", "CC_SCHED_FEATURES", "CC_SCHED_CLASSES", "cc_graph_info", "cc_graph_edges", "cc_graph_set_stream", "cc_graph_reorder", "CC_REORDER_SRC", "CC_REORDER_LOWDEG", "CC_REORDER_HUB", "CC_REORDER_DEGREE", "cc_graph_hubs", "cc_graph_perm", "cc_graph_set_launch", "CC_LAUNCH_GRAPH", "CC_LAUNCH_HOST", "cc_strerror",
    "cc_last_error",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcontour.so")

CC_OK, CC_EINVAL, CC_EIDRANGE, CC_ENOMEM, CC_ECUDA, CC_ENOTCONVERGED, CC_ETIMEOUT = range(7)
CC_ID32, CC_ID64 = 32, 64
CC_COO, CC_CSR, CC_CSR_NATIVE, CC_CSR_NATIVE_SYM = 0, 1, 2, 3
CC_SYNC, CC_ASYNC, CC_ASYNC_COMPACT = 0, 1, 2
CC_ORDER_FULL, CC_ORDER_AUTO = 0, -1
CC_ORDER_11MM, CC_ORDER_1M1M = -2, -3
CC_NOALLOC_MAX_N = 4194304


class cc_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("order", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("check_interval", ctypes.c_int32), ("solve_ms", ctypes.c_double),
                ("edges_per_s", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("loop_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CCError(RuntimeError):
    """A libcontour call returned a status other than CC_OK."""

    def __init__(self, status, where, detail, stats=None):
        super().__init__(f"{where}: {cc_strerror(status)} ({detail})")
        self.status = status
        self.stats = stats


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_2311_02811_gb300.build.build() "
                      "(needs nvcc); there is no CPU fallback")

lib = ctypes.CDLL(LIB_PATH)
_p, _i64, _i32, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
lib.cc_init.argtypes = [ctypes.POINTER(_p), _i64, _int, _int, _p, _p, _i64, _int, _p]
lib.cc_init.restype = _int
lib.cc_run.argtypes = [_p, _int, _int, _int, _i32, _p, _p, _int, ctypes.POINTER(cc_stats)]
lib.cc_run.restype = _int
lib.cc_run_noalloc.argtypes = [_i64, _p, _p, _i64, _int, _int, _int, _i32, _p,
                               ctypes.POINTER(_i32), _p]
lib.cc_solve_host.argtypes = [_i64, _p, _p, _i64, _int, _int, _int, _i32, _p, _int,
                              ctypes.POINTER(cc_stats), _p]
lib.cc_solve_host.restype = _int
lib.cc_run_noalloc.restype = _int
lib.cc_graph_info.argtypes = [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
lib.cc_graph_info.restype = _int
lib.cc_graph_set_stream.argtypes = [_p, _p]
lib.cc_graph_set_stream.restype = _int
lib.cc_free.argtypes = [_p]
lib.cc_free.restype = None
lib.cc_strerror.argtypes = [_int]
lib.cc_strerror.restype = ctypes.c_char_p
lib.cc_last_error.argtypes = []
lib.cc_last_error.restype = ctypes.c_char_p


def cc_strerror(status: int) -> str:
    return lib.cc_strerror(status).decode()


def cc_last_error() -> str:
    return lib.cc_last_error().decode()


def _check(status, where, stats=None):
    if status != CC_OK:
        raise CCError(status, where, cc_last_error(), stats)


def _ptr(x):
    """(pointer, on_device) of a torch tensor / numpy array / None / int."""
    if x is None:
        return None, False
    if isinstance(x, int):
        return x, False
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return x.data_ptr(), x.device.type == "cuda"
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return x.ctypes.data, False
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is not None:
        return int(stream)
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return 0


def _id_bits(x, default=CC_ID32):
    dt = str(getattr(x, "dtype", ""))
    if "int64" in dt:
        return CC_ID64
    if "int32" in dt:
        return CC_ID32
    return default


class cc_graph:
    """A cc_graph* handle.  Device arrays that cc_init may borrow are referenced
    here so that Python keeps them alive until cc_free."""

    def __init__(self, ptr, keep):
        self._as_parameter_ = _p(ptr)
        self._keep = keep

    @property
    def ptr(self):
        return self._as_parameter_.value


def cc_init(n, a, b, m=None, id_bits=None, layout=CC_COO, on_device=None, stream=None):
    """Create a graph handle; see cc_init in contour.h."""
    pa, da = _ptr(a)
    pb, db = _ptr(b)
    if m is None:
        m = len(b) if b is not None else 0
    if id_bits is None:
        id_bits = _id_bits(b)
    if on_device is None:
        on_device = da or db
    g = _p()
    _check(lib.cc_init(ctypes.byref(g), int(n), int(id_bits), int(layout), pa, pb, int(m),
                       int(bool(on_device)), _stream(stream)), "cc_init")
    return cc_graph(g.value, (a, b) if on_device else ())


def cc_run(g, labels_out, order=2, mode=CC_ASYNC, check_interval=1, max_sweeps=1 << 20,
           init_labels=None, out_on_device=None, raise_on_error=True):
    """Label every vertex with its component's minimum id; returns cc_stats."""
    po, do = _ptr(labels_out)
    pi, _ = _ptr(init_labels)
    if out_on_device is None:
        out_on_device = do
    st = cc_stats()
    rc = lib.cc_run(g, int(order), int(mode), int(check_interval), int(max_sweeps), pi, po,
                    int(bool(out_on_device)), ctypes.byref(st))
    if raise_on_error:
        _check(rc, "cc_run", st)
        return st
    return rc, st


def cc_solve_host(n, src, dst, labels_out, order=2, mode=CC_ASYNC, check_interval=1, max_sweeps=1 << 20,
                  out_on_device=None, stream=None, raise_on_error=True):
    """One solve of int32 edges held in host memory, the upload overlapped with
    sweeps (cc_solve_host in contour.h); returns cc_stats."""
    def host_i32(x, what):
        if hasattr(x, "data_ptr") and x.device.type != "cpu":
            raise ValueError(f"cc_solve_host: {what} must be host memory (use cc_init + cc_run for device edges)")
        if "int32" not in str(getattr(x, "dtype", "")):
            raise ValueError(f"cc_solve_host: {what} must be int32")
        return _ptr(x)[0]

    ps = host_i32(src, "src")
    pd = host_i32(dst, "dst")
    po, do = _ptr(labels_out)
    if out_on_device is None:
        out_on_device = do
    st = cc_stats()
    rc = lib.cc_solve_host(int(n), ps, pd, len(src), int(order), int(mode), int(check_interval),
                           int(max_sweeps), po, int(bool(out_on_device)), ctypes.byref(st), _stream(stream))
    if raise_on_error:
        _check(rc, "cc_solve_host", st)
        return st
    return rc, st


def cc_run_noalloc(n, src, dst, labels_out, order=2, mode=CC_ASYNC, check_interval=1,
                   max_sweeps=1 << 20, stream=None, raise_on_error=True, m=None):
    """cc_run without any device allocation (int32 device arrays); returns sweeps.

    See cc_run_noalloc in contour.h: for callers that must not allocate device
    memory; scratch comes from a fixed array inside the library."""
    def dev_i32(x, what):
        # a host array would reach the kernels as a host address, and an
        # int64 tensor would be read as pairs of int32 ids: refuse both here
        # (the library also refuses memory that is not on the current device)
        if x is None or isinstance(x, int):
            return x
        if not hasattr(x, "data_ptr") or x.device.type != "cuda":
            raise ValueError(f"cc_run_noalloc: {what} must be a CUDA tensor (or a device pointer)")
        if str(x.dtype) != "torch.int32":
            raise ValueError(f"cc_run_noalloc: {what} must be int32, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"cc_run_noalloc: {what} must be contiguous")
        return x.data_ptr()

    ps = dev_i32(src, "src")
    pd = dev_i32(dst, "dst")
    po = dev_i32(labels_out, "labels_out")
    sw = _i32(0)
    m = m if m is not None else (len(src) if src is not None and not isinstance(src, int) else 0)
    rc = lib.cc_run_noalloc(int(n), ps, pd, int(m), int(order),
                            int(mode), int(check_interval), int(max_sweeps), po,
                            ctypes.byref(sw), _stream(stream))
    if raise_on_error:
        _check(rc, "cc_run_noalloc")
        return sw.value
    return rc, sw.value


lib.cc_batch_init.argtypes = [ctypes.POINTER(_p), _i32, _p, _p, _p, _p, _int, _p]
lib.cc_batch_init.restype = _int
lib.cc_batch_run.argtypes = [_p, _int, _int, _int, _i32, _p, _p, ctypes.POINTER(ctypes.c_double)]
lib.cc_batch_run.restype = _int
lib.cc_batch_set_schedule.argtypes = [_p, _p, _p, _p]
lib.cc_batch_set_schedule.restype = _int
lib.cc_batch_run_scheduled.argtypes = [_p, _i32, _p, _p, ctypes.POINTER(ctypes.c_double)]
lib.cc_batch_run_scheduled.restype = _int
lib.cc_batch_tuning.argtypes = [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
lib.cc_batch_tuning.restype = _int
lib.cc_batch_set_tuning.argtypes = [_p, _i32, _i32, _i32]
lib.cc_batch_set_tuning.restype = _int
lib.cc_batch_free.argtypes = [_p]
lib.cc_batch_free.restype = None
lib.cc_batch.argtypes = [_i32, _p, _p, _p, _p, _int, _int, _int, _p, _p, _p]
lib.cc_batch.restype = _int


class cc_batch_plan:
    """A cc_batch_plan* handle; keeps the borrowed device edge arrays alive."""

    def __init__(self, ptr, n_graphs, total_n, keep):
        self._as_parameter_ = _p(ptr)
        self.n_graphs = n_graphs
        self.total_n = total_n
        self._keep = keep


def _i64_host(a):
    import numpy as np
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


def _i32_host(a):
    import numpy as np
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def cc_batch_init(vtx_off, edge_off, src, dst, autotune=0, stream=None):
    """Plan a batched solve (offsets on the host, edges on the device)."""
    vo, eo = _i64_host(vtx_off), _i64_host(edge_off)
    ps, _ = _ptr(src)
    pd, _ = _ptr(dst)
    b = _p()
    G = len(vo) - 1
    _check(lib.cc_batch_init(ctypes.byref(b), G, vo.ctypes.data, eo.ctypes.data, ps, pd,
                             int(autotune), _stream(stream)), "cc_batch_init")
    return cc_batch_plan(b.value, G, int(vo[-1]) if G else 0, (src, dst))


def cc_batch_run(b, labels_out, order=2, mode=CC_ASYNC, check_interval=1, max_sweeps=1 << 20,
                 raise_on_error=True):
    """Solve every graph of the plan; returns (sweeps per graph, solve_ms)."""
    import numpy as np
    po, _ = _ptr(labels_out)
    sweeps = np.zeros(b.n_graphs, dtype=np.int32)
    ms = ctypes.c_double(0.0)
    rc = lib.cc_batch_run(b, int(order), int(mode), int(check_interval), int(max_sweeps), po,
                          sweeps.ctypes.data, ctypes.byref(ms))
    if raise_on_error:
        _check(rc, "cc_batch_run")
        return sweeps, ms.value
    return rc, sweeps, ms.value


def cc_batch_set_schedule(b, order, mode, check_interval):
    o, m_, c = _i32_host(order), _i32_host(mode), _i32_host(check_interval)
    _check(lib.cc_batch_set_schedule(b, o.ctypes.data, m_.ctypes.data, c.ctypes.data),
           "cc_batch_set_schedule")


def cc_batch_run_scheduled(b, labels_out, max_sweeps=1 << 20, raise_on_error=True):
    import numpy as np
    po, _ = _ptr(labels_out)
    sweeps = np.zeros(b.n_graphs, dtype=np.int32)
    ms = ctypes.c_double(0.0)
    rc = lib.cc_batch_run_scheduled(b, int(max_sweeps), po, sweeps.ctypes.data, ctypes.byref(ms))
    if raise_on_error:
        _check(rc, "cc_batch_run_scheduled")
        return sweeps, ms.value
    return rc, sweeps, ms.value


def cc_batch_tuning(b):
    x, y, z = _i32(), _i32(), _i32()
    _check(lib.cc_batch_tuning(b, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z)), "cc_batch_tuning")
    return x.value, y.value, z.value


def cc_batch_set_tuning(b, smem_budget, threads=512, edges_per_thread=4):
    _check(lib.cc_batch_set_tuning(b, int(smem_budget), int(threads), int(edges_per_thread)),
           "cc_batch_set_tuning")


lib.cc_batch_reorder.argtypes = [_p]
lib.cc_batch_reorder.restype = _int


def cc_batch_reorder(b):
    """Group every graph's edges by its lower-degree endpoint (labels unchanged)."""
    _check(lib.cc_batch_reorder(b), "cc_batch_reorder")
    if isinstance(b, cc_batch_plan):
        b._keep = ()


lib.cc_batch_edges.argtypes = [_p, ctypes.POINTER(_p), ctypes.POINTER(_p)]
lib.cc_batch_edges.restype = _int


def cc_batch_edges(b):
    """(src, dst) device pointers (ints) of the plan's edge arrays."""
    a, c = _p(), _p()
    _check(lib.cc_batch_edges(b, ctypes.byref(a), ctypes.byref(c)), "cc_batch_edges")
    return a.value, c.value


def cc_batch_free(b):
    lib.cc_batch_free(b)
    if isinstance(b, cc_batch_plan):
        b._as_parameter_ = _p(None)
        b._keep = ()


def cc_batch(vtx_off, edge_off, src, dst, labels_out, order=2, mode=CC_ASYNC, check_interval=1,
             stream=None):
    """One-shot batched solve; returns the sweeps per graph."""
    import numpy as np
    vo, eo = _i64_host(vtx_off), _i64_host(edge_off)
    ps, _ = _ptr(src)
    pd, _ = _ptr(dst)
    po, _ = _ptr(labels_out)
    sweeps = np.zeros(len(vo) - 1, dtype=np.int32)
    _check(lib.cc_batch(len(vo) - 1, vo.ctypes.data, eo.ctypes.data, ps, pd, int(order), int(mode),
                        int(check_interval), po, sweeps.ctypes.data, _stream(stream)), "cc_batch")
    return sweeps


CC_SCHED_FEATURES, CC_SCHED_CLASSES = 12, 18
_f = ctypes.c_float
lib.cc_sched_load.argtypes = [_p, ctypes.c_size_t]
lib.cc_sched_load.restype = _int
lib.cc_sched_blob_bytes.argtypes = []
lib.cc_sched_blob_bytes.restype = ctypes.c_size_t
lib.cc_sched_param_count.argtypes = []
lib.cc_sched_param_count.restype = _i32
lib.cc_sched_decode.argtypes = [_i32, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]
lib.cc_sched_decode.restype = _int
lib.cc_graph_features.argtypes = [_p, _p]
lib.cc_graph_features.restype = _int
lib.cc_batch_features.argtypes = [_p, _p]
lib.cc_batch_features.restype = _int
lib.cc_sched_predict.argtypes = [_p, _i32, _p, _p]
lib.cc_sched_predict.restype = _int
lib.cc_sched_predict_batch.argtypes = [_p, _i32, _p, _p]
lib.cc_sched_predict_batch.restype = _int
lib.cc_sched_load_batch.argtypes = [_p, ctypes.c_size_t]
lib.cc_sched_load_batch.restype = _int
lib.cc_sched_train.argtypes = [_p, _p, _i32, _p, _i32, _i32, _f, ctypes.c_uint64, _p, ctypes.POINTER(_f)]
lib.cc_sched_train.restype = _int
lib.cc_sched_train_step.argtypes = [_p, _p, _i32, _p, _f, ctypes.POINTER(_f)]
lib.cc_sched_train_step.restype = _int


def cc_sched_load(blob):
    """Install scheduler weights (bytes); None restores the plain fallback."""
    if blob is None:
        _check(lib.cc_sched_load(None, 0), "cc_sched_load")
        return
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(lib.cc_sched_load(buf, len(blob)), "cc_sched_load")


def cc_sched_load_batch(blob):
    """Install the weights batched solves use (bytes); None: batches use the
    single-graph weights."""
    if blob is None:
        _check(lib.cc_sched_load_batch(None, 0), "cc_sched_load_batch")
        return
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(lib.cc_sched_load_batch(buf, len(blob)), "cc_sched_load_batch")


SCHED_WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sched_weights.bin")
SCHED_BATCH_WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sched_weights_batch.bin")


def load_default_scheduler(path=None, batch_path=None):
    """Install the committed scheduler weights (written by sched_train.py):
    the single-graph model and, when present, the one for batched solves."""
    with open(path or SCHED_WEIGHTS_PATH, "rb") as f:
        cc_sched_load(f.read())
    bp = batch_path or SCHED_BATCH_WEIGHTS_PATH
    if os.path.exists(bp):
        with open(bp, "rb") as f:
            cc_sched_load_batch(f.read())


def unload_scheduler():
    """Remove both scheduler models (AUTO falls back to the plain schedule)."""
    cc_sched_load(None)
    cc_sched_load_batch(None)


def cc_sched_blob_bytes():
    return lib.cc_sched_blob_bytes()


def cc_sched_param_count():
    return lib.cc_sched_param_count()


def cc_sched_decode(cls):
    o, m_, c = _int(), _int(), _int()
    _check(lib.cc_sched_decode(int(cls), ctypes.byref(o), ctypes.byref(m_), ctypes.byref(c)), "cc_sched_decode")
    return o.value, m_.value, c.value


def cc_graph_features(g):
    import numpy as np
    out = np.zeros(CC_SCHED_FEATURES, dtype=np.float32)
    _check(lib.cc_graph_features(g, out.ctypes.data), "cc_graph_features")
    return out


def cc_batch_features(b):
    import numpy as np
    out = np.zeros((b.n_graphs, CC_SCHED_FEATURES), dtype=np.float32)
    _check(lib.cc_batch_features(b, out.ctypes.data), "cc_batch_features")
    return out


def cc_sched_predict(features, batch_model=False):
    """(classes, logits) of the single-graph model (or of the batch model)."""
    import numpy as np
    f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, CC_SCHED_FEATURES)
    cls = np.zeros(len(f), dtype=np.int32)
    logits = np.zeros((len(f), CC_SCHED_CLASSES), dtype=np.float32)
    fn = lib.cc_sched_predict_batch if batch_model else lib.cc_sched_predict
    _check(fn(f.ctypes.data, len(f), cls.ctypes.data, logits.ctypes.data), "cc_sched_predict")
    return cls, logits


def cc_sched_predict_batch(features):
    return cc_sched_predict(features, batch_model=True)


def cc_sched_train(features, labels, epochs=60, batch=256, lr=2e-3, seed=1, init_params=None):
    """Train the scheduler MLP on the GPU; returns (blob bytes, final mean loss)."""
    import numpy as np
    f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, CC_SCHED_FEATURES)
    y = np.ascontiguousarray(labels, dtype=np.int32)
    ip = None if init_params is None else np.ascontiguousarray(init_params, dtype=np.float32)
    blob = ctypes.create_string_buffer(cc_sched_blob_bytes())
    loss = _f(0)
    _check(lib.cc_sched_train(f.ctypes.data, y.ctypes.data, len(f), None if ip is None else ip.ctypes.data,
                              int(epochs), int(batch), float(lr), int(seed), blob, ctypes.byref(loss)),
           "cc_sched_train")
    return blob.raw, loss.value


def cc_sched_train_step(features_std, labels, params, lr):
    """One Adam step from zero moments; returns (new params, loss)."""
    import numpy as np
    f = np.ascontiguousarray(features_std, dtype=np.float32).reshape(-1, CC_SCHED_FEATURES)
    y = np.ascontiguousarray(labels, dtype=np.int32)
    p = np.array(params, dtype=np.float32)
    loss = _f(0)
    _check(lib.cc_sched_train_step(f.ctypes.data, y.ctypes.data, len(f), p.ctypes.data, float(lr),
                                   ctypes.byref(loss)), "cc_sched_train_step")
    return p, loss.value


CC_REORDER_SRC, CC_REORDER_LOWDEG, CC_REORDER_HUB, CC_REORDER_DEGREE = 1, 2, 3, 4
lib.cc_graph_reorder.argtypes = [_p, _int]
lib.cc_graph_reorder.restype = _int


def cc_graph_reorder(g, method=CC_REORDER_LOWDEG):
    """Reorder the handle's edges for label locality (labels are unchanged)."""
    _check(lib.cc_graph_reorder(g, int(method)), "cc_graph_reorder")
    if isinstance(g, cc_graph):
        g._keep = ()  # the handle now owns its edges


lib.cc_graph_edges.argtypes = [_p, ctypes.POINTER(_p), ctypes.POINTER(_p)]
lib.cc_graph_edges.restype = _int


def cc_graph_edges(g):
    """(src, dst) device pointers (ints) of the handle's edge arrays."""
    a, b = _p(), _p()
    _check(lib.cc_graph_edges(g, ctypes.byref(a), ctypes.byref(b)), "cc_graph_edges")
    return a.value, b.value


lib.cc_graph_hubs.argtypes = [_p, ctypes.POINTER(_p), ctypes.POINTER(_i32)]
lib.cc_graph_hubs.restype = _int


def cc_graph_hubs(g):
    """(device pointer, count) of the hub table of a CC_REORDER_HUB handle."""
    a, k = _p(), _i32(0)
    _check(lib.cc_graph_hubs(g, ctypes.byref(a), ctypes.byref(k)), "cc_graph_hubs")
    return a.value, k.value


lib.cc_graph_perm.argtypes = [_p, ctypes.POINTER(_p), ctypes.POINTER(_p)]
lib.cc_graph_perm.restype = _int


def cc_graph_perm(g):
    """(perm, inv) device pointers (ints) of a CC_REORDER_DEGREE handle's id maps
    (perm[x] = new id of vertex x); (None, None) for other handles."""
    a, b = _p(), _p()
    _check(lib.cc_graph_perm(g, ctypes.byref(a), ctypes.byref(b)), "cc_graph_perm")
    return a.value, b.value


CC_LAUNCH_GRAPH, CC_LAUNCH_HOST = 0, 1
lib.cc_graph_set_launch.argtypes = [_p, _int]
lib.cc_graph_set_launch.restype = _int


def cc_graph_set_launch(g, launch):
    """CC_LAUNCH_GRAPH (device-side loop) or CC_LAUNCH_HOST (host-polled blocks)."""
    _check(lib.cc_graph_set_launch(g, int(launch)), "cc_graph_set_launch")


def cc_graph_info(g):
    n, m = _i64(), _i64()
    _check(lib.cc_graph_info(g, ctypes.byref(n), ctypes.byref(m)), "cc_graph_info")
    return n.value, m.value


def cc_graph_set_stream(g, stream):
    _check(lib.cc_graph_set_stream(g, int(stream)), "cc_graph_set_stream")


lib.cc_release_memory.argtypes = []
lib.cc_release_memory.restype = _int


def cc_release_memory():
    """Return the library's unused pooled device memory to the device."""
    _check(lib.cc_release_memory(), "cc_release_memory")


def cc_free(g):
    lib.cc_free(g)
    if isinstance(g, cc_graph):
        g._as_parameter_ = _p(None)
        g._keep = ()
