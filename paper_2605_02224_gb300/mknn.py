"""Thin ctypes binding of the C ABI in include/mknn.h (argument marshalling only).

Every function keeps the C name. Device arrays are passed as integers
(e.g. torch.Tensor.data_ptr()); host arrays as numpy arrays. Failures raise
MknnError with the library's message. Nothing here computes any part of
the k-NN path: all of it runs in libmknn.so.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmknn.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBUSY", 5: "ETIMEOUT",
          6: "EDEGENERATE", 7: "EIO"}
MKNN_MAX_K = 128


class MknnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mknn_build_opts(C.Structure):
    _fields_ = [("keep_tets", C.c_int32), ("dynamic", C.c_int32), ("reserved", C.c_int32 * 6)]


class mknn_build_stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in (
        "n", "entries", "duplicates", "degenerate_prefix", "tets_final", "walk_steps",
        "conflict_tests", "orient_calls", "orient_exact", "insphere_calls", "insphere_exact")] + [
        ("build_seconds", C.c_double)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class mknn_knn_opts(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("sort", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("counters", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("order", C.c_void_p),
                ("placement", C.c_int32), ("reserved", C.c_int32 * 3)]


class mknn_batch_req(C.Structure):
    _fields_ = [("cloud", C.c_void_p), ("q", C.c_void_p), ("nq", C.c_int64),
                ("q_stride", C.c_int32), ("k", C.c_int32), ("m", C.c_void_p),
                ("m_scalar", C.c_int32), ("out_idx", C.c_void_p), ("out_d2", C.c_void_p)]


class mknn_batch_opts(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("sort", C.c_int32), ("item_rounds", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("graph", C.c_int32), ("placement", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class mknn_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("plain", C.c_int32), ("mem_budget", C.c_size_t),
                ("max_batch_queries", C.c_int64), ("lanes", C.c_int32),
                ("reserved", C.c_int32 * 7)]


class mknn_request(C.Structure):
    _fields_ = [("cloud", C.c_int32), ("k", C.c_int32), ("m", C.c_int32),
                ("reserved", C.c_int32), ("q", C.c_void_p), ("nq", C.c_int64),
                ("out_idx", C.c_void_p), ("out_d2", C.c_void_p)]


class mknn_serving_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "queries",
                                         "launches")] + \
               [(n, C.c_double) for n in ("elapsed_s", "qps", "p50_ms", "p99_ms", "mean_ms",
                                          "max_ms", "mean_requests_per_launch", "h2d_ms",
                                          "kernel_ms", "d2h_ms")]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


_lib = None


def lib():
    """The loaded libmknn.so. Raises if the library has not been built:
    there is no fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(
                f"{_LIB_PATH} not found: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        _lib = C.CDLL(_LIB_PATH)
        _declare(_lib)
    return _lib


def _declare(L):
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    pp = C.POINTER(C.c_void_p)
    sig = {
        "mknn_last_error": (C.c_char_p, []),
        "mknn_version": (C.c_char_p, []),
        "mknn_build": (i32, [vp, i64, vp, vp, pp]),
        "mknn_cloud_from_table": (i32, [vp, i64, vp, vp, pp]),
        "mknn_cloud_upload": (i32, [vp, vp]),
        "mknn_cloud_release_device": (i32, [vp]),
        "mknn_cloud_free": (i32, [vp]),
        "mknn_cloud_info": (i32, [vp, vp, vp, vp]),
        "mknn_cloud_order": (i32, [vp, vp]),
        "mknn_cloud_trees": (i32, [vp, vp, vp]),
        "mknn_cloud_table": (i32, [vp, vp, vp, vp]),
        "mknn_cloud_stats": (i32, [vp, vp]),
        "mknn_cloud_tets": (i32, [vp, vp, vp]),
        "mknn_cloud_save": (i32, [vp, C.c_char_p]),
        "mknn_cloud_load": (i32, [C.c_char_p, pp]),
        "mknn_knn": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_knn_workspace_size": (sz, [i64, vp]),
        "mknn_knn_ex": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp, vp]),
        "mknn_knn_host": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_knn_sites": (i32, [vp, vp, i64, i32, vp, i32, vp, vp, vp, vp]),
        "mknn_cloud_append": (i32, [vp, vp, i64, vp]),
        "mknn_insertion_order": (i32, [vp, i64, i32, C.c_uint64, vp]),
        "mknn_hilbert_index3": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32, i32]),
        "mknn_cloud_compact": (i32, [vp, vp]),
        "mknn_knn_sites_workspace_size": (C.c_size_t, [i64, vp]),
        "mknn_cloud_check": (i32, [vp, vp]),
        "mknn_query_order_workspace_size": (sz, [i64]),
        "mknn_query_order": (i32, [vp, vp, i64, i32, vp, vp, sz, vp]),
        "mknn_cloud_validate": (i32, [vp, vp, vp]),
        "mknn_knn_noalloc": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_knn_noalloc_max_queries": (i64, []),
        "mknn_read_probe": (i32, [vp, sz, i32, vp, vp]),
        "mknn_batch_create": (i32, [vp, i32, vp, pp]),
        "mknn_batch_run": (i32, [vp, vp]),
        "mknn_batch_info": (i32, [vp, vp, vp, vp]),
        "mknn_batch_placement": (i32, [vp, vp]),
        "mknn_batch_free": (i32, [vp]),
        "mknn_knn_batch": (i32, [vp, i32, vp, vp]),
        "mknn_batch_tune": (i32, [vp, i32, i64, vp]),
        "mknn_tune_save": (i32, [C.c_char_p]),
        "mknn_tune_load": (i32, [C.c_char_p]),
        "mknn_tune_clear": (i32, []),
        "mknn_server_create": (i32, [vp, pp]),
        "mknn_server_add_cloud": (i32, [vp, vp, vp]),
        "mknn_server_submit": (i32, [vp, vp, vp]),
        "mknn_server_poll": (i32, [vp, C.c_uint64, vp]),
        "mknn_server_drain": (i32, [vp, C.c_double]),
        "mknn_server_stats": (i32, [vp, vp]),
        "mknn_server_latencies": (i32, [vp, vp, i64, vp]),
        "mknn_server_reset_stats": (i32, [vp]),
        "mknn_server_destroy": (i32, [vp, C.c_double]),
        "mknn_orient3d": (i32, [vp, vp, vp, vp]),
        "mknn_insphere": (i32, [vp, vp, vp, vp, vp]),
        "mknn_orient3d_exact": (i32, [vp, vp, vp, vp]),
        "mknn_insphere_exact": (i32, [vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _check(status: int):
    if status != 0:
        raise MknnError(status, lib().mknn_last_error().decode())


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ---------------------------------------------------------------- build / cloud

def mknn_build(xyz, order=None, keep_tets: bool = False, dynamic: bool = False) -> int:
    """Builds the successor table on the host; returns the cloud handle."""
    x = _host(xyz, np.float32).reshape(-1, 3)
    o = None if order is None else _host(order, np.int64)
    opts = mknn_build_opts(keep_tets=1 if keep_tets else 0, dynamic=1 if dynamic else 0)
    out = C.c_void_p()
    _check(lib().mknn_build(_ptr(x), x.shape[0], _ptr(o), C.addressof(opts), C.byref(out)))
    return out.value


def mknn_cloud_append(cloud: int, xyz, stream: int = 0):
    """Appends points (host float32 (count, 3), in birth order) to a cloud
    built with dynamic=True."""
    x = _host(xyz, np.float32).reshape(-1, 3)
    _check(lib().mknn_cloud_append(cloud, _ptr(x), x.shape[0], stream or None))


def mknn_cloud_compact(cloud: int, stream: int = 0):
    _check(lib().mknn_cloud_compact(cloud, stream or None))


ORDER_RANDOM, ORDER_BRIO_HILBERT, ORDER_FARTHEST_POINT = 0, 1, 2


def mknn_insertion_order(xyz, kind: int, seed: int = 0) -> np.ndarray:
    """Birth order (int64 input indices by rank) of host points (n, 3)."""
    x = _host(xyz, np.float32).reshape(-1, 3)
    out = np.empty(x.shape[0], np.int64)
    _check(lib().mknn_insertion_order(_ptr(x), x.shape[0], kind, seed, _ptr(out)))
    return out


def mknn_hilbert_index3(x: int, y: int, z: int, bits: int) -> int:
    return int(lib().mknn_hilbert_index3(x, y, z, bits))


def mknn_cloud_from_table(xyz_ranked, rowp, succ) -> int:
    x = _host(xyz_ranked, np.float32).reshape(-1, 3)
    r = _host(rowp, np.int64)
    s = _host(succ, np.int32)
    out = C.c_void_p()
    _check(lib().mknn_cloud_from_table(_ptr(x), x.shape[0], _ptr(r), _ptr(s) if s.size else None,
                                       C.byref(out)))
    return out.value


def mknn_cloud_upload(cloud: int, stream: int = 0):
    _check(lib().mknn_cloud_upload(cloud, stream or None))


def mknn_cloud_release_device(cloud: int):
    _check(lib().mknn_cloud_release_device(cloud))


def mknn_cloud_free(cloud: int):
    _check(lib().mknn_cloud_free(cloud))


def mknn_cloud_info(cloud: int):
    n, E, b = C.c_int64(), C.c_int64(), C.c_size_t()
    _check(lib().mknn_cloud_info(cloud, C.byref(n), C.byref(E), C.byref(b)))
    return n.value, E.value, b.value


def mknn_cloud_trees(cloud: int):
    t, e = C.c_int64(), C.c_int64()
    _check(lib().mknn_cloud_trees(cloud, C.byref(t), C.byref(e)))
    return t.value, e.value


def mknn_cloud_order(cloud: int) -> np.ndarray:
    n, _, _ = mknn_cloud_info(cloud)
    out = np.empty(n, np.int64)
    _check(lib().mknn_cloud_order(cloud, _ptr(out)))
    return out


def mknn_cloud_table(cloud: int):
    n, E, _ = mknn_cloud_info(cloud)
    xyz = np.empty((n, 3), np.float32)
    rowp = np.empty(n + 1, np.int64)
    succ = np.empty(E, np.int32)
    _check(lib().mknn_cloud_table(cloud, _ptr(xyz), _ptr(rowp), _ptr(succ) if E else None))
    return xyz, rowp, succ


def mknn_cloud_stats(cloud: int) -> dict:
    s = mknn_build_stats()
    _check(lib().mknn_cloud_stats(cloud, C.addressof(s)))
    return s.as_dict()


def mknn_cloud_tets(cloud: int) -> np.ndarray:
    cnt = C.c_int64()
    _check(lib().mknn_cloud_tets(cloud, None, C.byref(cnt)))
    out = np.empty((cnt.value, 4), np.int32)
    _check(lib().mknn_cloud_tets(cloud, _ptr(out) if cnt.value else None, C.byref(cnt)))
    return out


def mknn_cloud_save(cloud: int, path: str):
    _check(lib().mknn_cloud_save(cloud, path.encode()))


def mknn_cloud_load(path: str) -> int:
    out = C.c_void_p()
    _check(lib().mknn_cloud_load(path.encode(), C.byref(out)))
    return out.value


# ---------------------------------------------------------------- queries

def _opts(lanes=0, sort=0, blocks_per_sm=0, counters=None, workspace=None, workspace_bytes=0,
          order=None, placement=0):
    return mknn_knn_opts(lanes=lanes, sort=sort, blocks_per_sm=blocks_per_sm,
                         counters=_ptr(counters), workspace=_ptr(workspace),
                         workspace_bytes=workspace_bytes, order=_ptr(order),
                         placement=placement)


def mknn_query_order_workspace_size(nq: int) -> int:
    return int(lib().mknn_query_order_workspace_size(nq))


def mknn_query_order(cloud: int, q, nq: int, q_stride: int, perm_out, workspace=None,
                     workspace_bytes: int = 0, stream: int = 0):
    _check(lib().mknn_query_order(cloud, _ptr(q), nq, q_stride, _ptr(perm_out), _ptr(workspace),
                                  workspace_bytes, stream or None))


def mknn_knn(cloud: int, q, nq: int, q_stride: int, k: int, m, m_scalar: int, out_idx, out_d2,
             stream: int = 0):
    """Device pointers (ints or tensors) in, results written to out_idx/out_d2."""
    _check(lib().mknn_knn(cloud, _ptr(q), nq, q_stride, k, _ptr(m), m_scalar, _ptr(out_idx),
                          _ptr(out_d2), stream or None))


def mknn_knn_workspace_size(nq: int, **opt) -> int:
    o = _opts(**opt)
    return int(lib().mknn_knn_workspace_size(nq, C.addressof(o)))


def mknn_knn_ex(cloud: int, q, nq: int, q_stride: int, k: int, m, m_scalar: int, out_idx,
                out_d2, stream: int = 0, **opt):
    o = _opts(**opt)
    _check(lib().mknn_knn_ex(cloud, _ptr(q), nq, q_stride, k, _ptr(m), m_scalar, _ptr(out_idx),
                             _ptr(out_d2), C.addressof(o), stream or None))


def mknn_knn_sites(cloud: int, sites, nq: int, k: int, m, m_scalar: int, out_idx, out_d2,
                   stream: int = 0, **opt):
    """Same-manifold queries: query i is the cloud's site of rank sites[i]
    (device int32)."""
    o = _opts(**opt)
    _check(lib().mknn_knn_sites(cloud, _ptr(sites), nq, k, _ptr(m), m_scalar, _ptr(out_idx),
                                _ptr(out_d2), C.addressof(o), stream or None))


def mknn_knn_sites_workspace_size(nq: int, **opt) -> int:
    o = _opts(**opt)
    return int(lib().mknn_knn_sites_workspace_size(nq, C.addressof(o)))


def mknn_knn_host(cloud: int, q, k: int, m=None, m_scalar: int = 0, out_idx=None, out_d2=None,
                  stream: int = 0):
    """Host arrays in and out (numpy or pinned torch CPU tensors)."""
    if isinstance(q, np.ndarray):
        q = np.ascontiguousarray(q, np.float32)
        nq, stride = q.shape[0], q.shape[1]
    else:
        nq, stride = int(q.shape[0]), int(q.shape[1])
    if out_idx is None:
        out_idx = np.empty((nq, k), np.int32)
    if out_d2 is None:
        out_d2 = np.empty((nq, k), np.float32)
    if isinstance(m, np.ndarray):
        m = np.ascontiguousarray(m, np.int32)
    _check(lib().mknn_knn_host(cloud, _ptr(q), nq, stride, k, _ptr(m), m_scalar, _ptr(out_idx),
                               _ptr(out_d2), stream or None))
    return out_idx, out_d2


def mknn_knn_noalloc(cloud: int, q, nq: int, q_stride: int, k: int, m, m_scalar: int, out_idx,
                     out_d2, stream: int = 0):
    """mknn_knn for callers that cannot allocate device memory during a
    call: its scratch is a fixed array inside the library (up to
    mknn_knn_noalloc_max_queries() queries per call; concurrent calls on
    one device must be serialised)."""
    _check(lib().mknn_knn_noalloc(cloud, _ptr(q), nq, q_stride, k, _ptr(m), m_scalar,
                                  _ptr(out_idx), _ptr(out_d2), stream or None))


def mknn_knn_noalloc_max_queries() -> int:
    return int(lib().mknn_knn_noalloc_max_queries())


def mknn_read_probe(buf, nbytes: int, passes: int, sink, stream: int = 0):
    """Reads nbytes of the device buffer `passes` times (read-bandwidth probe)."""
    _check(lib().mknn_read_probe(_ptr(buf), nbytes, passes, _ptr(sink), stream or None))


# ---------------------------------------------------------------- batches

def batch_reqs(reqs):
    """reqs: list of dicts with cloud, q, nq, q_stride, k, m, m_scalar,
    out_idx, out_d2 (device pointers or tensors) -> ctypes array."""
    arr = (mknn_batch_req * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        arr[i] = mknn_batch_req(cloud=r["cloud"], q=_ptr(r["q"]), nq=int(r["nq"]),
                                q_stride=int(r.get("q_stride", 3)), k=int(r["k"]),
                                m=_ptr(r.get("m")), m_scalar=int(r.get("m_scalar", 0)),
                                out_idx=_ptr(r["out_idx"]), out_d2=_ptr(r["out_d2"]))
    return arr


def mknn_batch_create(reqs, lanes=0, sort=0, item_rounds=0, blocks_per_sm=0, graph=0,
                      placement=0) -> int:
    arr = batch_reqs(reqs)
    o = mknn_batch_opts(lanes=lanes, sort=sort, item_rounds=item_rounds,
                        blocks_per_sm=blocks_per_sm, graph=graph, placement=placement)
    out = C.c_void_p()
    _check(lib().mknn_batch_create(arr, len(reqs), C.addressof(o), C.byref(out)))
    return out.value


def mknn_batch_run(plan: int, stream: int = 0):
    _check(lib().mknn_batch_run(plan, stream or None))


def mknn_batch_info(plan: int, nreq: int):
    lanes = np.zeros(max(1, nreq), np.int32)
    items, grid = C.c_int64(), C.c_int32()
    _check(lib().mknn_batch_info(plan, _ptr(lanes), C.byref(items), C.byref(grid)))
    return lanes[:nreq], items.value, grid.value


def mknn_batch_placement(plan: int, nreq: int):
    out = np.zeros(max(1, nreq), np.int32)
    _check(lib().mknn_batch_placement(plan, _ptr(out)))
    return out[:nreq]


def mknn_batch_free(plan: int):
    _check(lib().mknn_batch_free(plan))


def mknn_knn_batch(reqs, stream: int = 0, **opt):
    arr = batch_reqs(reqs)
    o = mknn_batch_opts(**opt)
    _check(lib().mknn_knn_batch(arr, len(reqs), C.addressof(o), stream or None))


def mknn_batch_tune(reqs, sample: int = 1 << 16, stream: int = 0):
    arr = batch_reqs(reqs)
    _check(lib().mknn_batch_tune(arr, len(reqs), sample, stream or None))


def mknn_tune_save(path: str):
    _check(lib().mknn_tune_save(path.encode()))


def mknn_tune_load(path: str):
    _check(lib().mknn_tune_load(path.encode()))


def mknn_tune_clear():
    _check(lib().mknn_tune_clear())


# ---------------------------------------------------------------- serving

def mknn_server_create(slots=0, plain=0, mem_budget=0, max_batch_queries=0, lanes=0) -> int:
    o = mknn_server_opts(slots=slots, plain=plain, mem_budget=mem_budget,
                         max_batch_queries=max_batch_queries, lanes=lanes)
    out = C.c_void_p()
    _check(lib().mknn_server_create(C.addressof(o), C.byref(out)))
    return out.value


def mknn_server_add_cloud(server: int, cloud: int) -> int:
    cid = C.c_int32()
    _check(lib().mknn_server_add_cloud(server, cloud, C.byref(cid)))
    return cid.value


def mknn_server_submit(server: int, cloud_id: int, q, k: int, m: int, out_idx, out_d2) -> int:
    """q, out_idx, out_d2: host arrays (numpy or pinned torch CPU tensors)
    that stay alive until the request is done."""
    nq = int(q.shape[0])
    r = mknn_request(cloud=cloud_id, k=k, m=m, q=_ptr(q), nq=nq, out_idx=_ptr(out_idx),
                     out_d2=_ptr(out_d2))
    t = C.c_uint64()
    _check(lib().mknn_server_submit(server, C.addressof(r), C.byref(t)))
    return t.value


def mknn_server_poll(server: int, ticket: int) -> int:
    s = C.c_int32()
    _check(lib().mknn_server_poll(server, ticket, C.byref(s)))
    return s.value


def mknn_server_drain(server: int, timeout_s: float = 60.0):
    _check(lib().mknn_server_drain(server, timeout_s))


def mknn_server_stats(server: int) -> dict:
    s = mknn_serving_stats()
    _check(lib().mknn_server_stats(server, C.addressof(s)))
    return s.as_dict()


def mknn_server_latencies(server: int, cap: int) -> np.ndarray:
    out = np.zeros(max(1, cap), np.float64)
    n = C.c_int64()
    _check(lib().mknn_server_latencies(server, _ptr(out), cap, C.byref(n)))
    return out[:n.value]


def mknn_server_reset_stats(server: int):
    _check(lib().mknn_server_reset_stats(server))


def mknn_server_destroy(server: int, timeout_s: float = 60.0):
    _check(lib().mknn_server_destroy(server, timeout_s))


def mknn_cloud_check(cloud: int) -> int:
    f = C.c_int32()
    _check(lib().mknn_cloud_check(cloud, C.byref(f)))
    return f.value


# ---------------------------------------------------------------- diagnostics

def mknn_cloud_validate(cloud: int):
    """(tetrahedra not positively oriented, sites strictly inside a circumsphere)."""
    a, b = C.c_int64(), C.c_int64()
    _check(lib().mknn_cloud_validate(cloud, C.byref(a), C.byref(b)))
    return a.value, b.value


def _f3(p):
    return np.ascontiguousarray(p, np.float32).reshape(3)


def mknn_orient3d(a, b, c, d, exact: bool = False) -> int:
    f = lib().mknn_orient3d_exact if exact else lib().mknn_orient3d
    arr = [_f3(x) for x in (a, b, c, d)]
    return int(f(*[_ptr(x) for x in arr]))


def mknn_insphere(a, b, c, d, e, exact: bool = False) -> int:
    f = lib().mknn_insphere_exact if exact else lib().mknn_insphere
    arr = [_f3(x) for x in (a, b, c, d, e)]
    return int(f(*[_ptr(x) for x in arr]))


def mknn_version() -> str:
    return lib().mknn_version().decode()
