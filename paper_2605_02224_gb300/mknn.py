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
MKNN_MAX_K = 64


class MknnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mknn_build_opts(C.Structure):
    _fields_ = [("keep_tets", C.c_int32), ("reserved", C.c_int32 * 7)]


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
                ("reserved", C.c_int32 * 4)]


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
        "mknn_cloud_table": (i32, [vp, vp, vp, vp]),
        "mknn_cloud_stats": (i32, [vp, vp]),
        "mknn_cloud_tets": (i32, [vp, vp, vp]),
        "mknn_cloud_save": (i32, [vp, C.c_char_p]),
        "mknn_cloud_load": (i32, [C.c_char_p, pp]),
        "mknn_knn": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_knn_workspace_size": (sz, [i64, vp]),
        "mknn_knn_ex": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp, vp]),
        "mknn_knn_host": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_cloud_check": (i32, [vp, vp]),
        "mknn_query_order_workspace_size": (sz, [i64]),
        "mknn_query_order": (i32, [vp, vp, i64, i32, vp, vp, sz, vp]),
        "mknn_cloud_validate": (i32, [vp, vp, vp]),
        "mknn_knn_noalloc": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
        "mknn_knn_noalloc_max_queries": (i64, []),
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

def mknn_build(xyz, order=None, keep_tets: bool = False) -> int:
    """Builds the successor table on the host; returns the cloud handle."""
    x = _host(xyz, np.float32).reshape(-1, 3)
    o = None if order is None else _host(order, np.int64)
    opts = mknn_build_opts(keep_tets=1 if keep_tets else 0)
    out = C.c_void_p()
    _check(lib().mknn_build(_ptr(x), x.shape[0], _ptr(o), C.addressof(opts), C.byref(out)))
    return out.value


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
          order=None):
    return mknn_knn_opts(lanes=lanes, sort=sort, blocks_per_sm=blocks_per_sm,
                         counters=_ptr(counters), workspace=_ptr(workspace),
                         workspace_bytes=workspace_bytes, order=_ptr(order))


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
