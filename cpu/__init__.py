"""CPU baselines timed next to the GPU query path: an exact kd-tree with
prefix support and Algorithms 1-2 run query by query on the host
(`mknn_cpu.h`). ctypes marshalling only; the arithmetic is in mknn_cpu.cpp.
Not part of the GPU library, and no code shared with it."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libmknn_cpu.so")
SRC = os.path.join(HERE, "mknn_cpu.cpp")
HDR = os.path.join(HERE, "mknn_cpu.h")

_lib = None


def build() -> str:
    """Compiles libmknn_cpu.so next to this file (portable flags, no
    host-specific instruction set), unless it is newer than its sources."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                                           os.path.getmtime(HDR)):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"
    subprocess.run(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                    "-pthread", SRC, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libmknn_cpu.so is not built (cpu.build())")
        L = ctypes.CDLL(LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.mknn_cpu_kdtree_build.argtypes = [vp, i64, i32, ctypes.POINTER(vp)]
        L.mknn_cpu_kdtree_build.restype = ctypes.c_int
        L.mknn_cpu_kdtree_free.argtypes = [vp]
        L.mknn_cpu_kdtree_free.restype = None
        L.mknn_cpu_kdtree_knn.argtypes = [vp, vp, i64, i32, i32, vp, i32, vp, vp, i32, i32]
        L.mknn_cpu_kdtree_knn.restype = ctypes.c_int
        L.mknn_cpu_dpknn.argtypes = [vp, i64, vp, vp, vp, i64, i32, i32, vp, i32, vp, vp, vp, i32,
                                     i32]
        L.mknn_cpu_dpknn.restype = ctypes.c_int
        L.mknn_cpu_threads.argtypes = []
        L.mknn_cpu_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _m_args(m, nq):
    if m is None or np.ndim(m) == 0:
        return None, int(m or 0)
    arr = np.ascontiguousarray(m, dtype=np.int32).reshape(nq)
    return arr, 0


def threads() -> int:
    return int(lib().mknn_cpu_threads())


class KDTree:
    """Exact kd-tree over points in rank order (row r = rank r)."""

    def __init__(self, xyz_ranked, leaf: int = 8):
        P = np.ascontiguousarray(xyz_ranked, dtype=np.float32)
        h = ctypes.c_void_p()
        rc = lib().mknn_cpu_kdtree_build(_ptr(P), P.shape[0], leaf, ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"mknn_cpu_kdtree_build failed ({rc})")
        self.h = h
        self.n = P.shape[0]

    def knn(self, Q, k: int, m=None, threads: int = 0, sort: bool = True):
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        nq = Q.shape[0]
        marr, ms = _m_args(m, nq)
        oi = np.empty((nq, k), np.int32)
        od = np.empty((nq, k), np.float32)
        rc = lib().mknn_cpu_kdtree_knn(self.h, _ptr(Q), nq, Q.shape[1], k, _ptr(marr), ms,
                                        _ptr(oi), _ptr(od), int(sort), threads)
        if rc == -1:
            raise ValueError("mknn_cpu_kdtree_knn: invalid arguments")
        return oi, od

    def close(self):
        if self.h:
            lib().mknn_cpu_kdtree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dpknn(xyz_ranked, rowp, succ, Q, k: int, m=None, threads: int = 0, counters: bool = False,
          sort: bool = True):
    """Algorithms 1-2 on the host over a CSR successor table. Returns
    (idx, d2) or (idx, d2, counters int64 (nq, 8))."""
    P = np.ascontiguousarray(xyz_ranked, dtype=np.float32)
    rp = np.ascontiguousarray(rowp, dtype=np.int64)
    sc = np.ascontiguousarray(succ, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    nq = Q.shape[0]
    marr, ms = _m_args(m, nq)
    oi = np.empty((nq, k), np.int32)
    od = np.empty((nq, k), np.float32)
    cnt = np.zeros((nq, 8), np.int64) if counters else None
    rc = lib().mknn_cpu_dpknn(_ptr(P), P.shape[0], _ptr(rp), _ptr(sc), _ptr(Q), nq, Q.shape[1], k,
                              _ptr(marr), ms, _ptr(oi), _ptr(od), _ptr(cnt), int(sort), threads)
    if rc == -1:
        raise ValueError("mknn_cpu_dpknn: invalid arguments")
    return (oi, od, cnt) if counters else (oi, od)
