"""CPU oracle for the presorting k-d tree build (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
product path (``paper_1410_5420_gb300``) never does.

The arithmetic lives in ``kd_oracle.c`` (plain single-threaded C written
from Section 2.1 of the paper); this module compiles it with gcc into
``oracle/_build/`` and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kd_oracle.c")
_SRC_SEARCH = os.path.join(_HERE, "kd_search_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkd_oracle.so")

DTYPES = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.float32): 2}
ENAN = -6


def build(force: bool = False, mutant: int = 0, out: str | None = None) -> str:
    """Compile the oracle shared library (gcc, -O2, no vendor code).
    ``mutant`` > 0 plants one of the deliberate mistakes listed in
    kd_oracle.c (only the mutation tests do this)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = out or (_LIB if mutant == 0 else os.path.join(_BUILD, f"libkd_oracle_mutant{mutant}.so"))
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_SEARCH))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".tmp{os.getpid()}"
        # -ffp-contract=off: every floating-point operation of the search
        # distances is rounded separately, as their definition states
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", f"-DKDO_MUTANT={int(mutant)}",
                               "-shared", "-fPIC", "-pthread", _SRC, _SRC_SEARCH, "-o", tmp])
        os.replace(tmp, lib)
    return lib


_libs: dict = {}


def _load(mutant: int = 0):
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant=mutant))
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.kdo_presort.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, i64p]
        lib.kdo_build.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  vp, vp, vp, vp, i64p, vp]
        lib.kdo_first_split.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, i64p,
                                        ctypes.POINTER(ctypes.c_int32)]
        for f in (lib.kdo_presort, lib.kdo_build, lib.kdo_first_split):
            f.restype = ctypes.c_int
        lib.kdo_build_parallel.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                           vp, vp, i64p]
        lib.kdo_build_parallel.restype = ctypes.c_int
        lib.kdo_knn.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, vp,
                                ctypes.c_int64, ctypes.c_int, vp, vp]
        lib.kdo_knn.restype = ctypes.c_int
        lib.kdo_region.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, vp, vp,
                                   ctypes.c_int64, vp, vp, ctypes.c_int64]
        lib.kdo_region.restype = ctypes.c_int64
        _libs[mutant] = lib
    return _libs[mutant]


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle returned status {code}")
        self.code = code


def _prep(coords: np.ndarray):
    c = np.ascontiguousarray(coords)
    if c.ndim != 2:
        raise ValueError("coords must be n x k")
    if c.dtype not in DTYPES:
        raise ValueError(f"unsupported dtype {c.dtype}")
    return c, c.shape[0], c.shape[1], DTYPES[c.dtype]


def presort(coords: np.ndarray, mutant: int = 0) -> np.ndarray:
    """k x m array: row d is the deduplicated index array sorted by super key d."""
    c, n, k, dt = _prep(coords)
    out = np.empty((k, max(n, 1)), dtype=np.int32)
    m = ctypes.c_int64(0)
    rc = _load(mutant).kdo_presort(c.ctypes.data, n, k, dt, out.ctypes.data, ctypes.byref(m))
    if rc != 0:
        raise OracleError(rc)
    return out[:, : m.value].copy()


def build_tree(coords: np.ndarray, terminate_small: bool = True, mutant: int = 0):
    """Returns dict(m, node_tuple, left, right, dim, arrays) for the tree."""
    c, n, k, dt = _prep(coords)
    cap = max(n, 1)
    node = np.full(cap, -2, dtype=np.int32)
    left = np.full(cap, -2, dtype=np.int32)
    right = np.full(cap, -2, dtype=np.int32)
    dim = np.full(cap, 255, dtype=np.uint8)
    arrays = np.empty((k, cap), dtype=np.int32)
    m = ctypes.c_int64(0)
    rc = _load(mutant).kdo_build(c.ctypes.data, n, k, dt, 1 if terminate_small else 0,
                           node.ctypes.data, left.ctypes.data, right.ctypes.data,
                           dim.ctypes.data, ctypes.byref(m), arrays.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    mm = m.value
    return {"m": mm, "root": (mm - 1) // 2 if mm > 0 else -1,
            "node_tuple": node[:mm].copy(), "left": left[:mm].copy(),
            "right": right[:mm].copy(), "dim": dim[:mm].copy(),
            "arrays": arrays[:, :mm].copy()}


def first_split(coords: np.ndarray, mutant: int = 0):
    """(arrays k x m after the first split in dimension order, median tuple)."""
    c, n, k, dt = _prep(coords)
    out = np.empty((k, max(n, 1)), dtype=np.int32)
    m = ctypes.c_int64(0)
    med = ctypes.c_int32(-1)
    rc = _load(mutant).kdo_first_split(c.ctypes.data, n, k, dt, out.ctypes.data, ctypes.byref(m),
                                 ctypes.byref(med))
    if rc != 0:
        raise OracleError(rc)
    return out[:, : m.value].copy(), med.value


def knn(coords: np.ndarray, queries: np.ndarray, kn: int, cand: np.ndarray | None = None):
    """m nearest neighbours (squared Euclidean, ties by smaller index) of each
    query among the distinct tuples (``cand``, default: the presort's
    survivors).  Returns (idx nq x kn int32, dist2 nq x kn float64)."""
    c, n, k, dt = _prep(coords)
    q = np.ascontiguousarray(queries, dtype=c.dtype)
    if q.ndim != 2 or q.shape[1] != k:
        raise ValueError("queries must be nq x k")
    if cand is None:
        cand = presort(c)[0] if n else np.empty(0, np.int32)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    nq = q.shape[0]
    idx = np.empty((max(nq, 1), kn), dtype=np.int32)
    d2 = np.empty((max(nq, 1), kn), dtype=np.float64)
    rc = _load().kdo_knn(c.ctypes.data, n, k, dt, cand.ctypes.data, cand.size, q.ctypes.data, nq, kn,
                         idx.ctypes.data, d2.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return idx[:nq], d2[:nq]


def region(coords: np.ndarray, lo: np.ndarray, hi: np.ndarray, cand: np.ndarray | None = None) -> list:
    """For each box [lo[i], hi[i]] the sorted indices of the distinct tuples inside it."""
    c, n, k, dt = _prep(coords)
    lo = np.ascontiguousarray(lo, dtype=c.dtype)
    hi = np.ascontiguousarray(hi, dtype=c.dtype)
    if cand is None:
        cand = presort(c)[0] if n else np.empty(0, np.int32)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    nq = lo.shape[0]
    counts = np.empty(max(nq, 1), dtype=np.int64)
    cap = max(1, nq * max(cand.size, 1))
    out = np.empty(cap, dtype=np.int32)
    tot = _load().kdo_region(c.ctypes.data, n, k, dt, cand.ctypes.data, cand.size, lo.ctypes.data, hi.ctypes.data,
                             nq, counts.ctypes.data, out.ctypes.data, cap)
    if tot < 0:
        raise OracleError(int(tot))
    res, o = [], 0
    for i in range(nq):
        res.append(np.sort(out[o:o + counts[i]]))
        o += counts[i]
    return res


def build_tree_parallel(coords: np.ndarray, levels: int):
    """The paper's parallel scheme on 2^levels host threads (a CPU baseline;
    the same tree as build_tree).  Returns dict(m, node_tuple, left, right, dim)."""
    c, n, k, dt = _prep(coords)
    cap = max(n, 1)
    node = np.full(cap, -2, dtype=np.int32)
    left = np.full(cap, -2, dtype=np.int32)
    right = np.full(cap, -2, dtype=np.int32)
    dim = np.full(cap, 255, dtype=np.uint8)
    m = ctypes.c_int64(0)
    rc = _load().kdo_build_parallel(c.ctypes.data, n, k, dt, levels, node.ctypes.data, left.ctypes.data,
                                    right.ctypes.data, dim.ctypes.data, ctypes.byref(m))
    if rc != 0:
        raise OracleError(rc)
    mm = m.value
    return {"m": mm, "node_tuple": node[:mm].copy(), "left": left[:mm].copy(), "right": right[:mm].copy(),
            "dim": dim[:mm].copy()}
