"""Python binding of the C ABI (include/kdtree.h), same names as the C calls.

Only argument marshalling happens here: tensors and arrays become pointers
and sizes, outputs are allocated, status codes become exceptions.  Every
step of the presort and build runs in the library's CUDA kernels.
Device tensors (torch, CUDA) are passed as device pointers; numpy arrays and
CPU tensors as host pointers.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import KdCloud, KdConfig, KdTree

try:
    import torch
except Exception:  # pragma: no cover - torch is present on every target
    torch = None


class KdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_NP_DT = {np.dtype(np.int32): _lib.KD_I32, np.dtype(np.int64): _lib.KD_I64, np.dtype(np.float32): _lib.KD_F32}


def _torch_dt():
    return {torch.int32: _lib.KD_I32, torch.int64: _lib.KD_I64, torch.float32: _lib.KD_F32}


class Context:
    """A kd_ctx: device, stream, memory pool."""

    def __init__(self, ptr: int, device: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.device = device

    def check(self, rc: int):
        if rc != _lib.KD_OK:
            msg = _lib.load().kd_last_error(self.ptr)
            raise KdError(rc, msg.decode() if msg else "")

    def close(self):
        if self.ptr:
            _lib.load().kd_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Handle:
    ptr: ctypes.c_void_p
    n: int
    m: int
    k: int
    on_device: bool


def kd_create(device: int = 0, stream=None, mem_budget_bytes: int = 0, switch_threshold: int = 0,
              debug: int = 0, level_tile: int = 0, tune_cache: str | None = None,
              schedule: int = 0) -> Context:
    """kd_create.  ``stream``: a torch.cuda.Stream, an int handle, or None for
    torch's current stream on ``device``.  ``switch_threshold`` / ``level_tile``:
    0 for the tuned (or default) values; ``tune_cache``: the autotuner's file;
    ``schedule``: the level schedule (KD_SCHEDULE_MULTI / _DEFERRED / _EVERY_LEVEL)."""
    lib = _lib.load()
    if stream is None and torch is not None and torch.cuda.is_available():
        stream = torch.cuda.current_stream(device)
    sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    cfg = KdConfig(device, ctypes.c_void_p(sh), mem_budget_bytes, level_tile, switch_threshold, debug,
                   tune_cache.encode() if tune_cache else None, schedule)
    out = ctypes.c_void_p()
    rc = lib.kd_create(ctypes.byref(out), ctypes.byref(cfg))
    if rc != _lib.KD_OK:
        raise KdError(rc, "kd_create failed")
    return Context(out.value, device)


def _cloud(coords) -> tuple[KdCloud, object]:
    """KdCloud for a torch tensor or numpy array; returns (struct, keep-alive)."""
    if torch is not None and isinstance(coords, torch.Tensor):
        t = coords.contiguous()
        if t.dim() != 2 or t.dtype not in _torch_dt():
            raise ValueError("coords must be an n x k int32/int64/float32 tensor")
        return KdCloud(t.data_ptr(), t.shape[0], t.shape[1], _torch_dt()[t.dtype], int(t.is_cuda)), t
    a = np.ascontiguousarray(coords)
    if a.ndim != 2 or a.dtype not in _NP_DT:
        raise ValueError("coords must be an n x k int32/int64/float32 array")
    return KdCloud(a.ctypes.data, a.shape[0], a.shape[1], _NP_DT[a.dtype], 0), a


def kd_presort(ctx: Context, coords) -> Handle:
    """kd_presort: presort + dedup; the handle owns the device arrays."""
    c, keep = _cloud(coords)
    h = ctypes.c_void_p()
    ctx.check(_lib.load().kd_presort(ctx.ptr, ctypes.byref(c), ctypes.byref(h)))
    del keep
    n, m, k = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int()
    ctx.check(_lib.load().kd_handle_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(k)))
    return Handle(h, n.value, m.value, k.value, bool(c.on_device))


def kd_handle_arrays(ctx: Context, h: Handle) -> np.ndarray:
    """The k presorted deduplicated index arrays (k x m, host)."""
    out = np.empty((h.k, max(h.m, 1)), dtype=np.int32)
    ctx.check(_lib.load().kd_handle_arrays(ctx.ptr, h.ptr, ctypes.c_void_p(out.ctypes.data), 0))
    return out[:, : h.m]


def _alloc_tree(n: int, on_device: bool, device: int, children: bool):
    cap = max(n, 1)
    if on_device:
        dev = torch.device("cuda", device)
        node = torch.empty(cap, dtype=torch.int32, device=dev)
        left = torch.empty(cap, dtype=torch.int32, device=dev) if children else None
        right = torch.empty(cap, dtype=torch.int32, device=dev) if children else None
        dim = torch.empty(cap, dtype=torch.uint8, device=dev) if children else None
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    else:
        node = np.empty(cap, dtype=np.int32)
        left = np.empty(cap, dtype=np.int32) if children else None
        right = np.empty(cap, dtype=np.int32) if children else None
        dim = np.empty(cap, dtype=np.uint8) if children else None
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    tree = KdTree(0, -1, ptr(node), ptr(left), ptr(right), ptr(dim), int(on_device))
    return tree, {"node_tuple": node, "left": left, "right": right, "dim": dim}


def _result(tree: KdTree, arrays: dict) -> dict:
    m = tree.m
    out = {"m": m, "root": tree.root}
    for key, a in arrays.items():
        if a is not None:
            out[key] = a[:m]
    return out


def kd_build(ctx: Context, h: Handle, children: bool = True, on_device: bool | None = None) -> dict:
    """kd_build: consumes the handle.  Outputs live on the device if the
    input did (unless ``on_device`` says otherwise)."""
    dev = h.on_device if on_device is None else on_device
    tree, arrays = _alloc_tree(h.n, dev, ctx.device, children)
    ctx.check(_lib.load().kd_build(ctx.ptr, h.ptr, ctypes.byref(tree)))
    h.ptr = ctypes.c_void_p(0)
    return _result(tree, arrays)


def kd_release(ctx: Context, h: Handle) -> None:
    if h.ptr:
        ctx.check(_lib.load().kd_release(ctx.ptr, h.ptr))
        h.ptr = ctypes.c_void_p(0)


def build_tree(ctx: Context, coords, children: bool = True, on_device: bool | None = None) -> dict:
    """kd_presort followed by kd_build."""
    return kd_build(ctx, kd_presort(ctx, coords), children=children, on_device=on_device)


def kd_build_select(ctx: Context, coords, children: bool = True, on_device: bool | None = None) -> dict:
    """kd_build_select: the O(n log n) build with per-level median selection
    (one presorted index array); the same tree as build_tree."""
    c, keep = _cloud(coords)
    dev = bool(c.on_device) if on_device is None else on_device
    tree, arrays = _alloc_tree(c.n, dev, ctx.device, children)
    ctx.check(_lib.load().kd_build_select(ctx.ptr, ctypes.byref(c), ctypes.byref(tree)))
    del keep
    return _result(tree, arrays)


def _np_struct(ctype) -> np.dtype:
    """numpy dtype with the layout of a ctypes Structure of scalar fields."""
    names, formats, offsets = [], [], []
    conv = {ctypes.c_int: np.int32, ctypes.c_int32: np.int32, ctypes.c_int64: np.int64,
            ctypes.c_void_p: np.uint64, ctypes.c_size_t: np.uint64}
    for name, t in ctype._fields_:
        names.append(name)
        formats.append(conv[t])
        offsets.append(getattr(ctype, name).offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": ctypes.sizeof(ctype)})


class BatchTrees:
    """The trees of a batch: one output buffer per field for all clouds,
    cloud i at offs[i] .. offs[i] + n_i; ``trees[i]`` is cloud i's dict
    (views of the shared buffers)."""

    def __init__(self, m, root, offs, arrays):
        self.m, self.root, self.offs, self.arrays = m, root, offs, arrays

    def __len__(self):
        return len(self.m)

    def __getitem__(self, i):
        o, mi = int(self.offs[i]), int(self.m[i])
        out = {"m": mi, "root": int(self.root[i])}
        for key, a in self.arrays.items():
            if a is not None:
                out[key] = a[o:o + mi]
        return out

    def __iter__(self):
        return (self[i] for i in range(len(self)))


def kd_build_batch(ctx: Context, clouds: list, children: bool = True, on_device: bool | None = None) -> BatchTrees:
    """kd_build_batch over a list of clouds (same k and dtype).  Outputs
    live in one buffer per field (device when the first cloud is a CUDA
    tensor, unless ``on_device`` says otherwise)."""
    count = len(clouds)
    cdt = _np_struct(KdCloud)
    rows, keep = [], []
    tdts = _torch_dt() if torch is not None else {}
    for c in clouds:
        if torch is not None and isinstance(c, torch.Tensor) and c.dim() == 2 and c.is_contiguous() \
                and c.dtype in tdts:
            rows.append((c.data_ptr(), c.shape[0], c.shape[1], tdts[c.dtype], int(c.is_cuda)))
        else:
            s, kk = _cloud(c)
            keep.append(kk)
            rows.append((s.coords or 0, s.n, s.k, s.dtype, s.on_device))
    ca = np.array(rows, dtype=cdt) if rows else np.zeros(0, dtype=cdt)
    ns = ca["n"].astype(np.int64)
    offs = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(ns, out=offs[1:])
    dev = bool(ca["on_device"][0]) if on_device is None else on_device
    trees = _batch_call(ctx, ca, offs, dev, children)
    del keep
    return trees


def kd_build_batch_packed(ctx: Context, coords, sizes, children: bool = True,
                          on_device: bool | None = None) -> BatchTrees:
    """kd_build_batch over clouds stored back to back in one row-major
    (sum(sizes), k) array or tensor: cloud i is rows [sum(sizes[:i]),
    sum(sizes[:i+1])).  The descriptors come from the sizes in one vector
    step, where kd_build_batch inspects every cloud object."""
    if torch is not None and isinstance(coords, torch.Tensor):
        if coords.dim() != 2 or not coords.is_contiguous() or coords.dtype not in _torch_dt():
            raise ValueError("coords must be a contiguous (n, k) int32/int64/float32 tensor")
        base, k, dt, ondev, esz = coords.data_ptr(), coords.shape[1], _torch_dt()[coords.dtype], \
            int(coords.is_cuda), coords.element_size()
        keep = coords
    else:
        s, keep = _cloud(coords)
        base, k, dt, ondev = s.coords or 0, s.k, s.dtype, s.on_device
        esz = 8 if dt == _lib.KD_I64 else 4
    ns = np.asarray(sizes, dtype=np.int64)
    count = len(ns)
    offs = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(ns, out=offs[1:])
    ca = np.zeros(count, dtype=_np_struct(KdCloud))
    ca["coords"] = np.uint64(base) + offs[:-1].astype(np.uint64) * np.uint64(k * esz)
    ca["n"] = ns
    ca["k"] = k
    ca["dtype"] = dt
    ca["on_device"] = ondev
    dev = bool(ondev) if on_device is None else on_device
    trees = _batch_call(ctx, ca, offs, dev, children)
    del keep
    return trees


def _batch_call(ctx: Context, ca, offs, dev: bool, children: bool) -> BatchTrees:
    count = len(ca)
    tdt = _np_struct(KdTree)
    tree, arrays = _alloc_tree(int(offs[-1]), dev, ctx.device, children)
    ta = np.zeros(count, dtype=tdt)
    ta["root"] = -1
    for name, size in (("node_tuple", 4), ("left", 4), ("right", 4), ("dim", 1)):
        base = getattr(tree, name)
        if base:
            ta[name] = np.uint64(base) + offs[:-1].astype(np.uint64) * np.uint64(size)
    ta["on_device"] = int(dev)
    ctx.check(_lib.load().kd_build_batch(ctx.ptr, ctypes.c_void_p(ca.ctypes.data), count,
                                         ctypes.c_void_p(ta.ctypes.data)))
    return BatchTrees(ta["m"].copy(), ta["root"].copy(), offs, arrays)


class Ticket:
    def __init__(self, value: int, tree: KdTree, arrays: dict, keep):
        self.value = value
        self.tree = tree
        self.arrays = arrays
        self.keep = keep


def kd_submit(ctx: Context, coords, children: bool = True) -> Ticket:
    """kd_submit: enqueue a serving request (host outputs)."""
    c, keep = _cloud(coords)
    tree, arrays = _alloc_tree(c.n, False, ctx.device, children)
    t = ctypes.c_int64()
    ctx.check(_lib.load().kd_submit(ctx.ptr, ctypes.byref(c), ctypes.byref(tree), ctypes.byref(t)))
    return Ticket(t.value, tree, arrays, keep)


def kd_wait(ctx: Context, ticket: Ticket, timeout_ms: int = -1) -> dict:
    ctx.check(_lib.load().kd_wait(ctx.ptr, ticket.value, timeout_ms))
    return _result(ticket.tree, ticket.arrays)


def kd_serving_stats(ctx: Context) -> dict:
    n = ctypes.c_int64()
    p50, p99 = ctypes.c_double(), ctypes.c_double()
    ctx.check(_lib.load().kd_serving_stats(ctx.ptr, ctypes.byref(n), ctypes.byref(p50), ctypes.byref(p99)))
    return {"completed": n.value, "p50_us": p50.value, "p99_us": p99.value}


def _check_out_buffer(name: str, t, dev, need: int) -> None:
    """An output the library writes through a raw pointer: a contiguous
    int32 tensor on ``dev`` holding at least ``need`` elements."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or not t.is_contiguous() \
            or t.device != dev or t.numel() < need:
        raise ValueError(f"{name} must be a contiguous int32 tensor on {dev} with at least {need} elements")


def kd_presort_noalloc(ctx: Context, coords, arrays_out=None, m_out=None):
    """kd_presort_noalloc: presort + duplicate removal of one small cloud
    (device tensor, n <= KD_NOALLOC_MAX_N) into caller-owned device buffers;
    the library allocates nothing.  ``arrays_out`` (k x n int32) and
    ``m_out`` (1 int32) are made here when not given.  Asynchronous on the
    context's stream: read ``m_out`` (m, or KD_ENAN) after the stream.
    Returns (arrays_out, m_out)."""
    c, keep = _cloud(coords)
    dev = torch.device("cuda", ctx.device)
    if arrays_out is None:
        arrays_out = torch.empty((c.k, max(c.n, 1)), dtype=torch.int32, device=dev)
    if m_out is None:
        m_out = torch.empty(1, dtype=torch.int32, device=dev)
    # the library writes through raw pointers: k rows of n int32 at stride n
    # and one int32, on the context's device
    _check_out_buffer("arrays_out", arrays_out, dev, c.k * c.n)
    _check_out_buffer("m_out", m_out, dev, 1)
    ctx.check(_lib.load().kd_presort_noalloc(ctx.ptr, ctypes.byref(c), ctypes.c_void_p(arrays_out.data_ptr()),
                                             ctypes.c_void_p(m_out.data_ptr())))
    del keep
    return arrays_out, m_out


class Index:
    """A kd_index: the tree's tuples in address order on the device."""

    def __init__(self, ptr: int, k: int, dtype):
        self.ptr = ctypes.c_void_p(ptr)
        self.k = k
        self.dtype = dtype


def kd_index_create(ctx: Context, coords, tree: dict) -> Index:
    """kd_index_create for a tree (as returned by kd_build / build_tree)
    built from ``coords``."""
    c, keep = _cloud(coords)
    nt = tree["node_tuple"]
    on_dev = bool(torch is not None and isinstance(nt, torch.Tensor) and nt.is_cuda)
    if on_dev:
        nt = nt.contiguous()
        ptr = nt.data_ptr()
    else:
        nt = np.ascontiguousarray(nt if not hasattr(nt, "numpy") else nt.numpy(), dtype=np.int32)
        ptr = nt.ctypes.data
    t = KdTree(int(tree["m"]), -1, ctypes.c_void_p(ptr), None, None, None, int(on_dev))
    out = ctypes.c_void_p()
    ctx.check(_lib.load().kd_index_create(ctx.ptr, ctypes.byref(c), ctypes.byref(t), ctypes.byref(out)))
    del keep, nt
    dt = coords.dtype if hasattr(coords, "dtype") else None
    return Index(out.value, c.k, dt)


def kd_index_destroy(ctx: Context, index: Index) -> None:
    if index.ptr:
        ctx.check(_lib.load().kd_index_destroy(ctx.ptr, index.ptr))
        index.ptr = ctypes.c_void_p(0)


def _rows(x, k):
    """(pointer, keep-alive, on_device, n) of an n x k query array."""
    if torch is not None and isinstance(x, torch.Tensor):
        t = x.contiguous()
        if t.dim() != 2 or t.shape[1] != k:
            raise ValueError("queries must be n x k")
        return t.data_ptr(), t, bool(t.is_cuda), t.shape[0]
    a = np.ascontiguousarray(x)
    if a.ndim != 2 or a.shape[1] != k:
        raise ValueError("queries must be n x k")
    return a.ctypes.data, a, False, a.shape[0]


def kd_knn(ctx: Context, index: Index, queries, kn: int, with_dist: bool = True):
    """kd_knn: (idx nq x kn int32, dist2 nq x kn float64 or None); device
    tensors when the queries are a CUDA tensor, numpy arrays otherwise."""
    qp, keep, dev, nq = _rows(queries, index.k)
    if dev:
        idx = torch.empty((nq, kn), dtype=torch.int32, device=queries.device)
        d2 = torch.empty((nq, kn), dtype=torch.float64, device=queries.device) if with_dist else None
        ip, dp = idx.data_ptr(), (d2.data_ptr() if with_dist else None)
    else:
        idx = np.empty((nq, kn), dtype=np.int32)
        d2 = np.empty((nq, kn), dtype=np.float64) if with_dist else None
        ip, dp = idx.ctypes.data, (d2.ctypes.data if with_dist else None)
    ctx.check(_lib.load().kd_knn(ctx.ptr, index.ptr, ctypes.c_void_p(qp), nq, kn, int(dev), ctypes.c_void_p(ip),
                                 ctypes.c_void_p(dp) if dp else None))
    del keep
    return idx, d2


def kd_knn_all(ctx: Context, index: Index, m: int, kn: int, on_device: bool = True, with_dist: bool = True):
    """kd_knn_all: (idx m x kn, dist2 m x kn or None), row a for the tuple at
    tree address a; ``m`` is the tree's tuple count."""
    if on_device:
        idx = torch.empty((m, kn), dtype=torch.int32, device="cuda")
        d2 = torch.empty((m, kn), dtype=torch.float64, device="cuda") if with_dist else None
        ip, dp = idx.data_ptr(), (d2.data_ptr() if with_dist else None)
    else:
        idx = np.empty((m, kn), dtype=np.int32)
        d2 = np.empty((m, kn), dtype=np.float64) if with_dist else None
        ip, dp = idx.ctypes.data, (d2.ctypes.data if with_dist else None)
    ctx.check(_lib.load().kd_knn_all(ctx.ptr, index.ptr, kn, int(on_device), ctypes.c_void_p(ip),
                                     ctypes.c_void_p(dp) if dp else None))
    return idx, d2


def kd_reverse_knn(ctx: Context, index: Index, m: int, kn: int, on_device: bool = True):
    """kd_reverse_knn: (offsets m+1 int64, rev int32) with the reverse
    neighbours of the tuple at address a in rev[offsets[a]:offsets[a+1]]."""
    if on_device:
        offs = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        rev = torch.empty(max(m * kn, 1), dtype=torch.int32, device="cuda")
        op, rp = offs.data_ptr(), rev.data_ptr()
    else:
        offs = np.empty(m + 1, dtype=np.int64)
        rev = np.empty(max(m * kn, 1), dtype=np.int32)
        op, rp = offs.ctypes.data, rev.ctypes.data
    ctx.check(_lib.load().kd_reverse_knn(ctx.ptr, index.ptr, kn, int(on_device), ctypes.c_void_p(op),
                                         ctypes.c_void_p(rp)))
    return offs, rev


def kd_region(ctx: Context, index: Index, lo, hi):
    """kd_region: (offsets nq+1 int64, idx int32) with box i's tuples at
    idx[offsets[i]:offsets[i+1]]; device tensors for CUDA boxes."""
    lp, keep_lo, dev, nq = _rows(lo, index.k)
    hp, keep_hi, dev2, nq2 = _rows(hi, index.k)
    if dev != dev2 or nq != nq2:
        raise ValueError("lo and hi must match")
    lib = _lib.load()
    if dev:
        offs = torch.empty(nq + 1, dtype=torch.int64, device=lo.device)
        op = offs.data_ptr()
    else:
        offs = np.empty(nq + 1, dtype=np.int64)
        op = offs.ctypes.data
    ctx.check(lib.kd_region(ctx.ptr, index.ptr, ctypes.c_void_p(lp), ctypes.c_void_p(hp), nq, int(dev),
                            ctypes.c_void_p(op), None, 0))
    total = int(offs[-1].item() if dev else offs[-1])
    if dev:
        idx = torch.empty(max(total, 1), dtype=torch.int32, device=lo.device)
        ipt = idx.data_ptr()
    else:
        idx = np.empty(max(total, 1), dtype=np.int32)
        ipt = idx.ctypes.data
    if total:
        ctx.check(lib.kd_region(ctx.ptr, index.ptr, ctypes.c_void_p(lp), ctypes.c_void_p(hp), nq, int(dev),
                                ctypes.c_void_p(op), ctypes.c_void_p(ipt), total))
    del keep_lo, keep_hi
    return offs, idx[:total]


_DT_CODES = {"int32": _lib.KD_I32, "int64": _lib.KD_I64, "float32": _lib.KD_F32}


def _dtype_code(dtype) -> int:
    if isinstance(dtype, int):
        return dtype
    return _DT_CODES[str(np.dtype(str(dtype).replace("torch.", "")))]


def kd_autotune(ctx: Context, k: int, dtype, n: int, reps: int = 3) -> dict:
    """kd_autotune: time every (on-chip subtree size, level tile) pair on a
    synthetic cloud of n tuples; returns the chosen pair."""
    sm, lt = ctypes.c_int(), ctypes.c_int()
    ctx.check(_lib.load().kd_autotune(ctx.ptr, k, _dtype_code(dtype), n, reps, ctypes.byref(sm), ctypes.byref(lt)))
    return {"switch_threshold": sm.value, "level_tile": lt.value}


def kd_tuning_get(ctx: Context, k: int, dtype, n: int) -> dict:
    """kd_tuning_get: the pair a build of clouds of at most n tuples uses."""
    sm, lt = ctypes.c_int(), ctypes.c_int()
    ctx.check(_lib.load().kd_tuning_get(ctx.ptr, k, _dtype_code(dtype), n, ctypes.byref(sm), ctypes.byref(lt)))
    return {"switch_threshold": sm.value, "level_tile": lt.value}


def kd_launch_count(ctx: Context) -> int:
    return int(_lib.load().kd_launch_count(ctx.ptr))


def kd_kernel_stats(ctx: Context) -> dict:
    """Per kernel family: device ms, launches, elements processed and
    algorithmic bytes moved (collected when the context was created with
    debug & 2)."""
    out = {}
    for f, name in enumerate(_lib.FAMILIES):
        ms, n, u, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        ctx.check(_lib.load().kd_kernel_stats(ctx.ptr, f, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(u),
                                              ctypes.byref(b)))
        out[name] = {"ms": ms.value, "launches": n.value, "units": u.value, "bytes": b.value}
    return out


def kd_trace_counters(ctx: Context) -> list:
    """Finisher phase block-time sums in ns (context created with debug & 4)."""
    out = (ctypes.c_double * 8)()
    ctx.check(_lib.load().kd_trace_counters(ctx.ptr, out, 8))
    return list(out)


def kd_kernel_stats_reset(ctx: Context) -> None:
    ctx.check(_lib.load().kd_kernel_stats_reset(ctx.ptr))


def kd_destroy(ctx: Context) -> None:
    ctx.close()
