"""Independent slow builders used to pin the oracle (pure Python / numpy).

None of this shares code with ``oracle/`` or the CUDA package.  Each builder
reaches the same tree by a different route, all from the paper's definitions:

* ``resort_build`` re-sorts every segment at every level by the level's
  super key (the O(n log^2 n) approach the Introduction contrasts with);
* ``levelwise_build`` processes a whole level at a time with ``np.lexsort``
  and no presorted arrays at all;
* ``superkey`` / ``presort_sorted`` restate the cyclic super key (Section
  2.1) with Python's ``sorted`` as the sorting primitive.
"""
from __future__ import annotations

import itertools

import numpy as np


def superkey(c, t: int, p: int):
    k = len(c[t])
    return tuple(c[t][(p + i) % k] for i in range(k))


def _py(coords: np.ndarray):
    return [tuple(float(v) if isinstance(v, np.floating) else int(v) for v in row) for row in coords]


def presort_sorted(coords: np.ndarray):
    """k lists: indices sorted by super key d (ties by index), then one index
    kept per run of identical tuples (the first, i.e. the smallest)."""
    c = _py(coords)
    n = len(c)
    k = coords.shape[1] if coords.ndim == 2 else 0
    out = []
    for d in range(k):
        order = sorted(range(n), key=lambda t: (superkey(c, t, d), t))
        kept = [next(g)[1] for _, g in itertools.groupby(((c[t], t) for t in order), key=lambda x: x[0])]
        out.append(kept)
    return out


def unique_representatives(coords: np.ndarray):
    c = _py(coords)
    first = {}
    for t, row in enumerate(c):
        first.setdefault(row, t)
    return sorted(first.values())


def resort_build(coords: np.ndarray):
    """Recursive build that sorts each segment by its level's super key."""
    c = _py(coords)
    k = coords.shape[1]
    reps = unique_representatives(coords)
    m = len(reps)
    node = [-2] * m
    left = [-2] * m
    right = [-2] * m
    dim = [255] * m

    def child(lo, hi):
        return -1 if hi < lo else lo + (hi - lo) // 2

    def rec(ids, lo, hi, depth):
        if hi < lo:
            return
        p = depth % k
        ids = sorted(ids, key=lambda t: superkey(c, t, p))
        mid = lo + (hi - lo) // 2
        node[mid] = ids[mid - lo]
        left[mid] = child(lo, mid - 1)
        right[mid] = child(mid + 1, hi)
        dim[mid] = p
        rec(ids[: mid - lo], lo, mid - 1, depth + 1)
        rec(ids[mid - lo + 1:], mid + 1, hi, depth + 1)

    rec(reps, 0, m - 1, 0)
    return {"m": m, "node_tuple": np.array(node, dtype=np.int32),
            "left": np.array(left, dtype=np.int32), "right": np.array(right, dtype=np.int32),
            "dim": np.array(dim, dtype=np.uint8)}


def levelwise_build(coords: np.ndarray):
    """Level-synchronous build with numpy: for every level, order each live
    segment by the level's super key with one lexsort over (segment, key)."""
    coords = np.asarray(coords)
    n, k = coords.shape
    # deduplicate: keep the first index of each distinct row
    if n == 0:
        return {"m": 0, "node_tuple": np.zeros(0, np.int32)}
    cols = [coords[:, j] for j in range(k)]
    # numeric compare: -0.0 and +0.0 must be the same value
    if coords.dtype.kind == "f":
        cols = [np.where(col == 0, np.zeros_like(col), col) for col in cols]
    order = np.lexsort(tuple([np.arange(n)] + cols[::-1]))
    rows = np.stack(cols, axis=1)[order]
    newrun = np.ones(n, dtype=bool)
    newrun[1:] = np.any(rows[1:] != rows[:-1], axis=1)
    reps = np.sort(order[newrun])
    m = len(reps)
    node = np.full(m, -2, dtype=np.int32)
    # segments: (lo, hi, ids)
    segs = [(0, m - 1, reps)]
    depth = 0
    while segs:
        p = depth % k
        nxt = []
        for lo, hi, ids in segs:
            if hi < lo:
                continue
            keys = [cols[(p + i) % k][ids] for i in range(k)]
            srt = ids[np.lexsort(tuple(keys[::-1]))]
            mid = lo + (hi - lo) // 2
            node[mid] = srt[mid - lo]
            nxt.append((lo, mid - 1, srt[: mid - lo]))
            nxt.append((mid + 1, hi, srt[mid - lo + 1:]))
        segs = nxt
        depth += 1
    return {"m": m, "node_tuple": node}


def check_invariants(coords: np.ndarray, tree) -> None:
    """Assert the Section 2.1 properties of an in-order-addressed tree."""
    c = _py(coords)
    k = coords.shape[1]
    m = tree["m"]
    node = [int(v) for v in tree["node_tuple"]]
    assert sorted(node) == unique_representatives(coords)
    levels = 0 if m == 0 else int(np.ceil(np.log2(m + 1)))

    def rec(lo, hi, depth):
        if hi < lo:
            return []
        assert depth < levels
        mid = lo + (hi - lo) // 2
        p = depth % k
        key = superkey(c, node[mid], p)
        ls = rec(lo, mid - 1, depth + 1)
        rs = rec(mid + 1, hi, depth + 1)
        for t in ls:
            assert superkey(c, t, p) < key
        for t in rs:
            assert superkey(c, t, p) > key
        if "dim" in tree:
            assert int(tree["dim"][mid]) == p
        if "left" in tree:
            lc = -1 if mid - 1 < lo else lo + (mid - 1 - lo) // 2
            rc = -1 if hi < mid + 1 else mid + 1 + (hi - mid - 1) // 2
            assert int(tree["left"][mid]) == lc and int(tree["right"][mid]) == rc
        return ls + [node[mid]] + rs

    rec(0, m - 1, 0)
