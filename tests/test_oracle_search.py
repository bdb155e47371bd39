"""Pins of the search oracle (CPU): m nearest neighbours and region search
by brute force, checked against an independent numpy restatement of the
same definitions, special cases and invariants."""
import numpy as np
import pytest

import kdgen
import oracle


def numpy_dist2(coords, q):
    """Squared distances of every row to one query, each operation rounded
    separately in dimension order (integers: exact |a - b| as uint64)."""
    acc = np.zeros(coords.shape[0], dtype=np.float64)
    for d in range(coords.shape[1]):
        if coords.dtype.kind == "f":
            u = np.abs(coords[:, d].astype(np.float64) - np.float64(q[d]))
        else:
            a = coords[:, d].astype(np.int64)
            b = np.int64(q[d])
            u = np.where(a > b, (a.astype(np.uint64) - np.uint64(b)), (np.uint64(b) - a.astype(np.uint64)))
            u = u.astype(np.float64)
        acc = acc + u * u
    return acc


def numpy_knn(coords, cand, queries, kn):
    idx = np.full((len(queries), kn), -1, np.int32)
    dist = np.full((len(queries), kn), np.inf)
    for i, q in enumerate(queries):
        d = numpy_dist2(coords[cand], q)
        order = np.lexsort((cand, d))[:kn]
        idx[i, : len(order)] = cand[order]
        dist[i, : len(order)] = d[order]
    return idx, dist


CASES = [
    ("int64 narrow (many ties)", lambda: kdgen.cloud_int_uniform(3000, 3, 5, 11, np.int64, dup_frac=0.02)),
    ("int32 k=2", lambda: kdgen.cloud_int_uniform(2500, 2, 12, 12, np.int32)),
    ("float32 mixture k=4", lambda: kdgen.cloud_gmm(2000, 4, 13)),
    ("int64 wide k=5", lambda: kdgen.cloud_int_uniform(1500, 5, 40, 14, np.int64)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_knn_matches_numpy_brute_force(case):
    coords = CASES[case][1]()
    cand = oracle.presort(coords)[0]
    rng = np.random.default_rng(case)
    queries = coords[rng.choice(len(coords), 40)].copy()
    if coords.dtype.kind == "f":
        queries += rng.normal(0, 1, queries.shape).astype(np.float32)
    else:
        queries += rng.integers(-2, 3, queries.shape).astype(coords.dtype)
    for kn in (1, 5, 16):
        got_i, got_d = oracle.knn(coords, queries, kn, cand)
        ref_i, ref_d = numpy_knn(coords, cand, queries, kn)
        np.testing.assert_array_equal(got_i, ref_i)
        np.testing.assert_array_equal(got_d, ref_d)


def test_knn_special_cases():
    coords = np.array([[0, 0], [3, 4], [0, 0], [6, 8], [-3, -4]], dtype=np.int32)
    cand = oracle.presort(coords)[0]
    assert sorted(cand.tolist()) == [0, 1, 3, 4]  # tuple 2 duplicates tuple 0
    idx, d = oracle.knn(coords, np.array([[0, 0]], np.int32), 6, cand)
    # distance 0 first, then the two points at 25 by index, then 100; two empty slots
    assert idx[0].tolist() == [0, 1, 4, 3, -1, -1]
    assert d[0, :4].tolist() == [0.0, 25.0, 25.0, 100.0] and np.isinf(d[0, 4:]).all()
    # -0.0 and +0.0 are the same coordinate value
    f = np.array([[-0.0, 1.0], [2.0, 2.0]], np.float32)
    idx, d = oracle.knn(f, np.array([[0.0, 1.0]], np.float32), 1)
    assert idx[0, 0] == 0 and d[0, 0] == 0.0


def test_region_matches_numpy_and_bounds():
    coords = kdgen.cloud_int_uniform(4000, 3, 8, 21, np.int64, dup_frac=0.01)
    cand = oracle.presort(coords)[0]
    rng = np.random.default_rng(5)
    lo = rng.integers(0, 200, (30, 3)).astype(np.int64)
    hi = lo + rng.integers(0, 80, (30, 3))
    got = oracle.region(coords, lo, hi, cand)
    for i in range(30):
        inside = np.all((coords[cand] >= lo[i]) & (coords[cand] <= hi[i]), axis=1)
        np.testing.assert_array_equal(got[i], np.sort(cand[inside]))
    # the whole space holds every distinct tuple once; an inverted box holds none
    big = oracle.region(coords, np.full((1, 3), -1, np.int64), np.full((1, 3), 1 << 20, np.int64), cand)
    assert sorted(big[0].tolist()) == sorted(cand.tolist())
    assert oracle.region(coords, np.full((1, 3), 5, np.int64), np.full((1, 3), 4, np.int64), cand)[0].size == 0
