"""Pins for the CPU oracle (no GPU).

The oracle (oracle/kd_oracle.c) is checked against things other than itself:
values the paper prints for its 15-tuple example (tests/golden), library
sorting as a special case of the presort, two independent brute-force
builders, closed forms (k = 1, all-identical input, tiny n), the Section 2.1
invariants, and a mutation check showing that each planted mistake fails
at least one of these pins.
"""
import os

import numpy as np
import pytest

import kdgen
import oracle
from bruteforce import (check_invariants, levelwise_build, presort_sorted, resort_build,
                        unique_representatives)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")
ARRAYS = {"xyz": 0, "yzx": 1, "zxy": 2}


def load_golden():
    tuples, facts = {}, []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            w = line.split()
            if w[0] == "tuple":
                tuples[int(w[1])] = tuple(int(v) for v in w[2:])
            else:
                facts.append(w)
    coords = np.array([tuples[i] for i in range(len(tuples))], dtype=np.int64)
    return coords, facts


def check_worked_example(mutant=0):
    coords, facts = load_golden()
    arrays = oracle.presort(coords, mutant=mutant)
    split, med = oracle.first_split(coords, mutant=mutant)
    tree = oracle.build_tree(coords, mutant=mutant)
    for w in facts:
        kind = w[0]
        if kind in ("prefix", "suffix"):
            vals = [int(v) for v in w[2:]]
            row = list(arrays[ARRAYS[w[1]]])
            got = row[: len(vals)] if kind == "prefix" else row[-len(vals):]
            assert got == vals, (w, got)
        elif kind == "root":
            assert tree["root"] == int(w[1]) and tree["node_tuple"][int(w[1])] == int(w[2])
            assert med == int(w[2])
        elif kind == "after_first_split":
            assert split[ARRAYS[w[1]], int(w[2])] == int(w[3]), w
        elif kind == "absent_after_first_split":
            mid = (split.shape[1] - 1) // 2
            for d in range(1, split.shape[0]):
                row = list(split[d, :mid]) + list(split[d, mid + 1:])
                assert int(w[1]) not in row
        elif kind == "node":
            depth, addr, tup = int(w[1]), int(w[2]), int(w[3])
            assert tree["node_tuple"][addr] == tup, w
            assert tree["dim"][addr] == depth % 3
        else:
            raise AssertionError(f"unknown golden fact {w}")
    return tree


def test_worked_example_printed_values():
    tree = check_worked_example()
    assert tree["m"] == 15


def test_worked_example_matches_bruteforce():
    coords, _ = load_golden()
    t = oracle.build_tree(coords)
    b = resort_build(coords)
    for f in ("node_tuple", "left", "right", "dim"):
        np.testing.assert_array_equal(t[f], b[f])


def _random_clouds():
    out = []
    for seed in range(6):
        n = [0, 1, 2, 3, 37, 200][seed]
        out.append(kdgen.cloud_int_uniform(n, 3, 3, seed, np.int64, dup_frac=0.1))
    out.append(kdgen.cloud_int_uniform(300, 2, 4, 11, np.int32, dup_frac=0.05))
    out.append(kdgen.cloud_int_uniform(150, 4, 2, 12, np.int64))  # many ties and duplicates
    out.append(kdgen.cloud_int_uniform(120, 5, 3, 13, np.int32) - 4)  # negatives
    f = kdgen.cloud_gmm(256, 3, 14, components=4, sigma_lo=0.5, sigma_hi=1.0)
    f = np.round(f * 2) / 2  # force coordinate ties
    out.append(f.astype(np.float32))
    g = kdgen.cloud_unit_cube(100, 3, 15, dup_frac=0.05) - np.float32(0.5)
    out.append(g)
    out.append(kdgen.cloud_int_uniform(64, 1, 5, 16, np.int64))
    return out


@pytest.mark.parametrize("idx", range(12))
def test_presort_is_library_sort(idx):
    coords = _random_clouds()[idx]
    got = oracle.presort(coords)
    ref = presort_sorted(coords)
    assert got.shape[0] == coords.shape[1]
    for d in range(coords.shape[1]):
        assert list(got[d]) == ref[d]


@pytest.mark.parametrize("idx", range(12))
@pytest.mark.parametrize("terminate_small", [True, False])
def test_build_equals_resort_bruteforce(idx, terminate_small):
    coords = _random_clouds()[idx]
    t = oracle.build_tree(coords, terminate_small=terminate_small)
    b = resort_build(coords)
    assert t["m"] == b["m"]
    for f in ("node_tuple", "left", "right", "dim"):
        np.testing.assert_array_equal(t[f], b[f])
    check_invariants(coords, t)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_build_equals_levelwise_numpy(seed):
    coords = kdgen.cloud_int_uniform(5000, 3, 8, seed, np.int64, dup_frac=0.02)
    t = oracle.build_tree(coords)
    b = levelwise_build(coords)
    assert t["m"] == b["m"]
    np.testing.assert_array_equal(t["node_tuple"], b["node_tuple"])


def test_small_workload_invariants_and_levelwise():
    coords = kdgen.small_int64()
    t = oracle.build_tree(coords)
    assert t["m"] == len(unique_representatives(coords)) < coords.shape[0]
    b = levelwise_build(coords)
    np.testing.assert_array_equal(t["node_tuple"], b["node_tuple"])


def test_k1_is_sorted_unique():
    coords = kdgen.cloud_int_uniform(500, 1, 7, 31, np.int64)
    t = oracle.build_tree(coords)
    vals = coords[:, 0]
    reps = unique_representatives(coords)
    expect = sorted(reps, key=lambda i: vals[i])
    np.testing.assert_array_equal(t["node_tuple"], np.array(expect, dtype=np.int32))


def test_all_identical_gives_single_node():
    coords = np.full((40, 3), 7, dtype=np.int32)
    t = oracle.build_tree(coords)
    assert t["m"] == 1 and t["node_tuple"][0] == 0 and t["left"][0] == -1 and t["right"][0] == -1


def test_tiny_n_termination_cases():
    # n = 1, 2, 3 follow the Section 2.1 termination paragraph
    c1 = np.array([[5, 1]], dtype=np.int32)
    assert list(oracle.build_tree(c1)["node_tuple"]) == [0]
    c2 = np.array([[9, 1], [2, 1]], dtype=np.int32)
    t2 = oracle.build_tree(c2)  # sorted order is 1, 0: node is the lower, right child the other
    assert list(t2["node_tuple"]) == [1, 0] and list(t2["right"]) == [1, -1] and list(t2["left"]) == [-1, -1]
    c3 = np.array([[9, 0], [2, 0], [5, 0]], dtype=np.int32)
    t3 = oracle.build_tree(c3)
    assert list(t3["node_tuple"]) == [1, 2, 0] and t3["root"] == 1
    assert list(t3["left"]) == [-1, 0, -1] and list(t3["right"]) == [-1, 2, -1]
    assert oracle.build_tree(np.zeros((0, 3), dtype=np.int64))["m"] == 0


def test_negative_zero_is_a_duplicate_and_nan_rejected():
    c = np.array([[0.0, 1.0], [-0.0, 1.0], [-1.0, 2.0]], dtype=np.float32)
    t = oracle.build_tree(c)
    assert t["m"] == 2 and sorted(t["node_tuple"]) == [0, 2]
    c[2, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_tree(c)
    assert e.value.code == oracle.ENAN


def test_depth_bound_and_shape_depends_only_on_m():
    for n in [1, 2, 5, 16, 17, 100, 1023, 1024]:
        a = oracle.build_tree(kdgen.cloud_int_uniform(n, 2, 30, n, np.int64))
        b = oracle.build_tree(kdgen.cloud_int_uniform(n, 3, 30, n + 1, np.int64))
        assert a["m"] == b["m"] == n
        np.testing.assert_array_equal(a["left"], b["left"])
        np.testing.assert_array_equal(a["right"], b["right"])
        check_invariants(kdgen.cloud_int_uniform(n, 2, 30, n, np.int64), a)


def test_partitioned_halves_stay_sorted():
    coords = kdgen.cloud_int_uniform(333, 3, 5, 41, np.int64, dup_frac=0.03)
    split, med = oracle.first_split(coords)
    m = split.shape[1]
    mid = (m - 1) // 2
    from bruteforce import superkey
    c = [tuple(int(v) for v in r) for r in coords]
    for d in range(3):
        for lo, hi in ((0, mid - 1), (mid + 1, m - 1)):
            seg = [int(v) for v in split[d, lo:hi + 1]]
            keys = [superkey(c, t, d) for t in seg]
            assert keys == sorted(keys)
            for t in seg:
                assert (superkey(c, t, 0) < superkey(c, med, 0)) == (lo == 0)


MUTANTS = [1, 2, 3, 4, 5, 6, 7]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_each_planted_mistake_fails_a_pin(mutant):
    """Every deliberate oracle mistake (see kd_oracle.c) is caught."""
    caught = []
    try:
        check_worked_example(mutant)
    except (AssertionError, oracle.OracleError, IndexError):
        caught.append("worked example")
    for coords in _random_clouds():
        try:
            got = oracle.presort(coords, mutant=mutant)
            ref = presort_sorted(coords)
            for d in range(coords.shape[1]):
                assert list(got[d]) == ref[d]
            t = oracle.build_tree(coords, mutant=mutant)
            b = resort_build(coords)
            for f in ("node_tuple", "left", "right", "dim"):
                np.testing.assert_array_equal(t[f], b[f])
        except (AssertionError, oracle.OracleError, IndexError):
            caught.append("bruteforce")
            break
    assert caught, f"mutant {mutant} not detected by any pin"


@pytest.mark.parametrize("levels", [1, 3])
def test_parallel_scheme_builds_the_same_tree(levels):
    """The paper's parallel execution scheme (a host baseline) gives the
    single-threaded oracle's tree."""
    import kdgen
    for coords in (kdgen.cloud_int_uniform(40000, 3, 10, 41, np.int64, dup_frac=0.01),
                   kdgen.cloud_gmm(30000, 4, 42)):
        ref = oracle.build_tree(coords)
        got = oracle.build_tree_parallel(coords, levels)
        assert got["m"] == ref["m"]
        for f in ("node_tuple", "left", "right", "dim"):
            np.testing.assert_array_equal(got[f], ref[f])
