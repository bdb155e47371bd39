"""Searches over a GPU-built tree (kd_index_create, kd_knn, kd_region)
through the C ABI, compared with the brute-force search oracle: the same
neighbour indices and bit-identical squared distances, the same region
result sets.  GPU only."""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu


def queries_near(coords, nq, seed):
    rng = np.random.default_rng(seed)
    q = coords[rng.choice(len(coords), nq)].copy()
    if coords.dtype.kind == "f":
        q += rng.normal(0, 2, q.shape).astype(np.float32)
    else:
        q += rng.integers(-3, 4, q.shape).astype(coords.dtype)
    return q


CASES = [
    ("float32 mixture k=3", lambda: kdgen.cloud_gmm(20000, 3, 31), 1, 8),
    ("int64 narrow k=3, ties and duplicates", lambda: kdgen.cloud_int_uniform(12000, 3, 6, 32, np.int64,
                                                                           dup_frac=0.02), 2, 16),
    ("int32 k=2", lambda: kdgen.cloud_int_uniform(9000, 2, 14, 33, np.int32), 3, 5),
    ("int64 wide k=5", lambda: kdgen.cloud_int_uniform(7000, 5, 40, 34, np.int64), 4, 32),
    ("unit cube k=4", lambda: kdgen.cloud_unit_cube(5000, 4, 35), 5, 1),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_knn_equals_brute_force(cuda_lib, case):
    import torch
    name, gen, seed, kn = CASES[case]
    coords = gen()
    ctx = cuda_lib.kd_create(0)
    try:
        tree = cuda_lib.build_tree(ctx, torch.from_numpy(coords).cuda())
        ix = cuda_lib.kd_index_create(ctx, torch.from_numpy(coords).cuda(), tree)
        q = queries_near(coords, 300, seed)
        ref_i, ref_d = oracle.knn(coords, q, kn)
        gi, gd = cuda_lib.kd_knn(ctx, ix, torch.from_numpy(q).cuda(), kn)
        np.testing.assert_array_equal(gi.cpu().numpy(), ref_i, err_msg=name)
        np.testing.assert_array_equal(gd.cpu().numpy(), ref_d, err_msg=name)
        # host queries and host outputs give the same answer
        hi_, hd = cuda_lib.kd_knn(ctx, ix, q, kn)
        np.testing.assert_array_equal(hi_, ref_i)
        np.testing.assert_array_equal(hd, ref_d)
        cuda_lib.kd_index_destroy(ctx, ix)
    finally:
        ctx.close()


def test_knn_more_neighbours_than_tuples_and_errors(cuda_lib):
    coords = np.array([[0, 0], [3, 4], [0, 0], [6, 8]], dtype=np.int32)
    ctx = cuda_lib.kd_create(0)
    try:
        tree = cuda_lib.build_tree(ctx, coords)
        ix = cuda_lib.kd_index_create(ctx, coords, tree)
        idx, d = cuda_lib.kd_knn(ctx, ix, np.array([[0, 0], [5, 5]], np.int32), 5)
        ref_i, ref_d = oracle.knn(coords, np.array([[0, 0], [5, 5]], np.int32), 5)
        np.testing.assert_array_equal(idx, ref_i)
        np.testing.assert_array_equal(d, ref_d)
        assert idx[0].tolist()[:3] == [0, 1, 3] and idx[0, 3] == -1
        with pytest.raises(cuda_lib.KdError):
            cuda_lib.kd_knn(ctx, ix, np.zeros((1, 2), np.int32), 33)
        cuda_lib.kd_index_destroy(ctx, ix)
        f = kdgen.cloud_gmm(500, 3, 2)
        tf = cuda_lib.build_tree(ctx, f)
        ixf = cuda_lib.kd_index_create(ctx, f, tf)
        bad = f[:2].copy()
        bad[1, 2] = np.nan
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.kd_knn(ctx, ixf, bad, 3)
        assert e.value.code == -6
        cuda_lib.kd_index_destroy(ctx, ixf)
    finally:
        ctx.close()


@pytest.mark.parametrize("case", range(3))
def test_region_equals_brute_force(cuda_lib, case):
    import torch
    name, gen, seed, _ = CASES[case]
    coords = gen()
    rng = np.random.default_rng(seed)
    ctx = cuda_lib.kd_create(0)
    try:
        tree = cuda_lib.build_tree(ctx, torch.from_numpy(coords).cuda())
        ix = cuda_lib.kd_index_create(ctx, torch.from_numpy(coords).cuda(), tree)
        centres = queries_near(coords, 200, seed + 7)
        if coords.dtype.kind == "f":
            half = rng.uniform(0.0, 20.0, centres.shape).astype(np.float32)
        else:
            half = rng.integers(0, 40, centres.shape).astype(coords.dtype)
        lo, hi = centres - half, centres + half
        lo[0], hi[0] = hi[0], lo[0]  # an empty (inverted) box
        ref = oracle.region(coords, lo, hi)
        for dev in (True, False):
            L = torch.from_numpy(lo).cuda() if dev else lo
            H = torch.from_numpy(hi).cuda() if dev else hi
            offs, idx = cuda_lib.kd_region(ctx, ix, L, H)
            offs = offs.cpu().numpy() if dev else offs
            idx = idx.cpu().numpy() if dev else idx
            for i in range(len(lo)):
                np.testing.assert_array_equal(np.sort(idx[offs[i]:offs[i + 1]]), ref[i], err_msg=f"{name} box {i}")
        cuda_lib.kd_index_destroy(ctx, ix)
    finally:
        ctx.close()


@pytest.mark.parametrize("case", [0, 1])
def test_all_points_and_reverse_neighbours(cuda_lib, case):
    import torch
    name, gen, seed, kn = CASES[case]
    coords = gen()[:6000]
    ctx = cuda_lib.kd_create(0)
    try:
        tree = cuda_lib.build_tree(ctx, torch.from_numpy(coords).cuda())
        ix = cuda_lib.kd_index_create(ctx, torch.from_numpy(coords).cuda(), tree)
        m = tree["m"]
        node = tree["node_tuple"].cpu().numpy()
        gi, gd = cuda_lib.kd_knn_all(ctx, ix, m, kn)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        # oracle: every tree tuple as a query, its own tuple (distance 0, first) dropped
        ref_i, ref_d = oracle.knn(coords, coords[node], kn + 1)
        assert (ref_i[:, 0] == node).all()
        np.testing.assert_array_equal(gi, ref_i[:, 1:], err_msg=name)
        np.testing.assert_array_equal(gd, ref_d[:, 1:], err_msg=name)
        offs, rev = cuda_lib.kd_reverse_knn(ctx, ix, m, kn)
        offs, rev = offs.cpu().numpy(), rev.cpu().numpy()
        addr_of = {int(t): a for a, t in enumerate(node)}
        lists = [[] for _ in range(m)]
        for a in range(m):
            for u in ref_i[a, 1:]:
                if u >= 0:
                    lists[addr_of[int(u)]].append(int(node[a]))
        assert offs[-1] == sum(len(x) for x in lists)
        for a in range(m):
            assert sorted(rev[offs[a]:offs[a + 1]].tolist()) == sorted(lists[a]), (name, a)
        cuda_lib.kd_index_destroy(ctx, ix)
    finally:
        ctx.close()
