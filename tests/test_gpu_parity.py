"""CUDA path vs the CPU oracle, through the C ABI (GPU only).

Integer/index work: bit-exact.  Every case compares m, node_tuple, left,
right and dim element by element; presorted arrays are compared too.
Sizes span several sort tiles (4096 keys), level-pass tiles (2048
positions) and finisher subtrees (2048 / 1024 tuples), with ragged tails.
"""
import numpy as np
import pytest

import kdgen
import oracle
from bruteforce import superkey

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.kd_create(0)
    yield c
    c.close()


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def assert_same_tree(got, ref):
    assert got["m"] == ref["m"]
    assert got["root"] == ref["root"]
    for f in FIELDS:
        np.testing.assert_array_equal(to_np(got[f]), ref[f], err_msg=f)


def gpu_tree(api, ctx, coords, device=True, **kw):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(coords))
    if device:
        x = x.cuda()
    return api.build_tree(ctx, x, **kw)


def test_worked_example_matches_oracle_and_paper(cuda_lib, ctx):
    from test_oracle import load_golden
    coords, facts = load_golden()
    got = gpu_tree(cuda_lib, ctx, coords)
    ref = oracle.build_tree(coords)
    assert_same_tree(got, ref)
    node = to_np(got["node_tuple"])
    for w in facts:
        if w[0] == "node":
            assert node[int(w[2])] == int(w[3])
        if w[0] == "root":
            assert node[int(w[1])] == int(w[2])


CASES = [
    # (name, generator)
    ("i64_small_dups", lambda: kdgen.cloud_int_uniform(3000, 3, 6, 101, np.int64, dup_frac=0.05)),
    ("i32_neg", lambda: kdgen.cloud_int_uniform(5000, 3, 31, 102, np.int32) - (1 << 30)),
    ("f32_gmm", lambda: kdgen.cloud_gmm(9000, 3, 103)),
    ("f32_ties", lambda: (np.round(kdgen.cloud_gmm(7000, 3, 104, components=3) * 4) / 4).astype(np.float32)),
    ("k1", lambda: kdgen.cloud_int_uniform(6000, 1, 12, 105, np.int64)),
    ("k2", lambda: kdgen.cloud_int_uniform(12000, 2, 40, 106, np.int64)),
    ("k4", lambda: kdgen.cloud_int_uniform(12000, 4, 40, 107, np.int64)),
    ("k5", lambda: kdgen.cloud_int_uniform(9000, 5, 8, 108, np.int32, dup_frac=0.02)),
    ("k6", lambda: kdgen.cloud_int_uniform(15000, 6, 40, 109, np.int64)),
    ("k8", lambda: kdgen.cloud_int_uniform(7000, 8, 3, 110, np.int32)),
    ("many_dups", lambda: kdgen.cloud_int_uniform(20000, 3, 4, 111, np.int64)),
]


@pytest.mark.parametrize("name,gen", CASES, ids=[c[0] for c in CASES])
def test_presort_arrays_match_oracle(cuda_lib, ctx, name, gen):
    import torch
    coords = gen()
    h = cuda_lib.kd_presort(ctx, torch.from_numpy(coords).cuda())
    arrays = cuda_lib.kd_handle_arrays(ctx, h)
    cuda_lib.kd_release(ctx, h)
    np.testing.assert_array_equal(arrays, oracle.presort(coords))


@pytest.mark.parametrize("name,gen", CASES, ids=[c[0] for c in CASES])
def test_tree_matches_oracle(cuda_lib, ctx, name, gen):
    coords = gen()
    assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 31, 32, 33, 1023, 1024, 1025, 2047, 2048, 2049, 4095,
                               4096, 4097, 8193, 40961, 100003])
def test_ragged_sizes(cuda_lib, ctx, n):
    coords = kdgen.cloud_int_uniform(n, 3, 30, 1000 + n, np.int64)
    assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))


# One finisher unit whose last block level is each depth dl = 0..4 (the
# unit holds 33..64, 65..128, ..., 513..1024 tuples): that level writes its
# primary array in final segment order itself, every other array goes
# through the multisplit.
UNIT_SIZES = [34, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 257, 511, 512, 513, 777, 1000]


@pytest.mark.parametrize("k", [2, 3, 5])
@pytest.mark.parametrize("n", UNIT_SIZES)
def test_finisher_unit_sizes(cuda_lib, ctx, n, k):
    coords = kdgen.cloud_int_uniform(n, k, 30, 4000 + 7 * n + k, np.int64)
    assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8])
def test_small_switch_threshold_runs_many_level_passes(cuda_lib, k):
    """A small on-chip threshold forces many fused level passes and catch-up
    passes on a size the oracle builds quickly."""
    ctx = cuda_lib.kd_create(0, switch_threshold=700)
    try:
        coords = kdgen.cloud_int_uniform(60000 + 37 * k, k, 20, 2000 + k, np.int64, dup_frac=0.01)
        assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))
    finally:
        ctx.close()


@pytest.mark.parametrize("k,threshold", [(2, 4096), (3, 4096), (4, 2048), (3, 1024), (8, 1024)])
def test_each_on_chip_subtree_size(cuda_lib, k, threshold):
    """Every on-chip subtree capacity (1024, 2048, 4096 tuples) finishes the
    same tree, including ragged units and narrow integers with ties."""
    ctx = cuda_lib.kd_create(0, switch_threshold=threshold)
    try:
        coords = kdgen.cloud_int_uniform(50000 + 11 * k, k, 12, 3000 + k, np.int64, dup_frac=0.01)
        assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))
    finally:
        ctx.close()


def test_small_workload_bit_exact(cuda_lib, ctx):
    coords = kdgen.small_int64()  # n=16384, k=3, int64 in [0, 2^20), 1% duplicates
    ref = oracle.build_tree(coords)
    assert ref["m"] < coords.shape[0]
    assert_same_tree(gpu_tree(cuda_lib, ctx, coords), ref)


def test_host_buffers_path(cuda_lib, ctx):
    coords = kdgen.cloud_gmm(30001, 3, 7)
    got = cuda_lib.build_tree(ctx, coords)  # numpy in, numpy out
    assert isinstance(got["node_tuple"], np.ndarray)
    assert_same_tree(got, oracle.build_tree(coords))


def test_deterministic(cuda_lib, ctx):
    coords = kdgen.cloud_gmm(200000, 3, 8)
    a = gpu_tree(cuda_lib, ctx, coords)
    b = gpu_tree(cuda_lib, ctx, coords)
    for f in FIELDS:
        np.testing.assert_array_equal(to_np(a[f]), to_np(b[f]))


def test_edge_cases_and_errors(cuda_lib, ctx):
    import torch
    # all identical -> one node
    t = gpu_tree(cuda_lib, ctx, np.full((5000, 3), 9, dtype=np.int32))
    assert t["m"] == 1 and to_np(t["node_tuple"])[0] == 0
    # -0.0 equals +0.0
    c = np.array([[0.0, 1.0], [-0.0, 1.0], [2.0, -3.0]], dtype=np.float32)
    assert_same_tree(gpu_tree(cuda_lib, ctx, c), oracle.build_tree(c))
    # NaN is rejected and the context stays usable
    bad = kdgen.cloud_gmm(1000, 3, 9)
    bad[17, 1] = np.nan
    with pytest.raises(cuda_lib.KdError) as e:
        gpu_tree(cuda_lib, ctx, bad)
    assert e.value.code == -6
    with pytest.raises(cuda_lib.KdError):
        cuda_lib.build_tree(ctx, torch.zeros((10, 9), dtype=torch.int32, device="cuda"))
    ok = kdgen.cloud_gmm(3000, 3, 10)
    assert_same_tree(gpu_tree(cuda_lib, ctx, ok), oracle.build_tree(ok))


def test_batch_equals_single_builds(cuda_lib, ctx):
    import torch
    clouds = kdgen.batch_clouds(count=40, seed=44, lo_log2=2.0, hi_log2=14.0)
    clouds.insert(3, np.zeros((0, 3), dtype=np.float32))
    dev = [torch.from_numpy(c).cuda() for c in clouds]
    outs = cuda_lib.kd_build_batch(ctx, dev)
    for c, got in zip(clouds, outs):
        assert_same_tree(got, oracle.build_tree(c))


def test_batch_packed_equals_list(cuda_lib, ctx):
    """Clouds stored back to back in one tensor give the same trees as the
    same clouds passed one tensor each."""
    import torch
    clouds = kdgen.batch_clouds(count=60, seed=46, lo_log2=2.0, hi_log2=13.0)
    packed = torch.from_numpy(np.concatenate(clouds)).cuda()
    a = cuda_lib.kd_build_batch_packed(ctx, packed, [c.shape[0] for c in clouds])
    b = cuda_lib.kd_build_batch(ctx, [torch.from_numpy(c).cuda() for c in clouds])
    for i, c in enumerate(clouds):
        for f in FIELDS:
            np.testing.assert_array_equal(to_np(a[i][f]), to_np(b[i][f]), err_msg=f)
        assert_same_tree(a[i], oracle.build_tree(c))


def test_batch_host_buffers_int64(cuda_lib, ctx):
    clouds = [kdgen.cloud_int_uniform(n, 4, 10, 50 + n, np.int64, dup_frac=0.03) for n in (1, 5000, 300, 9000)]
    outs = cuda_lib.kd_build_batch(ctx, clouds)
    for c, got in zip(clouds, outs):
        assert_same_tree(got, oracle.build_tree(c))


def test_pinned_host_inputs_and_outputs(cuda_lib, ctx):
    """Page-locked host coordinates in and page-locked host outputs out (the
    bench's end-to-end path): the coordinates go up in chunks, the children
    and split dimensions come back while the level passes run and the node
    tuples chunk by chunk behind the finisher."""
    import ctypes
    import torch
    from paper_1410_5420_gb300 import _lib
    n = (1 << 20) + 333  # above 2^20 (chunked upload) and more than 64 on-chip units
    coords = kdgen.cloud_gmm(n, 3, 611)
    ref = oracle.build_tree(coords)
    pin = torch.from_numpy(coords).pin_memory()
    outs = {"node_tuple": torch.full((n,), -9, dtype=torch.int32).pin_memory(),
            "left": torch.full((n,), -9, dtype=torch.int32).pin_memory(),
            "right": torch.full((n,), -9, dtype=torch.int32).pin_memory(),
            "dim": torch.full((n,), 99, dtype=torch.uint8).pin_memory()}
    lib = _lib.load()
    c = _lib.KdCloud(pin.data_ptr(), n, 3, _lib.KD_F32, 0)
    h = ctypes.c_void_p()
    ctx.check(lib.kd_presort(ctx.ptr, ctypes.byref(c), ctypes.byref(h)))
    tr = _lib.KdTree(0, -1, *(ctypes.c_void_p(outs[f].data_ptr()) for f in FIELDS), 0)
    ctx.check(lib.kd_build(ctx.ptr, h, ctypes.byref(tr)))
    got = {"m": tr.m, "root": tr.root}
    got.update({f: outs[f].numpy()[: tr.m] for f in FIELDS})
    assert_same_tree(got, ref)
