"""Array 0 sorted by x_0 alone, then every run of equal x_0 ordered by the
other coordinates (GPU only).  Runs of every length class (one tuple, a
warp's worth, a block's worth, and longer than a block, where array 0 takes
the whole-key sort instead), with exact duplicates inside runs, against the
oracle: presorted arrays and trees, element by element."""
import numpy as np
import pytest

import kdgen
import oracle

from test_gpu_parity import assert_same_tree, gpu_tree

pytestmark = pytest.mark.gpu

# run lengths around the two on-chip limits (32 tuples per warp, 2048 per block)
SHORT = [1, 2, 3, 5, 31, 32, 33, 34, 100, 2047, 2048]
LONG = [2049, 5000]


def runs_cloud(lengths, k, dtype, seed, other_bits=5):
    """x_0 constant on consecutive runs of the given lengths (shuffled), the
    other coordinates drawn from 2^other_bits values, so that runs hold exact
    duplicates too."""
    n = int(sum(lengths))
    x0 = np.repeat(np.arange(len(lengths), dtype=np.int64) * 7 - 11, lengths)
    rest = kdgen.uniform_int(seed, n * (k - 1), 0, 1 << other_bits).reshape(n, k - 1)
    c = np.concatenate([x0[:, None], rest.astype(np.int64)], axis=1)
    perm = np.argsort(kdgen.uniform_int(seed + 1, n, 0, 1 << 62), kind="stable")
    c = c[perm]
    if dtype == np.float32:
        return np.ascontiguousarray((c.astype(np.float64) * 0.25).astype(np.float32))
    return np.ascontiguousarray(c.astype(dtype))


def check(cuda_lib, ctx, coords):
    import torch
    h = cuda_lib.kd_presort(ctx, torch.from_numpy(coords).cuda())
    arrays = cuda_lib.kd_handle_arrays(ctx, h)
    cuda_lib.kd_release(ctx, h)
    np.testing.assert_array_equal(arrays, oracle.presort(coords))
    assert_same_tree(gpu_tree(cuda_lib, ctx, coords), oracle.build_tree(coords))


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.kd_create(0)
    yield c
    c.close()


@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.float32], ids=["i32", "i64", "f32"])
@pytest.mark.parametrize("k", [2, 3, 5, 8])
def test_runs_within_block(cuda_lib, ctx, dtype, k):
    check(cuda_lib, ctx, runs_cloud(SHORT * 2, k, dtype, 700 + k))


@pytest.mark.parametrize("dtype", [np.int32, np.int64], ids=["i32", "i64"])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_run_longer_than_a_block_takes_whole_key_sort(cuda_lib, ctx, dtype, k):
    check(cuda_lib, ctx, runs_cloud(SHORT + LONG, k, dtype, 720 + k))


# runs that begin on a tile's last position (2047, 4095, ...), end on a
# tile's first, or span a whole tile (tiles of 2048 positions)
EDGES = [2047, 2, 2046, 2, 2046, 3, 2045, 1, 1, 2047, 33, 2015, 40, 2008, 2048, 2048, 1, 2047, 300]


@pytest.mark.parametrize("dtype", [np.int32, np.int64], ids=["i32", "i64"])
@pytest.mark.parametrize("k", [2, 3])
def test_runs_at_tile_edges(cuda_lib, ctx, dtype, k):
    check(cuda_lib, ctx, runs_cloud(EDGES, k, dtype, 750 + k, other_bits=7))


@pytest.mark.parametrize("length", [100, 300], ids=["runs_ordered_on_chip", "runs_costly_whole_key_sort"])
def test_run_cost_threshold(cuda_lib, ctx, length):
    """Runs of 100 tuples cost 100 compares per tuple (ordered on chip);
    runs of 300 cost 300, above the threshold, so array 0 takes the
    whole-key sort: both equal the oracle."""
    check(cuda_lib, ctx, runs_cloud([length] * 40, 3, np.int32, 760 + length, other_bits=8))


def test_all_tuples_share_x0(cuda_lib, ctx):
    c = runs_cloud([30000], 3, np.int64, 731, other_bits=9)
    check(cuda_lib, ctx, c)


def test_batch_with_runs(cuda_lib, ctx):
    clouds = [runs_cloud(SHORT, 3, np.int32, 740 + i) for i in range(3)]
    clouds.append(runs_cloud(SHORT + LONG, 3, np.int32, 744))
    clouds.append(kdgen.cloud_int_uniform(5000, 3, 20, 745, np.int32))
    outs = cuda_lib.kd_build_batch(ctx, clouds)
    for c, got in zip(clouds, outs):
        assert_same_tree(got, oracle.build_tree(c))


def test_mixture_runs_at_one_million(cuda_lib, ctx):
    """The float32 mixture at 2^20 (narrow components repeat x_0 values):
    the tree equals the oracle's."""
    c = kdgen.cloud_gmm(1 << 20, 3, 746, sigma_lo=0.001, sigma_hi=0.01)
    assert_same_tree(gpu_tree(cuda_lib, ctx, c), oracle.build_tree(c))
