"""The O(n log n) median-selection build (kd_build_select) against the CPU
oracle, through the C ABI (GPU only).

The selection build and the presorting build select the same unique median
at every level, so both must give the oracle's tree bit for bit: m,
node_tuple, left, right and dim.  Sizes span the finisher's units (512,
1024 and 2048 tuples), the level kernels' tiles (1024 and 2048 positions)
and several global levels."""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.kd_create(0)
    yield c
    c.close()


def same(got, ref, what=""):
    assert got["m"] == ref["m"], what
    assert got["root"] == ref["root"], what
    for f in FIELDS:
        a = got[f]
        np.testing.assert_array_equal(a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a), ref[f],
                                      err_msg=f"{what} {f}")


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    ("i64_small_dups", lambda: kdgen.small_int64(seed=7)),
    ("f32_gmm", lambda: kdgen.cloud_gmm(70001, 3, 201)),
    ("f32_ties", lambda: (np.round(kdgen.cloud_gmm(40000, 3, 202, components=3) * 4) / 4).astype(np.float32)),
    ("i32_neg", lambda: kdgen.cloud_int_uniform(30000, 3, 31, 203, np.int32) - (1 << 30)),
    ("k1", lambda: kdgen.cloud_int_uniform(9000, 1, 12, 204, np.int64)),
    ("k2", lambda: kdgen.cloud_int_uniform(50000, 2, 40, 205, np.int64)),
    ("k4", lambda: kdgen.cloud_int_uniform(50000, 4, 40, 206, np.int64)),
    ("k5_i32_dups", lambda: kdgen.cloud_int_uniform(30000, 5, 8, 207, np.int32, dup_frac=0.02)),
    ("k6", lambda: kdgen.cloud_int_uniform(40000, 6, 40, 208, np.int64)),
    ("k8_narrow", lambda: kdgen.cloud_int_uniform(20000, 8, 3, 209, np.int32)),
    ("k8_i64", lambda: kdgen.cloud_int_uniform(30000, 8, 40, 210, np.int64)),
    ("many_dups", lambda: kdgen.cloud_int_uniform(60000, 3, 4, 211, np.int64)),
]


@pytest.mark.parametrize("name,gen", CASES, ids=[c[0] for c in CASES])
def test_select_build_equals_oracle(cuda_lib, ctx, name, gen):
    coords = gen()
    same(cuda_lib.kd_build_select(ctx, dev(coords)), oracle.build_tree(coords), name)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 31, 32, 33, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049,
                               4095, 4097, 8193, 100003])
def test_select_build_ragged_sizes(cuda_lib, ctx, n):
    coords = kdgen.cloud_int_uniform(n, 3, 30, 3000 + n, np.int64)
    same(cuda_lib.kd_build_select(ctx, dev(coords)), oracle.build_tree(coords), f"n={n}")


def test_select_build_host_buffers_and_equal_to_presorting_build(cuda_lib, ctx):
    coords = kdgen.cloud_gmm(120001, 3, 212)
    got = cuda_lib.kd_build_select(ctx, coords)  # numpy in, numpy out
    assert isinstance(got["node_tuple"], np.ndarray)
    ref = oracle.build_tree(coords)
    same(got, ref)
    same(cuda_lib.build_tree(ctx, coords), ref)


def test_select_build_many_global_levels(cuda_lib, ctx):
    coords = kdgen.cloud_gmm((1 << 21) + 7, 3, 213)  # ten levels above the on-chip units
    same(cuda_lib.kd_build_select(ctx, dev(coords)), oracle.build_tree(coords))


def test_select_build_errors(cuda_lib, ctx):
    bad = kdgen.cloud_gmm(5000, 3, 214)
    bad[9, 2] = np.nan
    with pytest.raises(cuda_lib.KdError) as e:
        cuda_lib.kd_build_select(ctx, dev(bad))
    assert e.value.code == -6
    ok = kdgen.cloud_gmm(5000, 3, 215)
    same(cuda_lib.kd_build_select(ctx, dev(ok)), oracle.build_tree(ok))
