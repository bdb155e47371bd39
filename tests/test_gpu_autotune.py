"""Autotuner (GPU only): kd_autotune picks the on-chip subtree size and the
level-step tile per (k, dtype, size bucket) from device timings and keeps
them in a cache file; every candidate pair builds the oracle's tree, so a
tuned build and a default build are identical."""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")


def same(got, ref):
    assert got["m"] == ref["m"]
    for f in FIELDS:
        a = got[f]
        np.testing.assert_array_equal(a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a), ref[f], err_msg=f)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_autotune_cache_round_trip_and_tuned_build_equals_oracle(cuda_lib, tmp_path):
    cache = str(tmp_path / "kd_tune.txt")
    ctx = cuda_lib.kd_create(0, tune_cache=cache)
    try:
        chosen = cuda_lib.kd_autotune(ctx, 3, "float32", 1 << 18, reps=2)
        assert chosen["switch_threshold"] in (1024, 2048, 4096)
        assert chosen["level_tile"] in (1024, 2048)
        assert cuda_lib.kd_tuning_get(ctx, 3, "float32", (1 << 18) + 5) == chosen  # same bucket
    finally:
        ctx.close()
    rows = [line.split() for line in open(cache).read().splitlines()]
    assert rows == [["3", "2", "18", str(chosen["switch_threshold"]), str(chosen["level_tile"]), rows[0][5]]]
    ctx2 = cuda_lib.kd_create(0, tune_cache=cache)  # a new context reads the cache
    try:
        assert cuda_lib.kd_tuning_get(ctx2, 3, "float32", 1 << 18) == chosen
        coords = kdgen.cloud_gmm((1 << 18) + 123, 3, 31)
        same(cuda_lib.build_tree(ctx2, dev(coords)), oracle.build_tree(coords))
        # a fixed setting overrides the tuned one
        ctx3 = cuda_lib.kd_create(0, tune_cache=cache, switch_threshold=4096, level_tile=1024)
        assert cuda_lib.kd_tuning_get(ctx3, 3, "float32", 1 << 18) == {"switch_threshold": 4096, "level_tile": 1024}
        ctx3.close()
    finally:
        ctx2.close()


@pytest.mark.parametrize("k,dtype", [(3, np.float32), (2, np.int64), (4, np.int32), (5, np.int64)])
def test_every_candidate_builds_the_same_tree(cuda_lib, k, dtype):
    if dtype == np.float32:
        coords = kdgen.cloud_gmm(150001 + k, k, 40 + k)
    else:
        coords = kdgen.cloud_int_uniform(150001 + k, k, 30, 40 + k, dtype, dup_frac=0.01)
    ref = oracle.build_tree(coords)
    x = dev(coords)
    seen = set()
    for sm in (1024, 2048, 4096):
        for lt in (1024, 2048):
            ctx = cuda_lib.kd_create(0, switch_threshold=sm, level_tile=lt)
            try:
                used = cuda_lib.kd_tuning_get(ctx, k, coords.dtype, coords.shape[0])
                seen.add((used["switch_threshold"], used["level_tile"]))
                same(cuda_lib.build_tree(ctx, x), ref)
            finally:
                ctx.close()
    # subtrees of 4096 serve k <= 3, of 2048 k <= 4; tiles of 2048 serve k <= 4
    assert len(seen) == {2: 6, 3: 6, 4: 4, 5: 1}[k]


def test_batched_build_uses_the_tuned_pair(cuda_lib, tmp_path):
    clouds = kdgen.batch_clouds(count=60, seed=45, lo_log2=6.0, hi_log2=15.0)
    big = max(c.shape[0] for c in clouds)
    ctx = cuda_lib.kd_create(0, tune_cache=str(tmp_path / "t.txt"))
    try:
        chosen = cuda_lib.kd_autotune(ctx, 3, "float32", big, reps=1)
        assert cuda_lib.kd_tuning_get(ctx, 3, "float32", big) == chosen
        outs = cuda_lib.kd_build_batch(ctx, [dev(c) for c in clouds])
        for c, got in zip(clouds, outs):
            same(got, oracle.build_tree(c))
    finally:
        ctx.close()
