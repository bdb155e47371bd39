"""Level schedules (GPU only): the default multi-level schedule, the
paper's deferred partitioning (Appendix "Deferred Merge Sort and
Partitioning") and its Section 2.1 form (every non-primary array
partitioned at every level) select the same medians, so each must give the
oracle's tree bit for bit, for single clouds and batches."""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")
SCHEDULES = (0, 1, 2)


def same(got, ref, what=""):
    assert got["m"] == ref["m"], what
    for f in FIELDS:
        a = got[f]
        np.testing.assert_array_equal(a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a), ref[f],
                                      err_msg=f"{what} {f}")


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 8])
def test_every_schedule_builds_the_oracle_tree(cuda_lib, k):
    coords = kdgen.cloud_int_uniform(90001 + k, k, 24, 500 + k, np.int64, dup_frac=0.01)
    ref = oracle.build_tree(coords)
    x = dev(coords)
    for sched in SCHEDULES:
        ctx = cuda_lib.kd_create(0, schedule=sched, switch_threshold=1024)
        try:
            same(cuda_lib.build_tree(ctx, x), ref, f"k={k} schedule={sched}")
        finally:
            ctx.close()


def test_every_schedule_builds_batches(cuda_lib):
    clouds = kdgen.batch_clouds(count=50, seed=46, lo_log2=6.0, hi_log2=16.0)
    refs = [oracle.build_tree(c) for c in clouds]
    devs = [dev(c) for c in clouds]
    for sched in SCHEDULES:
        ctx = cuda_lib.kd_create(0, schedule=sched)
        try:
            for c, got, ref in zip(clouds, cuda_lib.kd_build_batch(ctx, devs), refs):
                same(got, ref, f"schedule={sched} n={c.shape[0]}")
        finally:
            ctx.close()


def test_schedule_out_of_range_is_refused(cuda_lib):
    with pytest.raises(cuda_lib.KdError):
        cuda_lib.kd_create(0, schedule=3)
