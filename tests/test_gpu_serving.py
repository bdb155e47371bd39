"""Serving (kd_submit / kd_wait) and batching through the C ABI (GPU only).

Each served or batched tree must be bit-identical to the same cloud built
alone and to the CPU oracle, whatever else shared its batch.
"""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")


def same(got, ref):
    assert got["m"] == ref["m"]
    for f in FIELDS:
        np.testing.assert_array_equal(np.asarray(got[f]), ref[f], err_msg=f)


def request_stream(count, seed):
    reqs = kdgen.serving_requests(count=count, seed=seed, lo_log2=4.0, hi_log2=13.0)
    return [kdgen.serving_cloud(*r) for r in reqs]


def test_served_results_equal_oracle_and_single_builds(cuda_lib):
    ctx = cuda_lib.kd_create(0)
    try:
        clouds = request_stream(120, 77)
        tickets = [cuda_lib.kd_submit(ctx, c) for c in clouds]
        for c, t in zip(clouds, tickets):
            got = cuda_lib.kd_wait(ctx, t, 60000)
            same(got, oracle.build_tree(c))
        # the same clouds built one by one give the same trees
        for c in clouds[:10]:
            alone = cuda_lib.build_tree(ctx, c)
            same(alone, oracle.build_tree(c))
        stats = cuda_lib.kd_serving_stats(ctx)
        assert stats["completed"] == len(clouds)
        assert stats["p99_us"] >= stats["p50_us"] > 0
    finally:
        ctx.close()


def test_requests_arriving_during_work_are_admitted(cuda_lib):
    """Submit in waves without waiting: later waves arrive while earlier
    batches run on the device and are co-batched as workers free up."""
    ctx = cuda_lib.kd_create(0, mem_budget_bytes=256 << 20)
    try:
        waves = [request_stream(40, 100 + w) for w in range(4)]
        tickets = []
        for wave in waves:
            tickets += [(c, cuda_lib.kd_submit(ctx, c)) for c in wave]
        for c, t in tickets:
            same(cuda_lib.kd_wait(ctx, t, 60000), oracle.build_tree(c))
    finally:
        ctx.close()


def test_ticket_errors(cuda_lib):
    ctx = cuda_lib.kd_create(0)
    try:
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.kd_wait(ctx, cuda_lib.Ticket(987654, None, {}, None), 0)
        assert e.value.code == -1
        bad = kdgen.cloud_gmm(100, 3, 5)
        bad[3, 0] = np.nan
        t = cuda_lib.kd_submit(ctx, bad)
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.kd_wait(ctx, t, 60000)
        assert e.value.code == -6
        ok = kdgen.cloud_gmm(1000, 3, 6)
        same(cuda_lib.kd_wait(ctx, cuda_lib.kd_submit(ctx, ok), 60000), oracle.build_tree(ok))
    finally:
        ctx.close()


def test_batched_large_mixed_equals_plain(cuda_lib):
    import torch
    clouds = kdgen.batch_clouds(count=300, seed=9, lo_log2=6.0, hi_log2=16.0)
    ctx = cuda_lib.kd_create(0)
    try:
        outs = cuda_lib.kd_build_batch(ctx, [torch.from_numpy(c).cuda() for c in clouds])
        rng = np.random.default_rng(1)
        for i in rng.choice(len(clouds), 25, replace=False):
            same({k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in outs[i].items()},
                 oracle.build_tree(clouds[i]))
        for i in range(0, len(clouds), 37):
            alone = cuda_lib.build_tree(ctx, torch.from_numpy(clouds[i]).cuda())
            for f in FIELDS:
                assert torch.equal(alone[f], outs[i][f])
    finally:
        ctx.close()
