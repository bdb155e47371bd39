"""Every build workload at its full stated size, compared element by element
with the CPU oracle through the C ABI (GPU only).

- plain-large: n = 2^26 float32 Gaussian mixture (seed 2), k = 3, in the
  benchmark's launch configuration (device buffers, torch's stream).  Only
  this size runs the level scan's look-back across chunks of 4096 tiles and
  the sort scan's chains of 512 chunks.
- dimension sweep: n = 2^22 int64 uniform in [0, 2^40) at k = 2..6
  (seed 3 + k).
- batched: all 4096 clouds of the batched workload (seed 4) from one
  kd_build_batch call.
- served: a slice of the Poisson request stream (seed 5): the largest
  request of every (k, coordinate kind) pair (sizes near 2^20) and the first
  18 requests, submitted together through kd_submit.

m, node_tuple, left, right and dim must be bit-identical.  The oracle's C
calls release the interpreter lock, so it runs in host threads while the
GPU works.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")
THREADS = max(1, min(16, os.cpu_count() or 1))


def to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def assert_same_tree(got, ref, what=""):
    assert got["m"] == ref["m"], what
    assert got["root"] == ref["root"], what
    for f in FIELDS:
        np.testing.assert_array_equal(to_np(got[f]), ref[f], err_msg=f"{what} {f}")


@pytest.mark.slow
def test_plain_large_2p26_equals_oracle(cuda_lib):
    import torch
    coords = kdgen.large_gmm()
    with ThreadPoolExecutor(1) as pool:
        ref_f = pool.submit(oracle.build_tree, coords)
        stream = torch.cuda.current_stream()
        ctx = cuda_lib.kd_create(0, stream=stream)
        try:
            x = torch.from_numpy(coords).cuda()
            got = cuda_lib.build_tree(ctx, x, children=True, on_device=True)
            got = {key: (to_np(v) if key in FIELDS else v) for key, v in got.items()}
            del x
        finally:
            ctx.close()
        ref = ref_f.result()
    assert ref["m"] < coords.shape[0]  # the mixture has exact duplicates at 2^26
    assert_same_tree(got, ref, "2^26 float32 mixture")


@pytest.mark.slow
def test_dimension_sweep_2p22_equals_oracle(cuda_lib):
    import torch
    ks = [2, 3, 4, 5, 6]
    clouds = {k: kdgen.sweep_int64(k) for k in ks}
    with ThreadPoolExecutor(len(ks)) as pool:
        refs = {k: pool.submit(oracle.build_tree, clouds[k]) for k in ks}
        ctx = cuda_lib.kd_create(0)
        try:
            got = {}
            for k in ks:
                t = cuda_lib.build_tree(ctx, torch.from_numpy(clouds[k]).cuda(), children=True, on_device=True)
                got[k] = {key: (to_np(v) if key in FIELDS else v) for key, v in t.items()}
        finally:
            ctx.close()
        for k in ks:
            assert_same_tree(got[k], refs[k].result(), f"n=2^22 int64 k={k}")


@pytest.mark.slow
def test_batched_4096_clouds_equal_oracle(cuda_lib):
    import torch
    clouds = kdgen.batch_clouds(count=4096, seed=4)
    with ThreadPoolExecutor(THREADS) as pool:
        refs = [pool.submit(oracle.build_tree, c) for c in clouds]
        ctx = cuda_lib.kd_create(0)
        try:
            outs = cuda_lib.kd_build_batch(ctx, [torch.from_numpy(c).cuda() for c in clouds])
            host = {f: to_np(outs.arrays[f]) for f in FIELDS}
            trees = cuda_lib.BatchTrees(outs.m, outs.root, outs.offs, host)
        finally:
            ctx.close()
        for i, r in enumerate(refs):
            assert_same_tree(trees[i], r.result(), f"cloud {i} (n={clouds[i].shape[0]})")


def served_slice():
    reqs = kdgen.serving_requests(count=20000, seed=5)
    pick = set(range(18))
    for k in (2, 3, 4):
        for kind in (0, 1):
            best = max((i for i, r in enumerate(reqs) if r[1] == k and r[2] == kind), key=lambda i: reqs[i][0])
            pick.add(best)
    return [reqs[i] for i in sorted(pick)]


@pytest.mark.slow
def test_served_slice_up_to_2p20_equals_oracle(cuda_lib):
    sl = served_slice()
    assert max(r[0] for r in sl) > (1 << 19) and {r[1] for r in sl} == {2, 3, 4}
    clouds = [kdgen.serving_cloud(*r) for r in sl]
    with ThreadPoolExecutor(THREADS) as pool:
        refs = [pool.submit(oracle.build_tree, c) for c in clouds]
        ctx = cuda_lib.kd_create(0, mem_budget_bytes=64 << 30)
        try:
            tickets = [cuda_lib.kd_submit(ctx, c) for c in clouds]
            got = [cuda_lib.kd_wait(ctx, t, 600000) for t in tickets]
        finally:
            ctx.close()
        for r, c, g, ref in zip(sl, clouds, got, refs):
            assert_same_tree(g, ref.result(), f"request n={r[0]} k={r[1]} kind={r[2]}")
