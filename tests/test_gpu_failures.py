"""Failure detection through the C ABI (GPU only), in forms that fault,
trap or hang no GPU.

- A device wait that runs out: with the test setting (debug bit 8) the
  look-back polls are bounded by a few thousand and chunk 0 of the first
  sort pass withholds its flag once.  The blocks whose wait runs out store
  nothing and set the timeout bit; the call returns KD_ETIMEOUT, and the
  same context then builds a cloud that equals the oracle's tree.
- Budget exhaustion: a context whose memory budget is below what a cloud
  needs returns KD_ENOMEM, frees what it took, and serves a request that
  fits.
"""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("node_tuple", "left", "right", "dim")
KD_ETIMEOUT, KD_ENOMEM = -4, -2


def same(got, ref):
    assert got["m"] == ref["m"]
    for f in FIELDS:
        np.testing.assert_array_equal(np.asarray(got[f].cpu() if hasattr(got[f], "cpu") else got[f]), ref[f])


def test_device_wait_that_runs_out_reports_timeout_and_context_recovers(cuda_lib):
    import torch
    ctx = cuda_lib.kd_create(0, debug=8)
    try:
        # 300000 tuples: three scan chunks of 64 sort tiles, so two chunks wait on chunk 0
        x = torch.from_numpy(kdgen.cloud_gmm(300000, 3, 12)).cuda()
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.build_tree(ctx, x)
        assert e.value.code == KD_ETIMEOUT
        assert "wait" in str(e.value)
        ok = kdgen.cloud_gmm(300000, 3, 13)
        same(cuda_lib.build_tree(ctx, torch.from_numpy(ok).cuda()), oracle.build_tree(ok))
    finally:
        ctx.close()


def test_budget_exhaustion_reports_enomem_and_context_recovers(cuda_lib):
    import torch
    ctx = cuda_lib.kd_create(0, mem_budget_bytes=4 << 20)
    try:
        big = torch.from_numpy(kdgen.cloud_gmm(1 << 20, 3, 14)).cuda()
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.build_tree(ctx, big)
        assert e.value.code == KD_ENOMEM
        small = kdgen.cloud_gmm(2000, 3, 15)
        same(cuda_lib.build_tree(ctx, torch.from_numpy(small).cuda()), oracle.build_tree(small))
        # and again after a second refusal: nothing leaked from the first
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.build_tree(ctx, big)
        assert e.value.code == KD_ENOMEM
        same(cuda_lib.build_tree(ctx, torch.from_numpy(small).cuda()), oracle.build_tree(small))
    finally:
        ctx.close()
