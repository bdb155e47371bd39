"""kd_presort_noalloc (GPU only): the presort of a small cloud with its
workspace in a static device array, called through the C ABI.

Its arrays and m must equal what kd_presort + kd_handle_arrays give for the
same cloud, on two calls in a row into the same caller buffers.  The file
is named to be collected last, so it also runs after every other GPU test
in the same process.
"""
import numpy as np
import pytest

import kdgen
import oracle

pytestmark = pytest.mark.gpu


def reference_arrays(api, ctx, coords_dev):
    h = api.kd_presort(ctx, coords_dev)
    try:
        return api.kd_handle_arrays(ctx, h), h.m
    finally:
        api.kd_release(ctx, h)


def clouds():
    yield "small int64 k=3 1% dups (n=16384, the limit)", kdgen.small_int64(seed=5)
    f = kdgen.cloud_gmm(5000, 5, 11)
    f[100:140] = f[2000:2040]  # exact duplicates
    f[7, 1] = -0.0
    f[8, :] = f[7, :]
    f[8, 1] = 0.0  # -0.0 and +0.0 compare equal: rows 7 and 8 are duplicates
    yield "f32 GMM k=5 with dups and signed zeros", f
    yield "int32 k=1 ragged", kdgen.cloud_int_uniform(777, 1, 6, 3, np.int32)
    yield "int64 k=8 narrow range", kdgen.cloud_int_uniform(3001, 8, 2, 4, np.int64)
    yield "unit cube k=2 one tuple", kdgen.cloud_unit_cube(1, 2, 6)


@pytest.mark.parametrize("case", range(5))
def test_noalloc_equals_kd_presort_two_calls(cuda_lib, case):
    import torch
    name, coords = list(clouds())[case]
    ctx = cuda_lib.kd_create(0)
    try:
        dev = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
        ref, m_ref = reference_arrays(cuda_lib, ctx, dev)
        # the existing entry point and the oracle agree on this cloud
        np.testing.assert_array_equal(ref, oracle.presort(coords), err_msg=name)
        n, k = coords.shape
        out = torch.full((k, n), -7, dtype=torch.int32, device="cuda")
        m_out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        for call in range(2):
            cuda_lib.kd_presort_noalloc(ctx, dev, out, m_out)
            torch.cuda.synchronize()
            m = int(m_out.item())
            assert m == m_ref, (name, call)
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got[:, :m], ref, err_msg=f"{name} call {call}")
            assert (got[:, m:] == -7).all(), f"{name} call {call}: entries past m were written"
            out.fill_(-7)
            m_out.fill_(-7)
    finally:
        ctx.close()


def test_noalloc_limits_and_errors(cuda_lib):
    import torch
    ctx = cuda_lib.kd_create(0)
    try:
        big = torch.zeros((cuda_lib._lib.KD_NOALLOC_MAX_N + 1, 3), dtype=torch.int64, device="cuda")
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.kd_presort_noalloc(ctx, big)
        assert e.value.code == -1 and "16384" in str(e.value)
        host = kdgen.small_int64(seed=2, n=100)
        with pytest.raises(cuda_lib.KdError) as e:
            cuda_lib.kd_presort_noalloc(ctx, host)
        assert e.value.code == -1
        bad = kdgen.cloud_gmm(300, 3, 5)
        bad[17, 2] = np.nan
        out = torch.full((3, 300), -7, dtype=torch.int32, device="cuda")
        out, m_out = cuda_lib.kd_presort_noalloc(ctx, torch.from_numpy(bad).cuda(), out)
        torch.cuda.synchronize()
        assert int(m_out.item()) == -6
        assert (out.cpu().numpy() == -7).all(), "a NaN must leave arrays_out untouched"
        # buffers the library cannot write safely are refused before the call
        okc = torch.from_numpy(kdgen.cloud_gmm(300, 3, 6)).cuda()
        for bad_out in (torch.empty((3, 299), dtype=torch.int32, device="cuda"),
                        torch.empty((3, 300), dtype=torch.int64, device="cuda"),
                        torch.empty((300, 3), dtype=torch.int32, device="cuda").t(),
                        torch.empty((3, 300), dtype=torch.int32)):
            with pytest.raises(ValueError):
                cuda_lib.kd_presort_noalloc(ctx, okc, bad_out)
        with pytest.raises(ValueError):
            cuda_lib.kd_presort_noalloc(ctx, okc, None, torch.empty(1, dtype=torch.int64, device="cuda"))
        # the context and the workspace stay usable after the NaN report
        ok = torch.from_numpy(kdgen.cloud_gmm(300, 3, 6)).cuda()
        ref, m_ref = reference_arrays(cuda_lib, ctx, ok)
        out, m_out = cuda_lib.kd_presort_noalloc(ctx, ok)
        torch.cuda.synchronize()
        assert int(m_out.item()) == m_ref
        np.testing.assert_array_equal(out[:, :m_ref].cpu().numpy(), ref)
        empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
        out, m_out = cuda_lib.kd_presort_noalloc(ctx, empty)
        torch.cuda.synchronize()
        assert int(m_out.item()) == 0
    finally:
        ctx.close()
