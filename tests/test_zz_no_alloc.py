"""The allocation-free sort entry point, for callers that cannot allocate
device memory (code under a framework whose caching allocator owns the device
budget, plugins whose host forbids allocation, latency-critical paths that
cannot risk cudaMalloc synchronising the device).  Through the C ABI, calls
in a row must give the permutation of the context-based sph_sort_keys and of
the oracle's (key, id) sort, on the default and on a side stream, with and
without ids, without changing the device's free memory; sizes beyond the
static scratch, runs of more than 64 equal keys and pointers that are not
device memory of the current device are rejected with their own messages.
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _keys(n, seed):
    rng = np.random.default_rng(seed)
    pool = rng.integers(0, 1 << 62, size=n // 3 + 1, dtype=np.int64).astype(np.uint64) | np.uint64(1 << 63)
    keys = pool[rng.integers(0, pool.size, size=n)]          # short runs of equal keys
    ids = rng.permutation(n).astype(np.uint32)
    return keys, ids


def _dev(keys, ids):
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    i = None if ids is None else torch.from_numpy(ids.view(np.int32)).cuda()
    return k, i


def test_noalloc_sort_matches_context_sort_and_oracle_twice():
    B = need_gpu()
    ctx = B.Context({}, B.SPH_SORT_NOALLOC_MAX)
    for n, seed in ((200_003, 1), (B.SPH_SORT_NOALLOC_MAX, 2), (1, 3), (777, 4)):
        keys, ids = _keys(n, seed)
        k, i = _dev(keys, ids)
        ref = B.sph_sort_keys(ctx, k, i)
        got = B.sph_sort_keys_noalloc(k, i)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        want = oracle.sort_perm(keys, ids)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want)
    ctx.close()


def test_noalloc_sort_without_ids_keeps_index_order():
    B = need_gpu()
    ctx = B.Context({}, B.SPH_SORT_NOALLOC_MAX)
    keys, _ = _keys(100_001, 5)
    k, _ = _dev(keys, None)
    ref = B.sph_sort_keys(ctx, k, None)
    for _ in range(2):
        got = B.sph_sort_keys_noalloc(k, None)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    idx = np.arange(keys.size, dtype=np.uint32)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), oracle.sort_perm(keys, idx))
    ctx.close()


def test_noalloc_sort_on_a_side_stream():
    B = need_gpu()
    keys, ids = _keys(150_000, 6)
    k, i = _dev(keys, ids)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        got = B.sph_sort_keys_noalloc(k, i, stream=side)
    side.synchronize()
    assert np.array_equal(got.cpu().numpy().view(np.uint32), oracle.sort_perm(keys, ids))


def test_noalloc_sort_leaves_free_memory_unchanged():
    B = need_gpu()
    keys, ids = _keys(B.SPH_SORT_NOALLOC_MAX, 7)
    k, i = _dev(keys, ids)
    perm = torch.empty(keys.size, dtype=torch.int32, device="cuda")
    B.sph_sort_keys_noalloc(k, i, perm=perm)                 # the device's first call loads the code
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st = B.load().sph_sort_keys_noalloc(keys.size, k.data_ptr(), i.data_ptr(), perm.data_ptr(), None)
        assert st == B.SPH_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), oracle.sort_perm(keys, ids))


def test_noalloc_sort_rejects_oversize_and_long_tie_runs():
    B = need_gpu()
    n = B.SPH_SORT_NOALLOC_MAX + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = B.load().sph_sort_keys_noalloc(n, k.data_ptr(), None, k.data_ptr(), None)
    assert st == B.SPH_ERR_CAPACITY
    assert b"exceeds the static scratch" in B.load().sph_last_error(None)
    # 65 equal keys: more than the tie ordering handles
    keys = np.full(65, np.uint64(1 << 63) | np.uint64(12345), dtype=np.uint64)
    kk, ii = _dev(keys, np.arange(65, dtype=np.uint32)[::-1].copy())
    with pytest.raises(B.SphError) as e:
        B.sph_sort_keys_noalloc(kk, ii)
    assert e.value.code == B.SPH_ERR_CAPACITY and "64 equal keys" in str(e.value)
    # the scratch keeps no error: the next call succeeds
    keys2, ids2 = _keys(64, 8)
    k2, i2 = _dev(keys2, ids2)
    got = B.sph_sort_keys_noalloc(k2, i2)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), oracle.sort_perm(keys2, ids2))


def test_noalloc_sort_rejects_host_pointers():
    B = need_gpu()
    host = np.zeros(16, dtype=np.uint64)
    dev = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = B.load().sph_sort_keys_noalloc(16, host.ctypes.data, None, dev.data_ptr(), None)
    assert st == B.SPH_ERR_ARG
    assert b"keys" in B.load().sph_last_error(None)
