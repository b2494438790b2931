"""The allocation-free sort entry point (for callers that cannot allocate
device memory, e.g. under a framework allocator that owns the budget or on a
latency-critical path): two calls in a row through the C ABI must give the
same permutation as the context-based sph_sort_keys, and sizes beyond the
static scratch are rejected.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _keys(n, seed):
    rng = np.random.default_rng(seed)
    pool = rng.integers(0, 1 << 62, size=n // 3 + 1, dtype=np.int64).astype(np.uint64) | np.uint64(1 << 63)
    keys = pool[rng.integers(0, pool.size, size=n)]          # short runs of equal keys
    ids = rng.permutation(n).astype(np.uint32)
    return (torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(ids.view(np.int32)).cuda())


def test_noalloc_sort_matches_context_sort_twice():
    B = need_gpu()
    ctx = B.Context({}, B.SPH_SORT_NOALLOC_MAX)
    for n, seed in ((200_003, 1), (B.SPH_SORT_NOALLOC_MAX, 2)):
        k, i = _keys(n, seed)
        ref = B.sph_sort_keys(ctx, k, i)
        got = B.sph_sort_keys_noalloc(k, i)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    ctx.close()


def test_noalloc_sort_rejects_oversize():
    B = need_gpu()
    n = B.SPH_SORT_NOALLOC_MAX + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = B.load().sph_sort_keys_noalloc(n, k.data_ptr(), None, k.data_ptr(), None)
    assert st == B.SPH_ERR_CAPACITY
