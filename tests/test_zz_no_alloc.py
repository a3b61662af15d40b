"""The allocation-free sort entry point, for callers that cannot allocate device memory (an
application that owns every free byte of the GPU in its own pool, or a latency-critical stream that
must not meet the device-wide synchronisation cudaMalloc/cudaFree can bring).

It must give exactly what the workspace-taking sort gives, on consecutive calls that reuse the
library's one fixed scratch array, and refuse sizes beyond that array. This file is collected last,
so a run that stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

from paper_2310_03596_gb300 import gsph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return gsph.load()


def _pair(rng, n, bits):
    import torch
    k = rng.integers(0, 2 ** bits, size=n, dtype=np.uint64).astype(np.uint32)
    k[: n // 4] = np.sort(k[: n // 4])          # a sorted run and a run of equal keys
    k[n // 2: n // 2 + min(300, n // 4)] = 5
    keys = torch.from_numpy(k.view(np.int32)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    return keys, vals


def test_noalloc_sort_equals_workspace_sort_on_consecutive_calls(lib):
    import torch
    rng = np.random.default_rng(123)
    # two calls in a row per case: the second runs on whatever the first left in the shared array
    for n, bits in [(gsph.SORT_NOALLOC_MAX_N, 27), (70_001, 17), (4097, 9), (1, 32), (gsph.SORT_NOALLOC_MAX_N, 8)]:
        for _ in range(2):
            keys, vals = _pair(rng, n, bits)
            k2, v2 = keys.clone(), vals.clone()
            gsph.radix_sort_pairs(keys, vals, bits)
            gsph.radix_sort_pairs_noalloc(k2, v2, bits)
            torch.cuda.synchronize()
            assert torch.equal(keys, k2) and torch.equal(vals, v2), (n, bits)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch(lib):
    import torch
    n = gsph.SORT_NOALLOC_MAX_N + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    vals = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert lib.gsph_radix_sort_pairs_noalloc(keys.data_ptr(), vals.data_ptr(), n, 20, None) == gsph.INVALID_ARG
    assert lib.gsph_radix_sort_pairs_noalloc(None, None, 5, 20, None) == gsph.INVALID_ARG
    assert lib.gsph_radix_sort_pairs_noalloc(None, None, 0, 20, None) == gsph.OK
