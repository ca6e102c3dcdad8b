"""The leaf search entry point that allocates nothing.

Callers whose device memory is owned by another memory manager, or serving
loops with a fixed memory budget, cannot call cudaMalloc while they run; for
them shk_leaf_search_noalloc takes its working memory from a fixed array in
the library.  This test calls it through the C ABI twice in a row (the array
keeps the previous call's contents) and compares each result, bit for bit,
with the allocating shk_leaf_search on the same input.  It lives in its own
file, collected last, and passes alone or after the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest

import shk_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    from paper_2308_09561_gb300 import build_ext

    build_ext.build()
    import paper_2308_09561_gb300 as p

    p.load_library()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return p


def _case(count, seed, lo_m, hi_m):
    import torch

    keys, offs = inp.leaf_instances(count, seed, lo_m, hi_m)
    return (torch.from_numpy(keys.view(np.int64)).cuda(),
            torch.from_numpy(offs.view(np.int32)).cuda())


def test_noalloc_matches_allocating_entry_point_twice(pkg):
    import torch

    for count, seed, lo_m, hi_m, start in [(3000, 51, 1, 44, 0), (777, 52, 30, 46, 999)]:
        keys, off = _case(count, seed, lo_m, hi_m)
        want_s, want_f = pkg.shk_leaf_search(keys, off, start)
        seeds = torch.empty(count, dtype=torch.int64, device="cuda")
        fm = torch.empty(count, dtype=torch.int64, device="cuda")
        pkg.shk_leaf_search_noalloc(keys, off, seeds, fm, seed_start=start)
        assert torch.equal(seeds, want_s)
        assert torch.equal(fm, want_f)


def test_noalloc_rejects_batches_above_its_limit(pkg):
    import torch

    n = 65537
    off = torch.arange(n + 1, dtype=torch.int32, device="cuda") * 2
    keys = torch.zeros(2 * n, dtype=torch.int64, device="cuda")
    seeds = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_leaf_search_noalloc(keys, off, seeds)
    assert e.value.status == pkg.SHK_EINVAL
    assert "65536" in str(e.value)
