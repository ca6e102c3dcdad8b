"""The leaf search entry point that allocates nothing.

Callers whose device memory is owned by another memory manager, or serving
loops with a fixed memory budget, cannot call cudaMalloc while they run; for
them shk_leaf_search_noalloc takes its working memory from a fixed array in
the library.  This test calls it through the C ABI, twice in a row per case
(the array keeps the previous call's contents), compares every seed and
orientation mask with the CPU oracle, checks that the calls leave the device's
free memory unchanged, and checks its error path (a leaf above 64 keys) and
that a good call after a failed one is correct.  It lives in its own file,
collected last, and passes alone or after the other tests.
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


CASES = [(3000, 51, 1, 44, 0), (777, 52, 30, 46, 999)]


@pytest.fixture(scope="module")
def expected(orc):
    """Oracle seeds and orientation masks of every case."""
    out = []
    for count, seed, lo_m, hi_m, start in CASES:
        keys, offs = inp.leaf_instances(count, seed, lo_m, hi_m)
        out.append((keys, offs, start) + orc.leaf_search_batch(keys, offs, start))
    return out


def _dev(keys, offs):
    import torch

    return (torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(offs.view(np.int32)).cuda())


def test_noalloc_equals_oracle_twice_in_a_row_and_allocates_nothing(pkg, expected):
    import torch

    dev = [(_dev(k, o), start, s, f) for k, o, start, s, f in expected]
    outs = [(torch.empty(len(s), dtype=torch.int64, device="cuda"),
             torch.empty(len(s), dtype=torch.int64, device="cuda")) for _, _, s, _ in dev]
    # the first call on a device may still load the library's module (which
    # holds the fixed array); after it, no call may change the free memory
    (k0, o0), st0, _, _ = dev[0]
    pkg.shk_leaf_search_noalloc(k0, o0, outs[0][0], outs[0][1], seed_start=st0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rep in range(2):
        for ((k, o), start, want_s, want_f), (seeds, fm) in zip(dev, outs):
            seeds.fill_(-7)
            fm.fill_(-7)
            pkg.shk_leaf_search_noalloc(k, o, seeds, fm, seed_start=start)
            assert np.array_equal(seeds.cpu().numpy().view(np.uint64), want_s), rep
            assert np.array_equal(fm.cpu().numpy().view(np.uint64), want_f), rep
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_without_orientation_output(pkg, expected):
    import torch

    keys, offs, start, want_s, _ = expected[1]
    k, o = _dev(keys, offs)
    seeds = torch.empty(len(want_s), dtype=torch.int64, device="cuda")
    _, f = pkg.shk_leaf_search_noalloc(k, o, seeds, None, seed_start=start)
    assert f is None
    assert np.array_equal(seeds.cpu().numpy().view(np.uint64), want_s)


def test_noalloc_leaf_too_large_then_good_call(pkg, expected):
    """A leaf of 65 keys is reported through the shared device error flag as
    SHK_EINVAL; the next call clears that flag and is correct."""
    import torch

    bad_off = torch.tensor([0, 10, 75, 80], dtype=torch.int32, device="cuda")
    bad_keys = torch.from_numpy(inp.splitmix64_stream(53, 80).view(np.int64)).cuda()
    seeds = torch.empty(3, dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_leaf_search_noalloc(bad_keys, bad_off, seeds)
    assert e.value.status == pkg.SHK_EINVAL
    keys, offs, start, want_s, want_f = expected[1]
    k, o = _dev(keys, offs)
    s2 = torch.empty(len(want_s), dtype=torch.int64, device="cuda")
    f2 = torch.empty(len(want_s), dtype=torch.int64, device="cuda")
    pkg.shk_leaf_search_noalloc(k, o, s2, f2, seed_start=start)
    assert np.array_equal(s2.cpu().numpy().view(np.uint64), want_s)
    assert np.array_equal(f2.cpu().numpy().view(np.uint64), want_f)


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
