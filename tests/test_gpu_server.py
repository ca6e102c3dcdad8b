"""Serving: builds of different sizes submitted to one server (concurrent
builds on several streams, admission by device footprint) give exactly the
MPHF that the same build gives alone."""
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


def _requests(count, seed):
    u = inp.uniform01(seed, 3 * count)
    reqs = []
    for i in range(count):
        n_keys = int(10 ** (3 + 1.7 * u[3 * i]))  # log-uniform in [1e3, 5e4]
        n = (16, 24, 32)[int(u[3 * i + 1] * 3)]
        b = (500, 2000)[int(u[3 * i + 2] * 2)]
        reqs.append((inp.distinct_u64(n_keys, 10_000 + 7 * i), n, b))
    return reqs


def test_results_alone_equal_results_in_the_mix(pkg, orc):
    reqs = _requests(24, 5)
    alone = [pkg.shk_build(k, n, b).serialize() for k, n, b in reqs]
    srv = pkg.shk_server_create(0, 4)
    try:
        ids = [pkg.shk_server_submit(srv, k, n, b) for k, n, b in reqs]
        for i, rid in enumerate(ids):
            m, info = pkg.shk_server_wait(srv, rid)
            assert info["done"] == 1 and info["status"] == 0
            assert info["finish_ns"] >= info["start_ns"] >= info["submit_ns"]
            assert m.serialize() == alone[i]
        st = pkg.shk_server_get_stats(srv)
        assert st["submitted"] == st["completed"] == 24 and st["queued"] == st["running"] == 0
    finally:
        pkg.shk_server_destroy(srv)
    for i in (0, 7, 13):
        k, n, b = reqs[i]
        assert alone[i] == orc.build_mphf(k, n=n, b=b)


def test_admission_respects_the_device_budget(pkg):
    reqs = _requests(12, 6)
    srv = pkg.shk_server_create(24 << 20, 4)  # 24 MB: about two requests at a time
    try:
        ids = [pkg.shk_server_submit(srv, k, n, b) for k, n, b in reqs]
        infos = [pkg.shk_server_wait(srv, rid)[1] for rid in ids]
        st = pkg.shk_server_get_stats(srv)
        biggest = max(i["footprint_bytes"] for i in infos)
        assert st["peak_in_use_bytes"] <= max(st["budget_bytes"], biggest)
        assert all(i["status"] == 0 for i in infos)
    finally:
        pkg.shk_server_destroy(srv)


def test_a_failing_request_does_not_disturb_the_others(pkg):
    import torch

    good = inp.distinct_u64(20000, 31)
    bad = inp.distinct_u64(5000, 32)
    bad[10] = bad[20]
    want = pkg.shk_build(good, 24, 1000).serialize()
    srv = pkg.shk_server_create(0, 2)
    try:
        r_bad = pkg.shk_server_submit(srv, bad, 24, 1000)
        r_dev = pkg.shk_server_submit(srv, torch.from_numpy(good.view(np.int64)).cuda(), 24, 1000)
        r_host = pkg.shk_server_submit(srv, good, 24, 1000)
        m, info = pkg.shk_server_wait(srv, r_bad)
        assert m is None and info["status"] == pkg.SHK_EDUPKEY
        assert pkg.shk_server_wait(srv, r_dev)[0].serialize() == want
        m, info = None, None
        while m is None:
            m, info = pkg.shk_server_poll(srv, r_host)
        assert m.serialize() == want
        with pytest.raises(pkg.ShkError):
            pkg.shk_server_poll(srv, r_host)  # already collected
    finally:
        pkg.shk_server_destroy(srv)


def test_concurrent_builds_with_different_shared_memory_needs(pkg):
    """Builds whose kernels need different dynamic shared memory (bucket
    counts from 5 to 4000, bucket sizes 50 to 4096) run concurrently on 8
    workers and each equals the same build alone."""
    u = inp.uniform01(8, 64)
    reqs = []
    for i in range(32):
        n_keys = int(2e4 * 10 ** u[2 * i])  # 2e4 .. 2e5
        b = (50, 300, 1000, 4096)[int(u[2 * i + 1] * 4)]
        reqs.append((inp.distinct_u64(n_keys, 20_000 + i), 16, b))
    alone = [pkg.shk_build(k, n, b).serialize() for k, n, b in reqs]
    srv = pkg.shk_server_create(0, 8)
    try:
        ids = [pkg.shk_server_submit(srv, k, n, b) for k, n, b in reqs]
        for i, rid in enumerate(ids):
            m, info = pkg.shk_server_wait(srv, rid)
            assert info["status"] == 0
            assert m.serialize() == alone[i]
    finally:
        pkg.shk_server_destroy(srv)


def test_several_threads_waiting_on_one_request(pkg):
    """Four threads wait on the same request: exactly one collects the MPHF,
    the others learn that the id is no longer known."""
    import threading

    keys = inp.distinct_u64(200000, 33)
    want = pkg.shk_build(keys, 32, 2000).serialize()
    srv = pkg.shk_server_create(0, 1)
    got, errors = [], []

    def waiter(rid):
        try:
            got.append(pkg.shk_server_wait(srv, rid)[0].serialize())
        except pkg.ShkError as e:
            errors.append(e.status)

    try:
        rid = pkg.shk_server_submit(srv, keys, 32, 2000)
        ts = [threading.Thread(target=waiter, args=(rid,)) for _ in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert got == [want]
        assert errors == [pkg.SHK_EINVAL] * 3
    finally:
        pkg.shk_server_destroy(srv)
