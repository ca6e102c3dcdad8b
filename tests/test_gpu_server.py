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


def test_device_submitted_keys_overlap_on_the_gpu_and_equal_alone(pkg):
    """Continuous batching: 12 requests submitted as device tensors (kept on
    the device), 4 workers; the leaf-search kernels of at least two requests
    are resident at once (their device-time intervals intersect), and every
    result equals the same build alone."""
    import torch

    reqs = []
    for i in range(12):
        keys = inp.splitmix64_stream_torch(40_000 + i, 150_000 + 20_000 * i, device="cuda")
        reqs.append((keys, (48, 40)[i % 2]))
    alone = [pkg.shk_build(k, n, 2000).serialize() for k, n in reqs]
    srv = pkg.shk_server_create(0, 4)
    try:
        ids = [pkg.shk_server_submit(srv, k, n, 2000) for k, n in reqs]
        spans = []
        for i, rid in enumerate(ids):
            m, info = pkg.shk_server_wait(srv, rid)
            assert info["status"] == 0
            assert m.serialize() == alone[i]
            st = m.stats()
            assert st["leaf_t1_ns"] > st["leaf_t0_ns"] > 0
            spans.append((st["leaf_t0_ns"], st["leaf_t1_ns"]))
    finally:
        pkg.shk_server_destroy(srv)
    spans.sort()
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    assert overlaps >= 1, spans
    torch.cuda.synchronize()


def test_cancel_a_running_and_a_queued_request(pkg):
    """A running build stops at its next leaf-search work item and its request
    ends with SHK_ECANCELLED; a queued request never runs; a request
    submitted afterwards equals the same build alone."""
    import time

    big = inp.distinct_u64(3_000_000, 41)  # leaf 58: seconds of leaf search
    small = inp.distinct_u64(20000, 42)
    want = pkg.shk_build(small, 24, 1000).serialize()
    srv = pkg.shk_server_create(0, 1)
    try:
        r_big = pkg.shk_server_submit(srv, big, 58, 2000)
        r_q = pkg.shk_server_submit(srv, small, 24, 1000)
        t0 = time.time()
        while pkg.shk_server_get_stats(srv)["running"] == 0 and time.time() - t0 < 30:
            time.sleep(0.005)
        time.sleep(0.3)  # inside the leaf search
        pkg.shk_server_cancel(srv, r_q)
        pkg.shk_server_cancel(srv, r_big)
        m, info = pkg.shk_server_wait(srv, r_big)
        assert m is None and info["status"] == pkg.SHK_ECANCELLED
        assert (info["finish_ns"] - info["start_ns"]) / 1e9 < 5.0
        m, info = pkg.shk_server_wait(srv, r_q)
        assert m is None and info["status"] == pkg.SHK_ECANCELLED and info["start_ns"] == 0
        r_after = pkg.shk_server_submit(srv, small, 24, 1000)
        assert pkg.shk_server_wait(srv, r_after)[0].serialize() == want
    finally:
        pkg.shk_server_destroy(srv)


def test_deadline_stops_a_build_then_the_same_build_succeeds(pkg, orc):
    """A time budget far below the leaf search's time fails the build with
    SHK_ETIMEOUT (the leaf kernels see the deadline and return); the device
    stays usable and the same build without a budget equals the oracle."""
    keys = inp.distinct_u64(400_000, 43)
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_build(keys, 52, 2000, deadline_ms=2)
    assert e.value.status == pkg.SHK_ETIMEOUT
    small = inp.distinct_u64(5000, 44)
    assert pkg.shk_build(small, 20, 1000, deadline_ms=60_000).serialize() == orc.build_mphf(small, n=20, b=1000)


@pytest.mark.parametrize("kind,n,mode", [("u64", 48, 0), ("u64", 32, 1), ("str", 64, 1), ("u64", 16, 0)])
def test_footprint_estimate_covers_the_measured_peak(pkg, kind, n, mode):
    """The server's admission estimate is at least the device memory a build
    running alone holds at its peak (pool high watermark plus the result),
    and not more than four times it."""
    import torch

    for count in (20_000, 400_000):
        if kind == "u64":
            keys = inp.splitmix64_stream_torch(50_000 + count, count, device="cuda")
            kw = {}
        else:
            keys, offs = inp.ascii_strings_torch(count, 45, device="cuda")
            kw = {"kind": pkg.SHK_KEYS_STR, "str_offsets": offs}
        torch.cuda.synchronize()
        est = pkg.shk_build_footprint(keys, n, 2000, leaf_mode=mode, **kw)
        m = pkg.shk_build(keys, n, 2000, leaf_mode=mode, **kw)
        peak = m.stats()["device_bytes_peak"]
        m.close()
        assert 0 < peak <= est <= 4 * peak + (16 << 20), (count, peak, est)
