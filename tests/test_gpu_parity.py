"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Builds are compared byte for byte (seeds, Rice and Elias-Fano bits, shard
seeds, retrieval solution); queries rank for rank.  Small cases span many
buckets, several tree levels and ragged last leaves; the 10^6-key workload is
compared on sampled buckets and a sampled retrieval shard, plus the
bijection over all keys.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import shk_inputs as inp
from oracle.blobfmt import Blob

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


def _dev(keys):
    import torch

    return torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


def _golden_rows(name):
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _bijective(ranks_u64, N):
    return np.array_equal(np.sort(ranks_u64), np.arange(N, dtype=np.uint64))


CASES = [(10000, 32, 2000), (3000, 8, 100), (2500, 24, 500), (777, 40, 2000), (1500, 48, 2000),
         (1, 32, 2000), (2, 2, 2), (129, 16, 16), (4000, 2, 7), (63, 64, 64), (20000, 16, 300),
         (6000, 12, 4096)]


@pytest.mark.parametrize("N,n,b", CASES)
@pytest.mark.parametrize("sched", [0, 1, 2])
def test_build_bytes_equal_oracle(pkg, orc, N, n, b, sched):
    keys = inp.distinct_u64(N, 100 + N)
    m = pkg.shk_build(_dev(keys), n, b, sched=sched)
    got = m.serialize()
    want = orc.build_mphf(keys, n=n, b=b)
    assert got == want
    lo, hi = orc.fingerprints_u64(keys)
    ranks = m.query(_dev(keys)).cpu().numpy().view(np.uint64)
    assert np.array_equal(ranks, orc.query(want, lo, hi))
    assert _bijective(ranks, N)
    st = m.stats()
    assert st["n_keys"] == N and st["size_bits"] == 8 * len(got)
    m.close()


def test_one_launch_per_bucket_config(pkg, orc):
    """10,000 keys (stream seed 1), n = 32, b = 2000, one leaf launch per bucket."""
    keys = inp.distinct_u64(10000, 1)
    m = pkg.shk_build(_dev(keys), 32, 2000, sched=pkg.SHK_SCHED_PER_BUCKET)
    st = m.stats()
    assert st["leaf_launches"] == st["n_buckets"] == 5
    assert m.serialize() == orc.build_mphf(keys, n=32, b=2000)
    ranks = m.query(_dev(keys)).cpu().numpy().view(np.uint64)
    assert _bijective(ranks, 10000)


@pytest.mark.parametrize("U,passes", [(1, 1), (2, 3), (4, 16)])
def test_tuning_knobs_do_not_change_results(pkg, orc, U, passes):
    keys = inp.distinct_u64(8000, 7)
    m = pkg.shk_build(_dev(keys), 28, 900, seeds_per_lane=U, chunk_passes=passes)
    assert m.serialize() == orc.build_mphf(keys, n=28, b=900)


def test_host_keys_and_host_ranks(pkg, orc):
    keys = inp.distinct_u64(5000, 3)
    m = pkg.shk_build(keys, 20, 600)  # numpy host buffer
    assert m.serialize() == orc.build_mphf(keys, n=20, b=600)
    ranks = m.query(keys)  # host in, host out
    lo, hi = orc.fingerprints_u64(keys)
    assert np.array_equal(ranks, orc.query(m.serialize(), lo, hi))


def test_string_and_fp128_keys(pkg, orc):
    import torch

    data, offs = inp.ascii_strings(7000, 4)
    want = orc.build_mphf(kind=orc.KEYS_STR, str_data=data, str_offsets=offs, n=30, b=700)
    m = pkg.shk_build(torch.from_numpy(data).cuda(), 30, 700, kind=pkg.SHK_KEYS_STR,
                      str_offsets=torch.from_numpy(offs.view(np.int64)).cuda())
    assert m.serialize() == want
    m_host = pkg.shk_build(data, 30, 700, kind=pkg.SHK_KEYS_STR, str_offsets=offs)
    assert m_host.serialize() == want
    lo, hi = orc.fingerprints_str(data, offs)
    fp = np.stack([lo, hi], axis=1).copy()
    m2 = pkg.shk_build(_dev(fp.reshape(-1)), 30, 700, kind=pkg.SHK_KEYS_FP128)
    assert m2.serialize() == want
    r = m.query(torch.from_numpy(data).cuda(), kind=pkg.SHK_KEYS_STR,
                str_offsets=torch.from_numpy(offs.view(np.int64)).cuda())
    assert np.array_equal(r.cpu().numpy().view(np.uint64), orc.query(want, lo, hi))


@pytest.mark.parametrize("N", [30000, 180000])
def test_many_buckets(pkg, orc, N):
    """b = n = 2: 15,000 buckets (packed 16-bit shared-memory histogram) and
    90,000 buckets (global histogram); both radix passes."""
    keys = inp.distinct_u64(N, 600 + N)
    m = pkg.shk_build(_dev(keys), 2, 2)
    want = orc.build_mphf(keys, n=2, b=2)
    assert m.serialize() == want
    ranks = m.query(_dev(keys)).cpu().numpy().view(np.uint64)
    assert _bijective(ranks, N)


def test_long_and_many_strings(pkg, orc):
    """Strings of 8..160 bytes: many warps' bytes exceed the shared-memory
    staging buffer and are hashed from global memory; 15,000 buckets."""
    import torch

    data, offs = inp.ascii_strings(30000, 41, 8, 160)
    want = orc.build_mphf(kind=orc.KEYS_STR, str_data=data, str_offsets=offs, n=2, b=2)
    dd = torch.from_numpy(data).cuda()
    do = torch.from_numpy(offs.view(np.int64)).cuda()
    m = pkg.shk_build(dd, 2, 2, kind=pkg.SHK_KEYS_STR, str_offsets=do)
    assert m.serialize() == want
    lo, hi = orc.fingerprints_str(data, offs)
    r = m.query(dd, kind=pkg.SHK_KEYS_STR, str_offsets=do)
    assert np.array_equal(r.cpu().numpy().view(np.uint64), orc.query(want, lo, hi))


def test_oversized_bucket_is_rejected(pkg):
    """40,000 fingerprints in one bucket of 20,000 (b = 2): the packed
    histogram counter passes 2^15 and spills; the build reports the bucket
    above 8192 keys."""
    N = 40000
    fp = np.zeros((N, 2), np.uint64)
    fp[:, 0] = inp.distinct_u64(N, 77)
    fp[:, 1] = np.arange(N, dtype=np.uint64)  # hi < 2^64 / B: all in bucket 0
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_build(_dev(fp.reshape(-1)), 2, 2, kind=pkg.SHK_KEYS_FP128)
    assert e.value.status == pkg.SHK_EINVAL
    assert "8192" in str(e.value)


def test_empty_and_errors(pkg, orc):
    import torch

    m = pkg.shk_build(torch.zeros(0, dtype=torch.int64, device="cuda"), 32, 2000)
    assert m.serialize() == orc.build_mphf(np.zeros(0, np.uint64), n=32, b=2000)
    keys = inp.distinct_u64(3000, 5)
    keys[17] = keys[2500]
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_build(_dev(keys), 16, 100)
    assert e.value.status == pkg.SHK_EDUPKEY
    for n, b in [(1, 100), (65, 100), (32, 16), (32, 4097)]:
        with pytest.raises(pkg.ShkError) as e:
            pkg.shk_build(_dev(inp.distinct_u64(100, 1)), n, b)
        assert e.value.status == pkg.SHK_EINVAL
    # the library stays usable after errors
    k2 = inp.distinct_u64(500, 9)
    assert pkg.shk_build(_dev(k2), 16, 100).serialize() == orc.build_mphf(k2, n=16, b=100)


@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_tiny_builds_and_an_empty_shard_with_128bit_rows(pkg, orc, leaf_mode):
    """Leaf size 32 (128-bit retrieval rows): 1, 2, 3 and 33 keys, and a
    build whose middle bucket -- a shard of its own -- holds no key (128-bit
    fingerprints placed in buckets 0 and 2 of 3), equal the oracle's bytes
    and query to a bijection."""
    for N in (1, 2, 3, 33):
        keys = inp.distinct_u64(N, 800 + N)
        m = pkg.shk_build(_dev(keys), 32, 2000, leaf_mode=leaf_mode)
        want = orc.build_mphf(keys, n=32, b=2000, leaf_mode=leaf_mode)
        assert m.serialize() == want, N
        r = np.sort(m.query(_dev(keys)).cpu().numpy().view(np.uint64))
        assert np.array_equal(r, np.arange(N, dtype=np.uint64))
        m.close()
    # 65 keys, b = 32: B = 3 buckets; bucket = floor(hi * 3 / 2^64)
    lo = inp.splitmix64_stream(810, 65)
    u = inp.splitmix64_stream(811, 65) >> np.uint64(2)  # below 2^62
    third = np.uint64(2**64 // 3)
    hi = np.where(np.arange(65) < 33, u, u + np.uint64(2) * third)  # bucket 0 (hi < 2^62 < 2^64/3) or 2
    fp = np.stack([lo, hi], axis=1).copy().reshape(-1)
    m = pkg.shk_build(_dev(fp), 32, 32, kind=pkg.SHK_KEYS_FP128, shard_buckets=1, leaf_mode=leaf_mode)
    want = orc.build_mphf(kind=orc.KEYS_FP128, fp=fp, n=32, b=32, shard_buckets=1, leaf_mode=leaf_mode)
    assert m.serialize() == want
    assert np.array_equal(np.sort(m.query(_dev(fp), kind=pkg.SHK_KEYS_FP128).cpu().numpy().view(np.uint64)),
                          np.arange(65, dtype=np.uint64))
    m.close()


def test_deserialize_oracle_bytes(pkg, orc):
    keys = inp.distinct_u64(12000, 11)
    blob = orc.build_mphf(keys, n=36, b=1500)
    m = pkg.shk_deserialize(blob)
    assert m.serialize() == blob
    lo, hi = orc.fingerprints_u64(keys)
    ranks = m.query(_dev(keys)).cpu().numpy().view(np.uint64)
    assert np.array_equal(ranks, orc.query(blob, lo, hi))
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_deserialize(bytes(bad))
    assert e.value.status == pkg.SHK_EFORMAT
    with pytest.raises(pkg.ShkError):
        pkg.shk_deserialize(blob[:-8])


def _leaf_case(count, seed, lo_m, hi_m):
    keys, offs = inp.leaf_instances(count, seed, lo_m, hi_m)
    return keys, offs


@pytest.mark.parametrize("count,seed,lo_m,hi_m,start", [(3000, 3, 1, 40, 0), (500, 5, 2, 44, 12345),
                                                        (64, 6, 33, 33, 2**33), (40, 8, 45, 50, 0)])
def test_leaf_search_equals_oracle(pkg, orc, count, seed, lo_m, hi_m, start):
    import torch

    keys, offs = _leaf_case(count, seed, lo_m, hi_m)
    want_s, want_f = orc.leaf_search_batch(keys, offs, start)
    s, f = pkg.shk_leaf_search(_dev(keys), torch.from_numpy(offs.view(np.int32)).cuda(), start)
    assert np.array_equal(s.cpu().numpy().view(np.uint64), want_s)
    assert np.array_equal(f.cpu().numpy().view(np.uint64), want_f)


def test_leaf_search_largest_leaves(pkg, orc):
    """Leaves of 56..64 keys (seed searches of ~10^7 seeds each)."""
    import torch

    keys, offs = _leaf_case(12, 33, 56, 64)
    want_s, want_f = orc.leaf_search_batch(keys, offs, 0)
    s, f = pkg.shk_leaf_search(_dev(keys), torch.from_numpy(offs.view(np.int32)).cuda(), 0)
    assert np.array_equal(s.cpu().numpy().view(np.uint64), want_s)
    assert np.array_equal(f.cpu().numpy().view(np.uint64), want_f)


def test_leaf_search_rejects_bad_sizes(pkg):
    import torch

    keys = _dev(inp.splitmix64_stream(1, 200))
    off = torch.tensor([0, 10, 10, 20], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_leaf_search(keys, off)
    assert e.value.status == pkg.SHK_EINVAL
    off = torch.tensor([0, 65, 70], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_leaf_search(keys, off)
    assert e.value.status == pkg.SHK_EINVAL


def test_million_keys_leaf48_sampled(pkg, orc):
    """10^6 keys (stream seed 2), n = 48, b = 2000, persistent schedule:
    every key ranks bijectively; sampled buckets' codes and one retrieval
    shard equal the oracle's; the oracle's decoder reads the GPU bytes."""
    import torch

    N, n, b = 1_000_000, 48, 2000
    keys = inp.distinct_u64(N, 2)
    dk = _dev(keys)
    m = pkg.shk_build(dk, n, b)
    blob = m.serialize()
    ranks = m.query(dk)
    srt, _ = torch.sort(ranks)
    assert torch.equal(srt, torch.arange(N, device="cuda", dtype=torch.int64))
    bl = Blob(blob)
    assert bl.total_words == bl.nwords
    B = bl.h["B"]
    K = bl.K()
    O = bl.O()
    lo, hi = orc.fingerprints_u64(keys)
    bkt = (hi.astype(object) * B) >> 64
    bkt = np.array(bkt, dtype=np.int64)
    order = np.lexsort((lo, hi))
    assert np.array_equal(np.bincount(bkt, minlength=B), np.diff(K.astype(np.int64)))
    for i in (0, 1, 2, 3, 137, B - 1):
        sel = order[K[i]:K[i + 1]]
        seeds, ks, llo, lhi, f = orc.bucket_build(lo[sel], hi[sel], n)
        codes, end = bl.rice_codes(int(O[i]), [int(k) for k in ks])
        assert codes == [int(s) for s in seeds]
        assert end == O[i + 1]
    # retrieval shard 0 = buckets 0..5 (128-bit rows at leaf size 48)
    S = bl.h["shard_buckets"]
    assert S == 6 and bl.h["ribbon_width"] == 128
    parts = [orc.bucket_build(lo[order[K[j]:K[j + 1]]], hi[order[K[j]:K[j + 1]]], n) for j in range(S)]
    slo = np.concatenate([p[2] for p in parts])
    shi = np.concatenate([p[3] for p in parts])
    sf = np.concatenate([p[4] for p in parts])
    seed, sol = orc.ribbon_shard(slo, shi, sf, bl.h["eps_num"], 128)
    assert seed == bl.shard_seeds[0]
    got = [Blob.bit(bl.ribbon, p) for p in range(sol.size)]
    assert got == [int(v) for v in sol]
    samp = np.arange(0, N, 37)
    r_or = orc.query(blob, lo[samp], hi[samp])
    assert np.array_equal(r_or, ranks.cpu().numpy().view(np.uint64)[samp])
    m.close()


@pytest.mark.parametrize("ci", range(10))
def test_every_leaf_kernel_configuration_gives_the_same_build(pkg, orc, ci):
    cfgs = pkg.shk_leaf_configs()
    assert len(cfgs) == 10
    U, W, R = cfgs[ci]
    keys = inp.distinct_u64(6000, 77)
    want = orc.build_mphf(keys, n=28, b=700)
    for sched in (0, 1):
        m = pkg.shk_build(_dev(keys), 28, 700, seeds_per_lane=U, warps_per_block=W, key_unroll=R,
                          chunk_passes=3, sched=sched)
        assert m.stats()["leaf_cfg"] == [U, W, R, 3]
        assert m.serialize() == want


def test_autotuner_picks_a_supported_configuration(pkg):
    cfgs = pkg.shk_leaf_configs()
    for m in (8, 24, 40, 64):
        r = pkg.shk_leaf_tune(m)
        assert (r["seeds_per_lane"], r["warps_per_block"], r["key_unroll"]) in cfgs
        assert r["passes"] >= 1 and r["evals_per_s"] > 0
    keys = inp.distinct_u64(3000, 78)
    st = pkg.shk_build(_dev(keys), 40, 1000).stats()
    r = pkg.shk_leaf_tune(40)
    assert st["leaf_cfg"][:3] == [r["seeds_per_lane"], r["warps_per_block"], r["key_unroll"]]


def test_leaf_search_graph_replay_reads_new_contents(pkg, orc):
    import torch

    keys1, offs = inp.leaf_instances(700, 61, 2, 40)
    keys2 = inp.splitmix64_stream(62, keys1.size)
    dk = _dev(keys1)
    off = torch.from_numpy(offs.view(np.int32)).cuda()
    seeds = torch.empty(700, dtype=torch.int64, device="cuda")
    fm = torch.empty(700, dtype=torch.int64, device="cuda")
    r0 = pkg.shk_leaf_graph_replays()
    for keys in (keys1, keys2, keys1):
        dk.copy_(_dev(keys))
        pkg.shk_leaf_search(dk, off, 0, seeds_out=seeds, f_out=fm)
        want_s, want_f = orc.leaf_search_batch(keys, offs, 0)
        assert np.array_equal(seeds.cpu().numpy().view(np.uint64), want_s)
        assert np.array_equal(fm.cpu().numpy().view(np.uint64), want_f)
    assert pkg.shk_leaf_graph_replays() == r0 + 3


RF_CASES = [(10000, 32, 2000), (5000, 24, 800), (3000, 36, 1000), (4000, 48, 2000), (777, 40, 2000),
            (2, 2, 2), (129, 16, 16), (300, 40, 300), (2500, 8, 100)]


@pytest.mark.parametrize("N,n,b", RF_CASES)
@pytest.mark.parametrize("sched", [0, 1, 2])
def test_rotation_fitting_build_bytes_equal_oracle(pkg, orc, N, n, b, sched):
    """Leaf mode 1 (rotation fitting with partial hash calculation)."""
    keys = inp.distinct_u64(N, 400 + N)
    m = pkg.shk_build(_dev(keys), n, b, sched=sched, leaf_mode=pkg.SHK_LEAF_ROTATION)
    got = m.serialize()
    want = orc.build_mphf(keys, n=n, b=b, leaf_mode=1)
    assert got == want
    lo, hi = orc.fingerprints_u64(keys)
    ranks = m.query(_dev(keys)).cpu().numpy().view(np.uint64)
    assert np.array_equal(ranks, orc.query(want, lo, hi))
    assert _bijective(ranks, N)
    m2 = pkg.shk_deserialize(got)
    assert np.array_equal(m2.query(_dev(keys)).cpu().numpy().view(np.uint64), ranks)


def test_rotation_fitting_million_keys_sampled(pkg, orc):
    """10^6 keys, n = 48, rotation fitting: bijection over all keys and the
    codes of sampled buckets equal the oracle's."""
    import torch

    N, n, b = 1_000_000, 48, 2000
    keys = inp.distinct_u64(N, 2)
    dk = _dev(keys)
    m = pkg.shk_build(dk, n, b, leaf_mode=pkg.SHK_LEAF_ROTATION)
    blob = m.serialize()
    ranks = m.query(dk)
    srt, _ = torch.sort(ranks)
    assert torch.equal(srt, torch.arange(N, device="cuda", dtype=torch.int64))
    bl = Blob(blob)
    assert bl.h["leaf_mode"] == 1
    B = bl.h["B"]
    K, O = bl.K(), bl.O()
    lo, hi = orc.fingerprints_u64(keys)
    order = np.lexsort((lo, hi))
    for i in (0, 211, B - 1):
        sel = order[K[i]:K[i + 1]]
        seeds, ks, _, _, _ = orc.bucket_build(lo[sel], hi[sel], n, rf=True)
        codes, end = bl.rice_codes(int(O[i]), [int(k) for k in ks])
        assert codes == [int(s) for s in seeds] and end == O[i + 1]
    samp = np.arange(0, N, 101)
    assert np.array_equal(orc.query(blob, lo[samp], hi[samp]), ranks.cpu().numpy().view(np.uint64)[samp])


@pytest.mark.parametrize("S", [1, 8])
def test_shard_size_option(pkg, orc, S):
    """Shards of one bucket (2,000 keys) and of eight (about 16,000 keys: too
    large for precomputed rows in shared memory, so the retrieval kernel
    eliminates on one thread) equal the oracle's bytes."""
    keys = inp.distinct_u64(50000, 400 + S)
    m = pkg.shk_build(_dev(keys), 24, 2000, shard_buckets=S)
    assert m.serialize() == orc.build_mphf(keys, n=24, b=2000, shard_buckets=S)
    m.close()


@pytest.mark.parametrize("eps", [983, 655])
def test_retrieval_overhead_option(pkg, orc, eps):
    """Builds at eps = 1.5 % and 1 % (shard seeds retried more often) equal
    the oracle's bytes."""
    keys = inp.distinct_u64(40000, 300 + eps)
    for leaf_mode in (0, 1):
        m = pkg.shk_build(_dev(keys), 16, 2000, eps_num=eps, leaf_mode=leaf_mode)
        assert m.serialize() == orc.build_mphf(keys, n=16, b=2000, eps_num=eps, leaf_mode=leaf_mode)
        m.close()


@pytest.mark.parametrize("S,eps", [(1, 0), (16, 655), (0, 16), (0, 655)])
def test_128bit_retrieval_options(pkg, orc, S, eps):
    """128-bit retrieval rows (leaf size 32): shards of one bucket, shards of
    ~32,000 keys at eps = 1 %, and default shards at eps = 0.024 % and 1 %.
    The shards need different numbers of seeds, run on the persistent warps'
    speculative (shard, seed) items.  Every build equals the oracle's bytes."""
    keys = inp.distinct_u64(50000, 700 + S + eps)
    m = pkg.shk_build(_dev(keys), 32, 2000, shard_buckets=S, eps_num=eps, leaf_mode=1)
    assert m.serialize() == orc.build_mphf(keys, n=32, b=2000, shard_buckets=S, eps_num=eps, leaf_mode=1)
    m.close()


def test_string_keys_leaf64_rotation_fitting_sampled(pkg, orc):
    """The 10^8-string workload's parameters on 2 * 10^5 strings (lengths
    10..50, bytes 1..127, stream seed 4): n = 64, b = 2000, rotation fitting,
    eps = 1.5 %.  Every key ranks bijectively; bucket sizes, the split codes
    of a sampled bucket, its smallest leaf and its full leaf with the
    smallest value equal the oracle's; sampled ranks equal the oracle's
    decoding of the GPU bytes."""
    import torch

    N, n, b = 200_000, 64, 2000
    data, offs = inp.ascii_strings(N, 4)
    dd = torch.from_numpy(data).cuda()
    do = torch.from_numpy(offs.view(np.int64)).cuda()
    m = pkg.shk_build(dd, n, b, kind=pkg.SHK_KEYS_STR, str_offsets=do, leaf_mode=pkg.SHK_LEAF_ROTATION,
                      eps_num=983)
    blob = m.serialize()
    ranks = m.query(dd, kind=pkg.SHK_KEYS_STR, str_offsets=do)
    srt, _ = torch.sort(ranks)
    assert torch.equal(srt, torch.arange(N, device="cuda", dtype=torch.int64))
    bl = Blob(blob)
    assert bl.h["leaf_mode"] == 1 and bl.h["eps_num"] == 983
    B = bl.h["B"]
    K, O = bl.K(), bl.O()
    lo, hi = orc.fingerprints_str(data, offs)
    bkt = np.array((hi.astype(object) * B) >> 64, dtype=np.int64)
    assert np.array_equal(np.bincount(bkt, minlength=B), np.diff(K.astype(np.int64)))
    order = np.lexsort((lo, hi))
    i = 37
    sel = order[K[i]:K[i + 1]]
    seeds, ks, llo, _, loff, lm = orc.bucket_splits(lo[sel], hi[sel], n)
    codes, end = bl.rice_codes(int(O[i]), [int(k) for k in ks])
    assert end == O[i + 1]
    codes = np.array(codes, dtype=np.uint64)
    leaf = seeds == np.uint64(2**64 - 1)
    assert np.array_equal(codes[~leaf], seeds[~leaf])
    gpu_leaf = codes[leaf]
    short = int(np.argmin(lm))
    full = [j for j in range(lm.size) if lm[j] == n and j != short]
    pick = [short, min(full, key=lambda j: int(gpu_leaf[j]))]
    packed = np.concatenate([llo[loff[j]:loff[j] + lm[j]] for j in pick])
    po = np.array([0, lm[pick[0]], lm[pick[0]] + lm[pick[1]]], np.uint32)
    assert np.array_equal(orc.leaf_search_batch(packed, po, 0, rf=True)[0], gpu_leaf[pick])
    samp = np.arange(0, N, 53)
    assert np.array_equal(orc.query(blob, lo[samp], hi[samp]), ranks.cpu().numpy().view(np.uint64)[samp])
    m.close()


@pytest.mark.parametrize("count,seed,lo_m,hi_m", [(2000, 81, 1, 40), (12, 82, 56, 64), (300, 83, 33, 48)])
def test_rotation_fitting_leaf_search_equals_oracle(pkg, orc, count, seed, lo_m, hi_m):
    import torch

    keys, offs = inp.leaf_instances(count, seed, lo_m, hi_m)
    want_v, want_f = orc.leaf_search_batch(keys, offs, 0, rf=True)
    v, f = pkg.shk_leaf_search_rf(_dev(keys), torch.from_numpy(offs.view(np.int32)).cuda())
    assert np.array_equal(v.cpu().numpy().view(np.uint64), want_v)
    assert np.array_equal(f.cpu().numpy().view(np.uint64), want_f)


def test_first_queries_from_several_threads(pkg, orc):
    """The query index is built by the first query; four host threads querying
    one object at once all get the oracle's ranks."""
    import threading

    keys = inp.distinct_u64(60000, 515)
    m = pkg.shk_build(keys, 32, 2000)
    lo, hi = orc.fingerprints_u64(keys)
    want = orc.query(m.serialize(), lo, hi)
    out = [None] * 4

    def work(i):
        out[i] = m.query(keys)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for r in out:
        assert np.array_equal(r, want)
    m.close()


def test_pooled_working_memory_is_kept_and_released(pkg):
    """A build's working memory stays in the library's pool after the build
    (the next build does not map it again) and shk_release_memory returns it;
    results do not depend on either."""
    import torch

    d = _dev(inp.distinct_u64(4_000_000, 516))
    pkg.shk_release_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    m = pkg.shk_build(d, 48, 2000, leaf_mode=pkg.SHK_LEAF_ROTATION)
    want = m.serialize()
    m.close()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 < free0 - (100 << 20)
    pkg.shk_release_memory()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 > free1 + (100 << 20)
    assert pkg.shk_build(d, 48, 2000, leaf_mode=pkg.SHK_LEAF_ROTATION).serialize() == want


def _mask(bits):
    return int(sum(int(b) << k for k, b in enumerate(bits)))


@pytest.mark.parametrize("rf", [False, True])
def test_full_leaf_batch(pkg, orc, rf):
    """The whole 65,536-leaf batch (sizes 40..64, stream seed 3) in the launch
    the bench times: every leaf's value gives an orientable graph and its f
    mask is the oracle's canonical orientation; the 8 leaves with the smallest
    values and 8 leaves of at most 42 keys get the oracle's minimal values."""
    import torch

    keys, offs = inp.leaf_instances(65536, 3)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    doff = torch.from_numpy(offs.view(np.int32)).cuda()
    if rf:
        vals, fm = pkg.shk_leaf_search_rf(dk, doff)
    else:
        vals, fm = pkg.shk_leaf_search(dk, doff, 0)
    v = vals.cpu().numpy().view(np.uint64)
    f = fm.cpu().numpy().view(np.uint64)
    o = offs.astype(np.int64)
    for i in range(o.size - 1):
        x = keys[o[i]:o[i + 1]]
        want = orc.orient_mode(x, int(v[i]), rf)  # raises if the graph is not orientable
        assert _mask(want) == int(f[i]), i
    sizes = np.diff(o)
    pick = list(np.argsort(v)[:8]) + list(np.nonzero(sizes <= 42)[0][:8])
    packed = np.concatenate([keys[o[i]:o[i + 1]] for i in pick])
    po = np.zeros(len(pick) + 1, np.uint32)
    po[1:] = np.cumsum([sizes[i] for i in pick])
    assert np.array_equal(orc.leaf_search_batch(packed, po, 0, rf=rf)[0], v[pick])
    # 256 leaves drawn uniformly from the batch (all sizes 40..64): the oracle's
    # minimal values and masks, stored by tests/golden/make_goldens.py
    rows = _golden_rows("config3_leaf_sample.txt")
    assert len(rows) == 256
    for idx, m, seed, fmask, rv, rfm in rows:
        i = int(idx)
        assert sizes[i] == int(m)
        assert int(v[i]) == (int(rv) if rf else int(seed)), i
        assert int(f[i]) == int(rfm if rf else fmask, 16), i


@pytest.mark.parametrize("mode", [0, 1])
def test_million_keys_leaf48_full_bytes_equal_oracle(pkg, mode):
    """The 10^6-key, leaf-48, bucket-2000 workload in the launch the bench
    times: the SHA-256 of the GPU's serialized MPHF equals that of the
    oracle's full build (tests/golden/config2_build_digest.txt, written from
    oracle/ only), plain and rotation-fitting leaves."""
    import hashlib

    keys = inp.distinct_u64(1_000_000, 2)
    m = pkg.shk_build(_dev(keys), 48, 2000, leaf_mode=mode)
    blob = m.serialize()
    m.close()
    want = {int(r[0]): (int(r[1]), r[2]) for r in _golden_rows("config2_build_digest.txt")}
    assert len(blob) == want[mode][0]
    assert hashlib.sha256(blob).hexdigest() == want[mode][1]


def test_strings_1e8_leaf64_rotation_fitting_sampled(pkg, orc):
    """The workload the bench times: 10^8 strings (lengths 10..50, bytes
    1..127, stream seed 4), n = 64, b = 2000, rotation fitting, eps = 1.5 %,
    generated on the device.  Every key ranks bijectively; every bucket's size
    equals the oracle's; the split codes of 50 random buckets and the values of
    64 leaves drawn uniformly from them equal the oracle's (oracle/sampled.py)."""
    import torch

    from oracle.sampled import sampled_parity

    N = 100_000_000
    dd, do = inp.ascii_strings_torch(N, 4, device="cuda")
    m = pkg.shk_build(dd, 64, 2000, kind=pkg.SHK_KEYS_STR, str_offsets=do, leaf_mode=pkg.SHK_LEAF_ROTATION,
                      eps_num=983)
    blob = m.serialize()
    ranks = m.query(dd, kind=pkg.SHK_KEYS_STR, str_offsets=do)
    srt, _ = torch.sort(ranks)
    assert torch.equal(srt, torch.arange(N, device="cuda", dtype=torch.int64))
    del srt, ranks
    m.close()
    data = dd.cpu().numpy()
    offs = do.cpu().numpy().view(np.uint64)
    del dd, do
    lo, hi = orc.fingerprints_str(data, offs)
    r = sampled_parity(blob, lo, hi, 64, True, n_buckets=50, n_leaves=64, nthreads=os.cpu_count() or 1)
    assert r["ok"], r
    assert r["buckets"] == 50_000 and r["sampled_buckets"] == 50 and r["sampled_leaves"] == 64
