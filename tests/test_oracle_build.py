"""Whole-build pins of the oracle: bijection (the MPHF definition, Sec. 1),
the encoded format read back by an independent reader, and edge cases."""
from __future__ import annotations

import math

import numpy as np
import pytest

import shk_inputs as inp
from oracle.blobfmt import Blob


def _check_bijection(orc, blob, lo, hi):
    r = orc.query(blob, lo, hi)
    assert np.array_equal(np.sort(r), np.arange(lo.size, dtype=np.uint64))
    return r


@pytest.mark.parametrize("N,n,b", [(10000, 32, 2000), (3000, 8, 100), (2500, 24, 500),
                                   (777, 40, 2000), (1500, 48, 2000), (1, 32, 2000),
                                   (2, 2, 2), (63, 64, 64), (129, 16, 16), (4000, 2, 7)])
def test_build_is_bijection(orc, N, n, b):
    keys = inp.distinct_u64(N, 100 + N)
    blob = orc.build_mphf(keys, n=n, b=b)
    lo, hi = orc.fingerprints_u64(keys)
    _check_bijection(orc, blob, lo, hi)


def test_empty_build(orc):
    blob = orc.build_mphf(np.zeros(0, np.uint64), n=32, b=2000)
    bl = Blob(blob)
    assert bl.h["N"] == 0 and bl.h["B"] == 0
    assert orc.query(blob, np.zeros(0, np.uint64), np.zeros(0, np.uint64)).size == 0


def test_string_keys_and_fp128_agree(orc):
    data, offs = inp.ascii_strings(5000, 4)
    blob = orc.build_mphf(kind=orc.KEYS_STR, str_data=data, str_offsets=offs, n=32, b=500)
    lo, hi = orc.fingerprints_str(data, offs)
    _check_bijection(orc, blob, lo, hi)
    fp = np.stack([lo, hi], axis=1)
    blob2 = orc.build_mphf(kind=orc.KEYS_FP128, fp=fp, n=32, b=500)
    assert blob == blob2
    assert data.min() >= 1 and data.max() <= 127
    lens = np.diff(offs.astype(np.int64))
    assert lens.min() >= 10 and lens.max() <= 50


def test_key_order_does_not_matter(orc):
    keys = inp.distinct_u64(6000, 3)
    a = orc.build_mphf(keys, n=24, b=1000)
    b = orc.build_mphf(keys[::-1].copy(), n=24, b=1000)
    assert a == b


def test_duplicates_and_bad_args(orc):
    keys = inp.distinct_u64(1000, 5)
    keys[10] = keys[500]
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, n=16, b=100)
    assert e.value.status == orc.EDUPKEY
    for n, b in [(1, 100), (65, 100), (32, 16), (32, 4097)]:
        with pytest.raises(orc.OracleError) as e:
            orc.build_mphf(inp.distinct_u64(100, 1), n=n, b=b)
        assert e.value.status == orc.EINVAL


def test_format_sections_decode(orc):
    """The Rice stream, both Elias-Fano sequences and the shard seeds read back
    by an independent reader equal what the oracle computes bucket by bucket."""
    N, n, b = 6000, 24, 700
    keys = inp.distinct_u64(N, 9)
    blob = orc.build_mphf(keys, n=n, b=b)
    bl = Blob(blob)
    h = bl.h
    assert h["magic"] == orc.MAGIC and h["N"] == N and h["n"] == n and h["b"] == b
    B = h["B"]
    assert B == math.ceil(N / b)
    assert bl.total_words == bl.nwords
    lo, hi = orc.fingerprints_u64(keys)
    bkt = np.array([orc.bucket_of(int(v), B) for v in hi])
    K = np.zeros(B + 1, np.uint64)
    np.cumsum(np.bincount(bkt, minlength=B), out=K[1:])
    assert np.array_equal(bl.K(), K)
    # Elias-Fano lower-bit width: floor(log2(U / (B+1)))
    q = int(K[-1]) // (B + 1)
    assert h["efK_l"] == (q.bit_length() - 1 if q else 0)
    assert h["efK_hi_bits"] == (int(K[-1]) >> h["efK_l"]) + B + 1
    O = bl.O()
    assert O[0] == 0 and O[-1] == h["rice_bits"]
    # the same Elias-Fano parameters for the Rice bit offsets; with
    # l = floor(log2(U / (B + 1))) the high parts take fewer than 3 (B + 1)
    # bits, so a sequence takes fewer than (B + 1)(l + 3) bits
    qo = int(O[-1]) // (B + 1)
    assert h["efO_l"] == (qo.bit_length() - 1 if qo else 0)
    assert h["efO_hi_bits"] == (int(O[-1]) >> h["efO_l"]) + B + 1
    for l_name, hi_name in (("efK_l", "efK_hi_bits"), ("efO_l", "efO_hi_bits")):
        assert (B + 1) * h[l_name] + h[hi_name] < (B + 1) * (h[l_name] + 3)
    assert np.all(np.diff(O.astype(np.int64)) >= 0)
    order = np.lexsort((lo, hi))
    for i in range(B):
        sel = order[K[i]:K[i + 1]]
        seeds, ks, _, _, _ = orc.bucket_build(lo[sel], hi[sel], n)
        codes, end = bl.rice_codes(int(O[i]), [int(k) for k in ks])
        assert codes == [int(s) for s in seeds]
        assert end == O[i + 1]
        # code length = k + 1 + (s >> k)
        assert end - O[i] == sum(int(k) + 1 + (int(s) >> int(k)) for s, k in zip(seeds, ks))
    # retrieval: shard slot counts add up
    S = h["shard_buckets"]
    slots = sum(orc.shard_slots(int(K[min(B, s * S + S)] - K[s * S]), h["eps_num"])
                for s in range(h["num_shards"]))
    assert h["ribbon_bits"] == slots


def test_every_key_retrieves_its_orientation(orc):
    """Sec. 2 Retrieval: the structure returns the stored f for every key;
    the rank uses h_{s,f(x)}(x) of its leaf (Sec. 4)."""
    N, n, b = 4000, 16, 400
    keys = inp.distinct_u64(N, 21)
    blob = orc.build_mphf(keys, n=n, b=b)
    lo, hi = orc.fingerprints_u64(keys)
    bl = Blob(blob)
    B, S = bl.h["B"], bl.h["shard_buckets"]
    K = bl.K()
    order = np.lexsort((lo, hi))
    ranks = orc.query(blob, lo, hi)
    for i in range(B):
        sel = order[K[i]:K[i + 1]]
        seeds, ks, llo, lhi, f = orc.bucket_build(lo[sel], hi[sel], n)
        # walk leaves in order and recompute each key's rank from f
        pos = 0
        leaf_sizes = _leaf_sizes(orc, int(K[i + 1] - K[i]), n)
        leaf_codes = [s for s, k in zip(seeds, ks)]
        # map keys to their ranks via lookup of (lo, hi)
        lookup = {(int(a), int(c)): int(r) for a, c, r in zip(lo[sel], hi[sel], ranks[sel])}
        for m in leaf_sizes:
            for j in range(m):
                r = lookup[(int(llo[pos + j]), int(lhi[pos + j]))]
                assert K[i] + pos <= r < K[i] + pos + m
            pos += m
        assert pos == K[i + 1] - K[i]
        del leaf_codes


def _leaf_sizes(orc, m, n):
    sh = orc.split_shape(m, n)
    if sh is None:
        return [m] if m else []
    unit, fan = sh
    out = []
    for j in range(fan):
        out += _leaf_sizes(orc, unit if j < fan - 1 else m - (fan - 1) * unit, n)
    return out


def test_bucket_occupancy_chi_square(orc):
    """Buckets ~ Binomial(N, 1/B): chi-square of occupancy (fingerprint sanity)."""
    N, B = 200000, 400
    keys = inp.distinct_u64(N, 31)
    _, hi = orc.fingerprints_u64(keys)
    occ = np.bincount(np.array([orc.bucket_of(int(v), B) for v in hi[:N]]), minlength=B)
    exp = N / B
    chi2 = float(((occ - exp) ** 2 / exp).sum())
    # mean B-1 = 399, sd sqrt(2*399) ~ 28
    assert abs(chi2 - (B - 1)) < 5 * math.sqrt(2 * (B - 1))


def test_bits_per_key_breakdown(orc):
    N, n, b = 20000, 32, 2000
    keys = inp.distinct_u64(N, 1)
    blob = orc.build_mphf(keys, n=n, b=b)
    bl = Blob(blob)
    h = bl.h
    total = 64 * bl.nwords
    parts = (64 * 16 + 64 * sum(v[1] for v in bl.sections.values()))
    assert parts == total
    # retrieval ~ (1 + eps) bits/key, seeds ~ log2(nn/n!)/n - 1 + overhead
    assert 1.0 < h["ribbon_bits"] / N < 1.1
    leaf_bits = h["rice_bits"] / N
    lower = (n * math.log2(n) - math.lgamma(n + 1) / math.log(2)) / n - 1
    assert lower < leaf_bits < lower + 0.25


def _preorder_kinds(orc, m, n):
    """Preorder list of (is_leaf, size) for the codes of a node of m keys."""
    sh = orc.split_shape(m, n)
    if sh is None:
        return [(True, m)] if m >= 2 else []
    unit, fan = sh
    out = [(False, m)]
    for j in range(fan):
        out += _preorder_kinds(orc, unit if j < fan - 1 else m - (fan - 1) * unit, n)
    return out


def test_leaves_made_by_splits_behave_like_random_leaves(orc):
    """Leaf seeds inside builds (keys chosen by split hashes) have the same
    mean number of trials as independent random leaves: 1/P(pseudoforest) of
    uniformly random loop-free graphs on 16 cells, 33.04 (Monte Carlo, 4e8)."""
    N, n, b = 240000, 16, 400
    keys = inp.distinct_u64(N, 4242)
    lo, hi = orc.fingerprints_u64(keys)
    B = (N + b - 1) // b
    bkt = np.array((hi.astype(object) * B) >> 64, dtype=np.int64)
    order = np.lexsort((lo, hi))
    K = np.zeros(B + 1, np.int64)
    np.cumsum(np.bincount(bkt, minlength=B), out=K[1:])
    trials = []
    for i in range(B):
        sel = order[K[i]:K[i + 1]]
        seeds, _, _, _, _ = orc.bucket_build(lo[sel], hi[sel], n)
        kinds = _preorder_kinds(orc, int(sel.size), n)
        assert len(kinds) == seeds.size
        trials += [int(s) + 1 for s, (leaf, m) in zip(seeds, kinds) if leaf and m == n]
    t = np.array(trials, np.float64)
    se = t.std() / math.sqrt(t.size)
    assert t.size > 12000
    assert abs(t.mean() - 33.04) < 5 * se + 0.2


@pytest.mark.parametrize("n", [4, 24, 40])
def test_leaf_order_is_the_stable_partition(orc, n):
    """Sec. 2 RecSplit: a split node sends each key to the child its split
    hash names, children in order, keys keeping their relative order (so
    every leaf stays in ascending fingerprint order); codes are in preorder.
    The leaf order is rederived here from the preorder codes."""
    keys = inp.distinct_u64(3000, 77)
    lo, hi = orc.fingerprints_u64(keys)
    o = np.lexsort((lo, hi))[:900]
    seeds, _, llo, lhi, _ = orc.bucket_build(lo[o], hi[o], n)
    codes = iter(int(v) for v in seeds)
    out = []

    def walk(pairs):
        m = len(pairs)
        sh = orc.split_shape(m, n)
        if sh is None:
            if m >= 2:
                next(codes)
            out.extend(pairs)
            return
        unit, fan = sh
        s = next(codes)
        child = [orc.split_child(a, s, m, unit, fan) for a, _ in pairs]
        for j in range(fan):
            walk([p for p, c in zip(pairs, child) if c == j])

    walk([(int(a), int(b)) for a, b in zip(lo[o], hi[o])])
    assert next(codes, None) is None
    assert out == [(int(a), int(b)) for a, b in zip(llo, lhi)]
    pos = 0
    for m in _leaf_sizes(orc, len(o), n):
        leaf = out[pos:pos + m]
        assert leaf == sorted(leaf, key=lambda p: (p[1], p[0]))
        pos += m


@pytest.mark.parametrize("n", [8, 24, 40])
def test_splits_only_equals_the_full_bucket_build(orc, n):
    """The splits-only bucket walk gives the full build's split codes, Rice
    parameters and leaf order, and its leaves searched one by one give the
    full build's leaf codes."""
    keys = inp.distinct_u64(4000, 21)
    lo, hi = orc.fingerprints_u64(keys)
    o = np.lexsort((lo, hi))[:1500]
    full = orc.bucket_build(lo[o], hi[o], n)
    seeds, ks, llo, lhi, loff, lm = orc.bucket_splits(lo[o], hi[o], n)
    leaf = seeds == np.uint64(2**64 - 1)
    assert np.array_equal(ks, full[1]) and np.array_equal(llo, full[2]) and np.array_equal(lhi, full[3])
    assert np.array_equal(seeds[~leaf], full[0][~leaf]) and int(leaf.sum()) == lm.size
    offs = np.zeros(lm.size + 1, np.uint32)
    offs[1:] = np.cumsum(lm)
    packed = np.concatenate([llo[a:a + m] for a, m in zip(loff, lm)])
    assert np.array_equal(orc.leaf_search_batch(packed, offs, 0)[0], full[0][leaf])
