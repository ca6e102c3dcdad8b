"""Sampled comparison of a large serialized build with the oracle -- TEST
INFRASTRUCTURE ONLY (tests and the benchmark's oracle leg).

A full oracle build of 10^8 keys would take days of CPU time, so a large build
is checked the way its size allows:
  * every key's bucket is recomputed by the oracle from its fingerprint, and
    all B bucket sizes must equal the serialized Elias-Fano key prefixes;
  * for buckets drawn uniformly at random, the oracle rebuilds the splitting
    tree (every split seed) and the codes must equal the serialized Rice
    codes of that bucket, which must end exactly at the next bucket's offset;
  * for leaves drawn uniformly from those buckets, the oracle's leaf search
    must give the serialized leaf value.
Everything expected comes from the oracle (C, oracle/shk_oracle.c); the
serialized object is read with the independent reader oracle/blobfmt.py.
"""
from __future__ import annotations

import time

import numpy as np

from . import bucket_splits, buckets, leaf_search_batch
from .blobfmt import Blob

_ALL_ONES = np.uint64(2**64 - 1)


def sampled_parity(blob: bytes, lo: np.ndarray, hi: np.ndarray, n: int, rf: bool, *,
                   n_buckets: int = 50, n_leaves: int = 64, seed: int = 2308, nthreads: int = 0) -> dict:
    """Compare `blob` (a serialized build over keys with fingerprints lo, hi)
    with the oracle on sampled buckets and leaves; returns a summary dict
    whose 'ok' is True when everything compared is equal."""
    bl = Blob(blob)
    B, N = bl.h["B"], bl.h["N"]
    if N != lo.size:
        return {"ok": False, "why": f"blob holds {N} keys, {lo.size} given"}
    bk = buckets(hi, B)
    counts = np.bincount(bk, minlength=B)
    K = bl.K().astype(np.int64)
    sizes_ok = bool(np.array_equal(np.diff(K), counts))
    O = bl.O()
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(B, min(n_buckets, B), replace=False))
    flag = np.zeros(B, bool)
    flag[sample] = True
    sel = np.nonzero(flag[bk])[0]
    split_ok, n_split = True, 0
    items = []  # (leaf keys in leaf order, serialized value)
    t_split = time.perf_counter()
    for b in sample:
        idx = sel[bk[sel] == b]
        idx = idx[np.lexsort((lo[idx], hi[idx]))]
        seeds, ks, llo, _, loff, lm = bucket_splits(lo[idx], hi[idx], n)
        codes, end = bl.rice_codes(int(O[b]), [int(k) for k in ks])
        codes = np.array(codes, dtype=np.uint64)
        is_leaf = seeds == _ALL_ONES
        if end != int(O[b + 1]) or not np.array_equal(codes[~is_leaf], seeds[~is_leaf]):
            split_ok = False
        n_split += int((~is_leaf).sum())
        values = codes[is_leaf]
        for j in range(lm.size):
            items.append((llo[loff[j]:loff[j] + lm[j]], values[j]))
    t_split = time.perf_counter() - t_split
    pick = np.sort(rng.choice(len(items), min(n_leaves, len(items)), replace=False))
    packed = np.concatenate([items[j][0] for j in pick])
    po = np.zeros(pick.size + 1, np.uint32)
    po[1:] = np.cumsum([items[j][0].size for j in pick])
    want_gpu = np.array([items[j][1] for j in pick], dtype=np.uint64)
    t_leaf = time.perf_counter()
    vals, _ = leaf_search_batch(packed, po, 0, nthreads=nthreads, rf=rf)
    t_leaf = time.perf_counter() - t_leaf
    leaf_ok = bool(np.array_equal(vals, want_gpu))
    sizes = np.diff(po.astype(np.int64))
    return {"ok": sizes_ok and split_ok and leaf_ok, "bucket_sizes_equal": sizes_ok, "buckets": B,
            "sampled_buckets": int(sample.size), "split_codes_compared": n_split, "split_codes_equal": split_ok,
            "sampled_leaves": int(pick.size), "leaf_sizes": [int(sizes.min()), int(sizes.max())],
            "leaf_values_equal": leaf_ok, "oracle_leaf_keys": int(po[-1]), "oracle_leaf_s": t_leaf,
            "oracle_split_s": t_split}
