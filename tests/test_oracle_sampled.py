"""The sampled comparison used for builds too large for a full oracle build
(oracle/sampled.py) accepts the oracle's own bytes and rejects bytes with one
changed split code, one changed leaf value or a moved bucket boundary (CPU)."""
from __future__ import annotations

import numpy as np

import shk_inputs as inp
from oracle.blobfmt import Blob


def _build(orc, rf):
    keys = inp.distinct_u64(20000, 31)
    lo, hi = orc.fingerprints_u64(keys)
    return orc.build_mphf(keys, n=16, b=500, leaf_mode=rf), lo, hi


def _flip_bit(blob: bytes, word: int, bit: int) -> bytes:
    w = np.frombuffer(blob, dtype="<u8").copy()
    w[word] ^= np.uint64(1 << bit)
    return w.tobytes()


def test_sampled_parity_accepts_oracle_bytes_and_rejects_changes(orc):
    from oracle.sampled import sampled_parity

    for rf in (0, 1):
        blob, lo, hi = _build(orc, rf)
        r = sampled_parity(blob, lo, hi, 16, bool(rf), n_buckets=40, n_leaves=64)
        assert r["ok"] and r["sampled_buckets"] == 40 and r["sampled_leaves"] == 64, r
        bl = Blob(blob)
        rice0 = bl.sections["rice"][0]
        # a low bit of the first code of bucket 0 (a split seed: every bucket splits at n = 16)
        bad = sampled_parity(_flip_bit(blob, rice0, 0), lo, hi, 16, bool(rf), n_buckets=40, n_leaves=64)
        assert not bad["ok"]
        # the Elias-Fano high part of the key prefixes: a bucket boundary moves
        kh0 = bl.sections["efK_high"][0]
        bad2 = sampled_parity(_flip_bit(blob, kh0, 3), lo, hi, 16, bool(rf), n_buckets=40, n_leaves=64)
        assert not bad2["ok"]
