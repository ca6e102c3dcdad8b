"""Independent reader of the serialized MPHF format -- TEST INFRASTRUCTURE.

Used by the tests and by the oracle leg of the benchmark to read a serialized
object (the GPU's or the oracle's) section by section.  Written from the
format description, sharing no code with the C oracle or the CUDA library:
a header of 16 little-endian u64 words, then the Rice stream, Elias-Fano of
key prefixes, Elias-Fano of bit offsets, one seed byte per retrieval shard,
and the retrieval solution, each section padded to whole u64 words; all bit
vectors LSB-first.
"""
from __future__ import annotations

import numpy as np

HEADER = ["magic", "N", "n", "b", "B", "shard_buckets", "eps_num", "num_shards",
          "rice_bits", "efK_l", "efK_hi_bits", "efO_l", "efO_hi_bits", "ribbon_bits",
          "leaf_mode", "ribbon_width"]


def _words(nbits):
    return (nbits + 63) // 64


class Blob:
    def __init__(self, data: bytes):
        w = np.frombuffer(data, dtype="<u8")
        self.h = {k: int(v) for k, v in zip(HEADER, w[:16])}
        h = self.h
        B = h["B"]
        pos = 16
        self.sections = {}

        def take(name, nbits):
            nonlocal pos
            nw = _words(nbits)
            self.sections[name] = (pos, nw, nbits)
            arr = w[pos:pos + nw]
            pos += nw
            return arr

        self.rice = take("rice", h["rice_bits"])
        self.kl = take("efK_low", (B + 1) * h["efK_l"])
        self.kh = take("efK_high", h["efK_hi_bits"])
        self.ol = take("efO_low", (B + 1) * h["efO_l"])
        self.oh = take("efO_high", h["efO_hi_bits"])
        nseed_words = (h["num_shards"] + 7) // 8
        seedw = w[pos:pos + nseed_words]
        self.sections["shard_seeds"] = (pos, nseed_words, 8 * h["num_shards"])
        pos += nseed_words
        self.shard_seeds = seedw.view(np.uint8)[: h["num_shards"]].copy()
        self.ribbon = take("ribbon", h["ribbon_bits"])
        self.total_words = pos
        self.nwords = w.size

    @staticmethod
    def bit(words, p):
        return int((int(words[p // 64]) >> (p % 64)) & 1)

    @classmethod
    def bits(cls, words, p, k):
        v = 0
        for j in range(k):
            v |= cls.bit(words, p + j) << j
        return v

    def ef_decode(self, low, high, l, nbits, count):
        out = []
        i = 0
        for p in range(nbits):
            if self.bit(high, p):
                out.append(((p - i) << l) | self.bits(low, i * l, l))
                i += 1
                if i == count:
                    break
        return np.array(out, dtype=np.uint64)

    def K(self):
        h = self.h
        return self.ef_decode(self.kl, self.kh, h["efK_l"], h["efK_hi_bits"], h["B"] + 1)

    def O(self):
        h = self.h
        return self.ef_decode(self.ol, self.oh, h["efO_l"], h["efO_hi_bits"], h["B"] + 1)

    def rice_codes(self, start_bit, ks):
        """Decode len(ks) Rice codes with the given parameters from start_bit."""
        p = start_bit
        out = []
        for k in ks:
            low = self.bits(self.rice, p, k)
            p += k
            q = 0
            while self.bit(self.rice, p):
                q += 1
                p += 1
            p += 1
            out.append((q << k) | low)
        return out, p
