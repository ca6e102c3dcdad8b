"""Seeded synthetic inputs for the MPHF build workloads.

This module only draws random inputs; it holds none of the construction's
arithmetic.  Both the CPU oracle tests and the CUDA path (tests, bench) take
their inputs from here so that they see exactly the same keys.

The generator is the splitmix64 stream (Steele, Lea, Flood, OOPSLA 2014):
state_i = seed + i * 0x9E3779B97F4A7C15, output_i = splitmix64-output(state_i),
i = 1, 2, ...  Uniform doubles in [0, 1) take the top 53 bits.

Workloads (stand-ins for the paper's random-string inputs, Sec. 8):
  * ``distinct_u64(count, seed)``: the stream's outputs in order, repeats
    skipped, until ``count`` distinct 64-bit keys.
  * ``leaf_instances(count, seed)``: independent leaves with sizes
    40 + floor(U * 25) in [40, 64] and uniform 64-bit keys from the same stream.
  * ``ascii_strings(count, seed)``: strings of length 10 + floor(U * 41) in
    [10, 50], bytes uniform in [1, 127].
"""
from __future__ import annotations

import numpy as np

_PHI = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, count: int, start: int = 1) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream from ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(start, start + count, dtype=np.uint64)
        z = np.uint64(seed & (2**64 - 1)) + i * _PHI
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def _as_i64(x: int) -> int:
    x &= 2**64 - 1
    return x - 2**64 if x >= 2**63 else x


def splitmix64_stream_torch(seed: int, count: int, start: int = 1, device="cuda"):
    """The outputs of ``splitmix64_stream`` computed on ``device`` with torch
    int64 arithmetic (wrapping multiply and add; logical right shifts by
    masking); returns the 64-bit patterns as an int64 tensor."""
    import torch

    i = torch.arange(start, start + count, dtype=torch.int64, device=device)
    z = i * _as_i64(int(_PHI)) + _as_i64(seed)
    for sh, c in ((30, int(_C1)), (27, int(_C2))):
        z = (z ^ ((z >> sh) & ((1 << (64 - sh)) - 1))) * _as_i64(c)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def uniform01(seed: int, count: int, start: int = 1) -> np.ndarray:
    return (splitmix64_stream(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0**-53)


def distinct_u64(count: int, seed: int) -> np.ndarray:
    """First ``count`` distinct outputs of the stream, in stream order.  The
    output function is a bijection and the states are distinct, so these are
    the first ``count`` outputs; ``splitmix64_stream_torch(seed, count)``
    gives the same keys on a device."""
    out = np.empty(0, np.uint64)
    start = 1
    need = count
    while out.size < count:
        chunk = splitmix64_stream(seed, need + 16, start)
        start += chunk.size
        cand = np.concatenate([out, chunk])
        _, first = np.unique(cand, return_index=True)
        out = cand[np.sort(first)][:count]
        need = count - out.size
    return out


def leaf_instances(count: int, seed: int, lo: int = 40, hi: int = 64):
    """(keys, offsets): leaf i holds keys[offsets[i]:offsets[i+1]]."""
    span = hi - lo + 1
    sizes = lo + np.floor(uniform01(seed, count) * span).astype(np.int64)
    offs = np.zeros(count + 1, np.int64)
    np.cumsum(sizes, out=offs[1:])
    keys = splitmix64_stream(seed, int(offs[-1]), start=count + 1)
    return keys, offs.astype(np.uint32)


def ascii_strings(count: int, seed: int, min_len: int = 10, max_len: int = 50,
                  chunk: int = 1 << 26):
    """(bytes, offsets) of ``count`` random strings, bytes uniform in [1, 127].
    Generated in chunks of ``chunk`` bytes (same values for any chunk size)."""
    span = max_len - min_len + 1
    lens = min_len + np.floor(uniform01(seed, count) * span).astype(np.int64)
    offs = np.zeros(count + 1, np.uint64)
    np.cumsum(lens, out=offs[1:].view(np.int64))
    total = int(offs[-1])
    data = np.empty(total, np.uint8)
    for a in range(0, total, chunk):
        n = min(chunk, total - a)
        raw = splitmix64_stream(seed, n, start=count + 1 + a)
        data[a:a + n] = (1 + (raw % np.uint64(127))).astype(np.uint8)
    return data, offs


def ascii_strings_torch(count: int, seed: int, min_len: int = 10, max_len: int = 50,
                        device="cuda", chunk: int = 1 << 27):
    """``ascii_strings`` computed on ``device`` with torch integer arithmetic:
    the same (bytes, offsets) bit for bit, as a uint8 and an int64 tensor.
    Lengths take the top 53 bits of the stream as a double exactly as numpy
    does; a byte is 1 + (r mod 127) with r mod 127 taken from the 32-bit
    halves of r (2^32 = 16 mod 127, since 2^7 = 1 mod 127)."""
    import torch

    span = max_len - min_len + 1
    z = splitmix64_stream_torch(seed, count, start=1, device=device)
    u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0**-53)
    lens = min_len + torch.floor(u * span).to(torch.int64)
    del z, u
    offs = torch.zeros(count + 1, dtype=torch.int64, device=device)
    torch.cumsum(lens, 0, out=offs[1:])
    total = int(offs[-1])
    data = torch.empty(total, dtype=torch.uint8, device=device)
    for a in range(0, total, chunk):
        n = min(chunk, total - a)
        r = splitmix64_stream_torch(seed, n, start=count + 1 + a, device=device)
        mod = (((r >> 32) & 0xFFFFFFFF) * 16 + (r & 0xFFFFFFFF)) % 127
        data[a:a + n] = (1 + mod).to(torch.uint8)
        del r, mod
    return data, offs
