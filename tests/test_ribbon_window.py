"""The 128-bit retrieval solve's elimination order, checked on the CPU.

The GPU solve (csrc/ribbon.cu, k_ribbon128) does not eliminate the way the
oracle does.  It takes a shard's rows in ascending start order.  It keeps only
a 128-slot window of the band, held in reduced form, so that no stored row
has a 1 in another stored row's pivot column.  A new row X is reduced in one
step: X is XORed with the stored rows at exactly the pivots where X itself has
a 1.  The new pivot is the result's first set column at or after the row's
start, cyclically in the ring of 128 slots.  That column is then cleared from
the stored rows that have it.  Rows leave the window as the start moves past
their pivot.

This file restates that procedure with Python integers as bit sets.  On rows
from the oracle's row hash, the canonical solution must equal the oracle's,
bit for bit.  The canonical solution is 0 on every non-pivot column; the
oracle gets it by plain sequential elimination (Sec. 2, Retrieval).  The
consistency verdict per seed must equal the oracle's too.
"""
from __future__ import annotations

import numpy as np
import pytest

import shk_inputs as inp

W = 128
RING = (1 << W) - 1


def _rot_left(v: int, r: int) -> int:
    r %= W
    return ((v << r) | (v >> (W - r))) & RING if r else v


def _rot_right(v: int, r: int) -> int:
    return _rot_left(v, (W - r) % W)


def window_solve(starts, coeffs, bits, m):
    """The window-reduced elimination; returns the solution bits, or None if
    the system is inconsistent."""
    order = sorted(range(len(starts)), key=lambda i: starts[i])
    ring = {}  # ring index -> (row in ring order, rhs); the row's pivot is the index
    band = [(0, 0)] * m  # per slot: (row in its pivot frame, rhs)
    fin = 0

    def retire(upto):
        nonlocal fin
        while fin < upto:
            j = fin % W
            if j in ring:
                row, rhs = ring.pop(j)
                band[fin] = (_rot_right(row, j), rhs)
            fin += 1

    for i in order:
        s = int(starts[i])
        retire(s)
        x = _rot_left(coeffs[i], s % W)  # ring order: bit c is slot s + ((c - s) mod 128)
        b = int(bits[i])
        r, rb = x, b
        for p, (row, rhs) in ring.items():  # one step: the stored rows at X's pivots
            if (x >> p) & 1:
                r ^= row
                rb ^= rhs
        if r == 0:
            if rb:
                return None
            continue
        rot = s % W
        q = min((c for c in range(W) if (r >> c) & 1), key=lambda c: (c - rot) % W)
        assert q not in ring  # the result is 0 on every stored pivot
        for p in list(ring):  # clear column q from the stored rows
            row, rhs = ring[p]
            if (row >> q) & 1:
                ring[p] = (row ^ r, rhs ^ rb)
        ring[q] = (r, rb)
    retire(m)
    # back substitution from the top: x[i] = rhs[i] + parity(row[i] bits 1.. & x[i+1..])
    sol = np.zeros(m, np.uint8)
    win = 0
    for i in range(m - 1, -1, -1):
        row, rhs = band[i]
        v = 0
        if row:
            v = (rhs ^ bin((row >> 1) & win).count("1")) & 1
        win = ((win << 1) | v) & RING
        sol[i] = v
    return sol


@pytest.mark.parametrize("k,seed", [(40, 1), (300, 2), (700, 3), (1500, 4)])
def test_window_reduced_elimination_equals_sequential(orc, k, seed):
    lo = inp.splitmix64_stream(61_000 + seed, k)
    hi = inp.splitmix64_stream(62_000 + seed, k)
    f = (inp.splitmix64_stream(63_000 + seed, k) & np.uint64(1)).astype(np.uint8)
    eps = orc.default_eps_num(W)
    m = orc.shard_slots(k, eps, W)
    want_seed, want = orc.ribbon_shard(lo, hi, f, eps, W)
    # every seed below the oracle's is inconsistent here too; the oracle's seed
    # gives the same canonical solution
    for r in range(want_seed + 1):
        starts, coeffs = orc.ribbon_rows(lo, hi, r, m, W)
        sol = window_solve([int(v) for v in starts], coeffs, f, m)
        if r < want_seed:
            assert sol is None, r
        else:
            assert sol is not None
            assert np.array_equal(sol, want)


def test_window_reduced_elimination_clumped_starts(orc):
    """Many rows with equal starts, and empty stretches between them: the
    window moves by more than one slot at a time and retires free slots."""
    rng = np.random.default_rng(7)
    k = 600
    m = orc.shard_slots(k, 6554, W)  # eps 10 %: solvable despite the clumps
    starts = (rng.integers(0, (m - W + 1) // 25, k) * 25).tolist()
    coeffs = [int(a) << 64 | int(b) | 1 for a, b in zip(rng.integers(0, 2**63, k), rng.integers(0, 2**63, k))]
    bits = rng.integers(0, 2, k)
    sol = window_solve(starts, coeffs, bits, m)
    assert sol is not None
    # the solution satisfies every equation, and is 0 off the pivots of
    # sequential elimination
    for s, c, b in zip(starts, coeffs, bits):
        acc = 0
        for j in range(W):
            if (c >> j) & 1:
                acc ^= int(sol[s + j])
        assert acc == b
    band = {}
    for i in sorted(range(k), key=lambda i: starts[i]):
        c, s = coeffs[i], starts[i]
        while c:
            if s not in band:
                band[s] = c
                break
            c ^= band[s]
            while c and not c & 1:
                c >>= 1
                s += 1
    assert all(sol[j] == 0 for j in range(m) if j not in band)
