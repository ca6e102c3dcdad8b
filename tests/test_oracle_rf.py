"""Pins of the rotation-fitting leaf mode of the oracle (Sec. 4, Rotation
Fitting; App. A.2, Partial Hash Calculation)."""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import shk_inputs as inp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def test_sets_split_keys_in_half(orc):
    xs = inp.splitmix64_stream(3, 100000)
    b = np.array([orc.rf_set(int(x)) for x in xs[:20000]])
    assert abs(b.mean() - 0.5) < 5 * math.sqrt(0.25 / b.size)


@pytest.mark.parametrize("m", [5, 17, 33, 48, 64])
def test_candidate_cells_rotation_and_partial_seed(orc, m):
    """Set B: cells of seed s moved by r (the mask rotation = addition mod m);
    set A: cells of seed s - (s mod 8) when m > 32 (fixed over 8 seeds)."""
    xs = inp.splitmix64_stream(40 + m, 60)
    for x in xs:
        x = int(x)
        for s in (0, 5, 8, 13, 1000003):
            base = orc.leaf_hash(x, s, m)
            sa = s - s % 8 if m > 32 else s
            for r in (0, 1, m - 1):
                got = orc.rf_cells(x, s * m + r, m)
                if orc.rf_set(x):
                    assert got == ((base[0] + r) % m, (base[1] + r) % m)
                else:
                    assert got == orc.leaf_hash(x, sa, m)
                assert got[0] != got[1]


@pytest.mark.parametrize("m", [2, 3, 5, 8, 12, 34])
def test_rf_value_is_the_minimum(orc, m):
    """The stored value is the smallest v = s*m + r whose graph is a
    pseudoforest; the filter changes nothing."""
    for t in range(6 if m > 12 else 15):
        x = inp.splitmix64_stream(500 * m + t, m)
        v = orc.rf_value(x)
        assert orc.rf_value(x, use_filter=False) == v
        cells = [orc.rf_cells(int(k), v, m) for k in x]
        assert orc.is_pseudoforest([a for a, _ in cells], [b for _, b in cells])
        for v2 in range(v):
            cells = [orc.rf_cells(int(k), v2, m) for k in x]
            assert not orc.is_pseudoforest([a for a, _ in cells], [b for _, b in cells])


@pytest.mark.parametrize("m", [3, 6, 10, 13])
def test_rf_orientation_is_lexicographic_minimum(orc, m):
    for t in range(8):
        x = inp.splitmix64_stream(900 * m + t, m)
        v = orc.rf_value(x)
        cells = [orc.rf_cells(int(k), v, m) for k in x]
        valid = [bits for bits in itertools.product((0, 1), repeat=m)
                 if len({cells[i][bits[i]] for i in range(m)}) == m]
        assert tuple(int(b) for b in orc.orient_mode(x, v, True)) == valid[0]


@pytest.mark.parametrize("row", [r for r in _rows("fig2_rotation_fitting.txt") if int(r[0]) in (8, 12, 16, 20, 24, 28)])
def test_rf_seeds_against_fig2(orc, row):
    """Fig. 2 (left), ShockHash + RF: mean seeds tried = floor(v/m) + 1.  Our
    plain series sits 5-11 % below the paper's; the RF series within 10 %."""
    m, fig = int(row[0]), float(row[1])
    L = 20000 if m <= 20 else 6000
    x = inp.splitmix64_stream(8000 + m, L * m)
    off = (np.arange(L + 1) * m).astype(np.uint32)
    v, _ = orc.leaf_search_batch(x, off, rf=True)
    seeds = (v // m).astype(np.float64) + 1
    se = seeds.std() / math.sqrt(L)
    assert 0.88 * fig - 4 * se <= seeds.mean() <= 1.06 * fig + 4 * se


def test_rf_candidates_match_plain_trials(orc):
    """Each rotation is a new chance (Sec. 4): the mean number of candidates
    v + 1 is close to the plain mean number of seeds (within 15 %)."""
    m, L = 20, 12000
    x = inp.splitmix64_stream(31337, L * m)
    off = (np.arange(L + 1) * m).astype(np.uint32)
    v, _ = orc.leaf_search_batch(x, off, rf=True)
    s, _ = orc.leaf_search_batch(x, off, rf=False)
    ratio = (v.astype(np.float64) + 1).mean() / (s.astype(np.float64) + 1).mean()
    assert 0.9 < ratio < 1.25


@pytest.mark.parametrize("N,n,b", [(5000, 24, 800), (3000, 36, 1000), (777, 40, 2000), (2, 2, 2), (129, 16, 16)])
def test_rf_build_is_bijection(orc, N, n, b):
    from oracle.blobfmt import Blob

    keys = inp.distinct_u64(N, 300 + N)
    blob = orc.build_mphf(keys, n=n, b=b, leaf_mode=1)
    assert Blob(blob).h["leaf_mode"] == 1
    lo, hi = orc.fingerprints_u64(keys)
    r = orc.query(blob, lo, hi)
    assert np.array_equal(np.sort(r), np.arange(N, dtype=np.uint64))
    assert blob != orc.build_mphf(keys, n=n, b=b) or N <= 2
