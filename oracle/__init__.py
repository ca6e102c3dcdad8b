"""CPU oracle for ShockHash-RS construction -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct C (``shk_oracle.c``) written from the paper's
definitions, wrapped with ctypes.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library: nothing here imports the
package ``paper_2308_09561_gb300`` and the package never imports this module.

The hash functions are readings (the paper defines none); each is pinned to
something outside the oracle: the mixer to splitmix64's published outputs, the
string fingerprint to SipHash-2-4's published test vector, and the leaf, split
and retrieval hashes to the exact statistics of the ideal random model they
stand for (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shk_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EDUPKEY, ENOMEM, ESEEDCAP, EFORMAT = 0, 1, 2, 3, 5, 7
KEYS_U64, KEYS_STR, KEYS_FP128 = 0, 1, 2
SEED_CAP = 1 << 40
HEADER_WORDS = 16
MAGIC = 0x32303053524B4853
DEFAULT_EPS_NUM = 3277  # epsilon = 3277 / 2^16 ~ 5 %


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build() -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP over buckets)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        sig = {
            "orc_mix64": (u64, [u64]),
            "orc_fp_u64": (None, [vp, u64, vp, vp]),
            "orc_fp_str": (None, [vp, vp, u64, vp, vp]),
            "orc_siphash24": (u64, [u64, u64, vp, u64]),
            "orc_bucket": (u64, [u64, u64]),
            "orc_buckets": (None, [vp, u64, u64, vp]),
            "orc_split_shape": (i32, [u32, u32, vp, vp]),
            "orc_split_child": (u32, [u64, u64, u32, u32, u32]),
            "orc_split_seed": (i32, [vp, u32, u32, vp]),
            "orc_rice_k_split": (u32, [u32, u32]),
            "orc_rice_k_leaf": (u32, [u32]),
            "orc_leaf_hash": (None, [u64, u64, u32, vp, vp]),
            "orc_is_pseudoforest": (i32, [vp, vp, u32]),
            "orc_covers_all": (i32, [vp, vp, u32]),
            "orc_pf_batch": (None, [vp, vp, u64, u32, vp, vp]),
            "orc_leaf_seed": (i32, [vp, u32, u64, u64, i32, vp]),
            "orc_leaf_seed_stats": (None, [vp, u32, u64, u64, vp, vp]),
            "orc_orient": (i32, [vp, u32, u64, vp]),
            "orc_leaf_search_batch": (i32, [vp, vp, u32, u64, vp, vp, i32, i32]),
            "orc_bucket_build": (i32, [vp, vp, u32, u32, vp, vp, u32, vp, vp, i32]),
            "orc_bucket_splits": (i32, [vp, vp, u32, u32, vp, vp, u32, vp, vp, vp, u32, vp]),
            "orc_rf_set": (i32, [u64]),
            "orc_rf_cells": (None, [u64, u64, u32, vp, vp]),
            "orc_rf_value": (i32, [vp, u32, u64, u64, i32, vp]),
            "orc_orient_mode": (i32, [i32, vp, u32, u64, vp]),
            "orc_ribbon_shard": (i32, [vp, vp, vp, u64, u32, u32, vp, vp]),
            "orc_ribbon_rows": (None, [vp, vp, u64, u32, u64, u32, vp, vp, vp]),
            "orc_shard_slots": (u64, [u64, u32, u32]),
            "orc_default_shard_buckets": (u32, [u32, u32]),
            "orc_default_eps_num": (u32, [u32]),
            "orc_ribbon_width": (u32, [u32]),
            "orc_build": (i32, [i32, vp, vp, u64, u32, u32, u32, u32, i32, i32, vp, vp]),
            "orc_query": (i32, [vp, u64, vp, vp, u64, vp]),
            "orc_free": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# --- primitives ---------------------------------------------------------------
def mix64(z: int) -> int:
    return int(_load().orc_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def fingerprints_u64(keys) -> tuple[np.ndarray, np.ndarray]:
    keys = _u64(keys)
    lo = np.empty_like(keys)
    hi = np.empty_like(keys)
    _load().orc_fp_u64(_p(keys), keys.size, _p(lo), _p(hi))
    return lo, hi


def fingerprints_str(data: np.ndarray, offsets) -> tuple[np.ndarray, np.ndarray]:
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = _u64(offsets)
    n = offsets.size - 1
    lo = np.empty(n, np.uint64)
    hi = np.empty(n, np.uint64)
    _load().orc_fp_str(_p(data), _p(offsets), n, _p(lo), _p(hi))
    return lo, hi


def siphash24(k0: int, k1: int, msg: bytes) -> int:
    """SipHash-2-4 of msg under the 128-bit key (k0, k1) (64-bit output)."""
    buf = np.frombuffer(bytes(msg) + b"\0", dtype=np.uint8)
    return int(_load().orc_siphash24(k0, k1, _p(buf), len(msg)))


def bucket_of(hi: int, B: int) -> int:
    return int(_load().orc_bucket(hi, B))


def buckets(hi, B: int) -> np.ndarray:
    """Bucket of every key (uint32), from the high fingerprint halves."""
    hi = _u64(hi)
    out = np.empty(hi.size, np.uint32)
    _load().orc_buckets(_p(hi), hi.size, B, _p(out))
    return out


def split_shape(m: int, n: int):
    """(unit, fanout) of a split node of m keys, or None for a leaf."""
    unit = ctypes.c_uint32()
    fan = ctypes.c_uint32()
    r = _load().orc_split_shape(m, n, ctypes.byref(unit), ctypes.byref(fan))
    return (unit.value, fan.value) if r else None


def split_child(x: int, seed: int, m: int, unit: int, fanout: int) -> int:
    return int(_load().orc_split_child(x, seed, m, unit, fanout))


def split_seed(x, n: int) -> int:
    x = _u64(x)
    s = ctypes.c_uint64()
    st = _load().orc_split_seed(_p(x), x.size, n, ctypes.byref(s))
    if st:
        raise OracleError(st, "split_seed")
    return s.value


def rice_k_split(m: int, n: int) -> int:
    return int(_load().orc_rice_k_split(m, n))


def rice_k_leaf(m: int) -> int:
    return int(_load().orc_rice_k_leaf(m))


def leaf_hash(x: int, seed: int, m: int) -> tuple[int, int]:
    h0 = ctypes.c_uint32()
    h1 = ctypes.c_uint32()
    _load().orc_leaf_hash(x, seed, m, ctypes.byref(h0), ctypes.byref(h1))
    return h0.value, h1.value


def is_pseudoforest(h0, h1) -> bool:
    a = np.ascontiguousarray(h0, dtype=np.uint32)
    b = np.ascontiguousarray(h1, dtype=np.uint32)
    return bool(_load().orc_is_pseudoforest(_p(a), _p(b), a.size))


def covers_all(h0, h1) -> bool:
    a = np.ascontiguousarray(h0, dtype=np.uint32)
    b = np.ascontiguousarray(h1, dtype=np.uint32)
    return bool(_load().orc_covers_all(_p(a), _p(b), a.size))


def pf_batch(h0, h1):
    """Pseudoforest and coverage flags for a batch of graphs, shape (count, m)."""
    a = np.ascontiguousarray(h0, dtype=np.uint32)
    b = np.ascontiguousarray(h1, dtype=np.uint32)
    count, m = a.shape
    pf = np.zeros(count, np.uint8)
    cov = np.zeros(count, np.uint8)
    _load().orc_pf_batch(_p(a), _p(b), count, m, _p(pf), _p(cov))
    return pf.astype(bool), cov.astype(bool)


def leaf_seed(x, start: int = 0, cap: int = SEED_CAP, use_filter: bool = True) -> int:
    x = _u64(x)
    s = ctypes.c_uint64()
    st = _load().orc_leaf_seed(_p(x), x.size, start, cap, int(use_filter), ctypes.byref(s))
    if st:
        raise OracleError(st, "leaf_seed")
    return s.value


def leaf_seed_stats(x, s0: int, count: int) -> tuple[int, int]:
    """(#seeds passing the filter, #seeds giving a pseudoforest) in a range."""
    x = _u64(x)
    c = ctypes.c_uint64()
    p = ctypes.c_uint64()
    _load().orc_leaf_seed_stats(_p(x), x.size, s0, count, ctypes.byref(c), ctypes.byref(p))
    return c.value, p.value


def orient(x, seed: int) -> np.ndarray:
    x = _u64(x)
    f = np.zeros(x.size, np.uint8)
    st = _load().orc_orient(_p(x), x.size, seed, _p(f))
    if st:
        raise OracleError(st, "orient")
    return f


def leaf_search_batch(x, leaf_off, seed_start: int = 0, nthreads: int = 0, rf: bool = False):
    """First passing seed (or rotation-fitting value) >= seed_start per leaf,
    and f as a bit mask per leaf."""
    x = _u64(x)
    off = np.ascontiguousarray(leaf_off, dtype=np.uint32)
    nl = off.size - 1
    seeds = np.zeros(nl, np.uint64)
    fm = np.zeros(nl, np.uint64)
    st = _load().orc_leaf_search_batch(_p(x), _p(off), nl, seed_start, _p(seeds), _p(fm), nthreads,
                                       int(rf))
    if st:
        raise OracleError(st, "leaf_search_batch")
    return seeds, fm


def rf_set(x: int) -> int:
    return int(_load().orc_rf_set(x))


def rf_cells(x: int, v: int, m: int) -> tuple[int, int]:
    h0 = ctypes.c_uint32()
    h1 = ctypes.c_uint32()
    _load().orc_rf_cells(x, v, m, ctypes.byref(h0), ctypes.byref(h1))
    return h0.value, h1.value


def rf_value(x, start: int = 0, cap: int = SEED_CAP, use_filter: bool = True) -> int:
    x = _u64(x)
    v = ctypes.c_uint64()
    st = _load().orc_rf_value(_p(x), x.size, start, cap, int(use_filter), ctypes.byref(v))
    if st:
        raise OracleError(st, "rf_value")
    return v.value


def orient_mode(x, value: int, rf: bool) -> np.ndarray:
    x = _u64(x)
    f = np.zeros(x.size, np.uint8)
    st = _load().orc_orient_mode(int(rf), _p(x), x.size, value, _p(f))
    if st:
        raise OracleError(st, "orient_mode")
    return f


def bucket_build(lo_sorted, hi_sorted, n: int, rf: bool = False):
    """One bucket: (codes [(seed, k)] in preorder, lo, hi in leaf order, f)."""
    lo = _u64(lo_sorted).copy()
    hi = _u64(hi_sorted).copy()
    size = lo.size
    cap = 2 * size + 8
    seeds = np.zeros(cap, np.uint64)
    ks = np.zeros(cap, np.uint8)
    nc = ctypes.c_uint32()
    f = np.zeros(max(size, 1), np.uint8)
    st = _load().orc_bucket_build(_p(lo), _p(hi), size, n, _p(seeds), _p(ks), cap, ctypes.byref(nc), _p(f),
                                  int(rf))
    if st:
        raise OracleError(st, "bucket_build")
    return seeds[: nc.value].copy(), ks[: nc.value].copy(), lo, hi, f[:size].copy()


def bucket_splits(lo_sorted, hi_sorted, n: int):
    """One bucket's splitting tree without leaf searches: (codes in preorder,
    all-ones in leaf slots; Rice parameters; lo, hi in leaf order; leaf
    offsets; leaf sizes) for leaves of two or more keys."""
    lo = _u64(lo_sorted).copy()
    hi = _u64(hi_sorted).copy()
    size = lo.size
    cap = 2 * size + 8
    seeds = np.zeros(cap, np.uint64)
    ks = np.zeros(cap, np.uint8)
    loff = np.zeros(max(size, 1), np.uint32)
    lm = np.zeros(max(size, 1), np.uint32)
    nc, nl = ctypes.c_uint32(), ctypes.c_uint32()
    st = _load().orc_bucket_splits(_p(lo), _p(hi), size, n, _p(seeds), _p(ks), cap, ctypes.byref(nc),
                                   _p(loff), _p(lm), loff.size, ctypes.byref(nl))
    if st:
        raise OracleError(st, "bucket_splits")
    return (seeds[: nc.value].copy(), ks[: nc.value].copy(), lo, hi, loff[: nl.value].copy(),
            lm[: nl.value].copy())


def shard_slots(keys: int, eps_num: int = DEFAULT_EPS_NUM, w: int = 64) -> int:
    return int(_load().orc_shard_slots(keys, eps_num, w))


def default_shard_buckets(b: int, w: int = 64) -> int:
    return int(_load().orc_default_shard_buckets(b, w))


def ribbon_rows(lo, hi, seed: int, m: int, w: int = 64):
    """(start, coeff) of every key's retrieval row under shard seed `seed` in
    a shard of m slots of width w; coeff as Python ints of w bits."""
    lo = _u64(lo)
    hi = _u64(hi)
    start = np.empty_like(lo)
    c0 = np.empty_like(lo)
    c1 = np.empty_like(lo)
    _load().orc_ribbon_rows(_p(lo), _p(hi), lo.size, seed, m, w, _p(start), _p(c0), _p(c1))
    return start, [int(a) | (int(b) << 64) for a, b in zip(c0, c1)]


def ribbon_width(n: int) -> int:
    """Retrieval row width for leaf size n (128 above 24, else 64)."""
    return int(_load().orc_ribbon_width(n))


def default_eps_num(w: int) -> int:
    return int(_load().orc_default_eps_num(w))


def ribbon_shard(lo, hi, f, eps_num: int = DEFAULT_EPS_NUM, w: int = 64):
    """Smallest consistent shard seed and the canonical solution bits (ribbon
    width w)."""
    lo = _u64(lo)
    hi = _u64(hi)
    f = np.ascontiguousarray(f, dtype=np.uint8)
    m = shard_slots(lo.size, eps_num, w)
    sol = np.zeros(max(m, 1), np.uint8)
    seed = ctypes.c_uint32()
    st = _load().orc_ribbon_shard(_p(lo), _p(hi), _p(f), lo.size, eps_num, w, ctypes.byref(seed), _p(sol))
    if st:
        raise OracleError(st, "ribbon_shard")
    return seed.value, sol[:m].copy()


def build_mphf(keys=None, *, kind: int = KEYS_U64, str_data=None, str_offsets=None, fp=None,
               n: int = 32, b: int = 2000, shard_buckets: int = 0,
               eps_num: int = 0, nthreads: int = 0, leaf_mode: int = 0) -> bytes:
    """Whole construction -> serialized MPHF bytes.  leaf_mode 0: plain
    ShockHash leaves; 1: rotation fitting with partial hash calculation.
    shard_buckets / eps_num 0: the defaults of the leaf size's ribbon width."""
    lib = _load()
    offs = None
    if kind == KEYS_U64:
        data = _u64(keys)
        N = data.size
    elif kind == KEYS_STR:
        data = np.ascontiguousarray(str_data, dtype=np.uint8)
        offs = _u64(str_offsets)
        N = offs.size - 1
    elif kind == KEYS_FP128:
        data = _u64(fp).reshape(-1)
        N = data.size // 2
    else:
        raise ValueError(kind)
    out = ctypes.c_void_p()
    ln = ctypes.c_uint64()
    st = lib.orc_build(kind, _p(data), _p(offs) if offs is not None else None, N, n, b,
                       shard_buckets, eps_num, nthreads, leaf_mode, ctypes.byref(out), ctypes.byref(ln))
    if st:
        raise OracleError(st, "build")
    try:
        return ctypes.string_at(out.value, ln.value)
    finally:
        lib.orc_free(out)


def query(blob: bytes, lo, hi) -> np.ndarray:
    lo = _u64(lo)
    hi = _u64(hi)
    buf = np.frombuffer(blob, dtype=np.uint8)
    ranks = np.zeros(lo.size, np.uint64)
    st = _load().orc_query(_p(buf), buf.size, _p(lo), _p(hi), lo.size, _p(ranks))
    if st:
        raise OracleError(st, "query")
    return ranks
