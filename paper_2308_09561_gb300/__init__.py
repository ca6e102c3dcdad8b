"""GB300 ShockHash-RS construction: thin Python binding of libshk_gpu.so.

The functions below carry the names of the C ABI (include/shk.h) and only
marshal arguments: every step of the construction runs in the library's CUDA
kernels.  If the library has not been built, or no CUDA device is present,
every call raises -- there is no CPU fallback.

PyTorch is used for device memory and streams only: tensors are passed to the
library as raw device pointers.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libshk_gpu.so")

(SHK_OK, SHK_EINVAL, SHK_EDUPKEY, SHK_ENOMEM, SHK_ECUDA, SHK_ESEEDCAP, SHK_ETIMEOUT, SHK_EFORMAT,
 SHK_ECANCELLED) = range(9)
SHK_KEYS_U64, SHK_KEYS_STR, SHK_KEYS_FP128 = 0, 1, 2
SHK_SCHED_PERSISTENT, SHK_SCHED_PER_BUCKET, SHK_SCHED_SINGLE_LAUNCH = 0, 1, 2
SHK_LEAF_PLAIN, SHK_LEAF_ROTATION = 0, 1

# exported symbols declared in include/shk.h
EXPORTS = ("shk_build", "shk_build_stats", "shk_query", "shk_serialize", "shk_deserialize",
           "shk_size_bits", "shk_free", "shk_last_error", "shk_leaf_search", "shk_leaf_search_noalloc",
           "shk_leaf_tune", "shk_leaf_configs", "shk_leaf_graph_replays", "shk_leaf_search_rf",
           "shk_server_create",
           "shk_server_submit", "shk_server_poll", "shk_server_wait", "shk_server_get_stats",
           "shk_server_destroy", "shk_version", "shk_release_memory", "shk_int_issue_rate",
           "shk_server_cancel", "shk_build_footprint")


class ShkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"shk error {status}: {message}")
        self.status = status


class _Keys(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("on_device", ctypes.c_int32), ("data", ctypes.c_void_p),
                ("str_offsets", ctypes.c_void_p), ("n_keys", ctypes.c_uint64)]


class _Opts(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in
                ("leaf_size", "bucket_size", "shard_buckets", "eps_num", "sched", "seeds_per_lane",
                 "chunk_passes", "profile", "warps_per_block", "key_unroll", "leaf_mode", "deadline_ms")]


_STAT_U64 = ["n_keys", "n_buckets", "n_leaves", "n_search_leaves", "n_split_nodes", "leaf_seeds_min",
             "leaf_seeds_executed", "leaf_key_evals", "kernel_launches", "size_bits"]
_STAT_F64 = ["ms_fingerprint", "ms_partition", "ms_split", "ms_leaf", "ms_orient", "ms_encode",
             "ms_ribbon", "ms_total"]


class _Stats(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_uint64) for n in _STAT_U64] + [(n, ctypes.c_double) for n in _STAT_F64]
                + [("leaf_launches", ctypes.c_uint64), ("leaf_cfg", ctypes.c_uint32 * 4),
                   ("leaf_hash_evals", ctypes.c_uint64), ("leaf_rf_cells", ctypes.c_double),
                   ("leaf_seeds_tested", ctypes.c_uint64), ("leaf_t0_ns", ctypes.c_uint64),
                   ("leaf_t1_ns", ctypes.c_uint64), ("device_bytes_peak", ctypes.c_uint64)])


class _ReqInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("n_keys", ctypes.c_uint64),
                ("footprint_bytes", ctypes.c_uint64), ("submit_ns", ctypes.c_uint64),
                ("start_ns", ctypes.c_uint64), ("finish_ns", ctypes.c_uint64)]


class _SrvStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "queued", "running", "budget_bytes",
                                               "in_use_bytes", "peak_in_use_bytes")] + [("workers", ctypes.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libshk_gpu.so; raise if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ShkError(SHK_ECUDA, f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "shk_build": (i32, [ctypes.POINTER(_Keys), ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]),
        "shk_build_stats": (i32, [vp, ctypes.POINTER(_Stats)]),
        "shk_query": (i32, [vp, ctypes.POINTER(_Keys), vp, i32, vp]),
        "shk_serialize": (i32, [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "shk_deserialize": (i32, [vp, ctypes.c_size_t, ctypes.POINTER(vp)]),
        "shk_size_bits": (u64, [vp]),
        "shk_free": (None, [vp]),
        "shk_last_error": (ctypes.c_char_p, []),
        "shk_leaf_search": (i32, [vp, vp, u32, u64, vp, vp, vp]),
        "shk_leaf_search_noalloc": (i32, [vp, vp, u32, u64, vp, vp, vp]),
        "shk_leaf_tune": (i32, [u32, vp, vp, i32, vp]),
        "shk_leaf_configs": (u32, [vp, u32]),
        "shk_leaf_graph_replays": (u64, []),
        "shk_leaf_search_rf": (i32, [vp, vp, u32, vp, vp, vp]),
        "shk_server_create": (i32, [u64, u32, ctypes.POINTER(vp)]),
        "shk_server_submit": (i32, [vp, ctypes.POINTER(_Keys), ctypes.POINTER(_Opts), ctypes.POINTER(u64)]),
        "shk_server_poll": (i32, [vp, u64, ctypes.POINTER(vp), ctypes.POINTER(_ReqInfo)]),
        "shk_server_wait": (i32, [vp, u64, ctypes.POINTER(vp), ctypes.POINTER(_ReqInfo)]),
        "shk_server_get_stats": (i32, [vp, ctypes.POINTER(_SrvStats)]),
        "shk_server_destroy": (None, [vp]),
        "shk_server_cancel": (i32, [vp, u64]),
        "shk_build_footprint": (i32, [ctypes.POINTER(_Keys), ctypes.POINTER(_Opts), ctypes.POINTER(u64)]),
        "shk_version": (ctypes.c_char_p, []),
        "shk_release_memory": (None, []),
        "shk_int_issue_rate": (i32, [u32, u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def shk_last_error() -> str:
    return load_library().shk_last_error().decode()


def _check(status: int):
    if status != SHK_OK:
        raise ShkError(status, shk_last_error())


def _torch():
    import torch

    return torch


def _stream_handle(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _as_keys(keys, kind: int, str_offsets=None):
    """Describe keys (torch tensor on CUDA/CPU or numpy array) for the C ABI.
    Returns (struct, keepalive)."""
    torch = _torch()
    keep = []
    k = _Keys()
    k.kind = kind
    if isinstance(keys, torch.Tensor):
        t = keys.contiguous()
        keep.append(t)
        k.on_device = 1 if t.is_cuda else 0
        k.data = t.data_ptr() if t.numel() else None
        nbytes, itemsize = t.numel() * t.element_size(), t.element_size()
    else:
        a = np.ascontiguousarray(keys)
        keep.append(a)
        k.on_device = 0
        k.data = a.ctypes.data if a.size else None
        nbytes, itemsize = a.nbytes, a.itemsize
    want = {SHK_KEYS_U64: 8, SHK_KEYS_FP128: 8, SHK_KEYS_STR: 1}.get(kind)
    if want is None:
        raise ValueError(f"unknown key kind {kind}")
    if itemsize != want:
        raise ValueError(f"key kind {kind} takes {want}-byte elements, got {itemsize}-byte ones")
    if kind == SHK_KEYS_U64:
        k.n_keys = nbytes // 8
    elif kind == SHK_KEYS_FP128:
        if nbytes % 16:
            raise ValueError("128-bit fingerprints need an even number of 64-bit words")
        k.n_keys = nbytes // 16
    else:
        if isinstance(str_offsets, torch.Tensor):
            o = str_offsets.contiguous()
            if bool(o.is_cuda) != bool(k.on_device):
                raise ValueError("string bytes and offsets must be on the same side")
            keep.append(o)
            k.str_offsets = o.data_ptr()
            k.n_keys = o.numel() - 1
        else:
            o = np.ascontiguousarray(str_offsets, dtype=np.uint64)
            keep.append(o)
            k.str_offsets = o.ctypes.data
            k.n_keys = o.size - 1
    return k, keep


@dataclass
class Mphf:
    """An MPHF resident on the GPU (owned handle; freed by shk_free / close)."""

    handle: int

    def close(self):
        if self.handle:
            shk_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def serialize(self) -> bytes:
        return shk_serialize(self.handle)

    def size_bits(self) -> int:
        return shk_size_bits(self.handle)

    def stats(self) -> dict:
        return shk_build_stats(self.handle)

    def query(self, keys, kind: int = SHK_KEYS_U64, str_offsets=None, out=None, stream=None):
        return shk_query(self.handle, keys, kind=kind, str_offsets=str_offsets, out=out, stream=stream)


def _opts(leaf_size, bucket_size, shard_buckets=0, eps_num=0, sched=SHK_SCHED_PERSISTENT, seeds_per_lane=0,
          chunk_passes=0, profile=False, warps_per_block=0, key_unroll=0, leaf_mode=SHK_LEAF_PLAIN,
          deadline_ms=0) -> _Opts:
    return _Opts(leaf_size, bucket_size, shard_buckets, eps_num, sched, seeds_per_lane, chunk_passes,
                 1 if profile else 0, warps_per_block, key_unroll, leaf_mode, deadline_ms)


def shk_build(keys, leaf_size: int, bucket_size: int, *, kind: int = SHK_KEYS_U64, str_offsets=None,
              shard_buckets: int = 0, eps_num: int = 0, sched: int = SHK_SCHED_PERSISTENT,
              seeds_per_lane: int = 0, chunk_passes: int = 0, profile: bool = False,
              warps_per_block: int = 0, key_unroll: int = 0, leaf_mode: int = SHK_LEAF_PLAIN,
              deadline_ms: int = 0, stream=None) -> Mphf:
    lib = load_library()
    k, keep = _as_keys(keys, kind, str_offsets)
    o = _opts(leaf_size, bucket_size, shard_buckets, eps_num, sched, seeds_per_lane, chunk_passes, profile,
              warps_per_block, key_unroll, leaf_mode, deadline_ms)
    out = ctypes.c_void_p()
    _check(lib.shk_build(ctypes.byref(k), ctypes.byref(o), _stream_handle(stream), ctypes.byref(out)))
    del keep
    return Mphf(out.value)


def shk_build_stats(handle) -> dict:
    s = _Stats()
    _check(load_library().shk_build_stats(handle, ctypes.byref(s)))
    out = {name: getattr(s, name) for name, _ in _Stats._fields_}
    out["leaf_cfg"] = list(s.leaf_cfg)
    return out


def shk_query(handle, keys, *, kind: int = SHK_KEYS_U64, str_offsets=None, out=None, stream=None):
    """Ranks of keys.  Device keys give a device int64 tensor (uint64 bits);
    host keys give a numpy uint64 array, unless out is given."""
    torch = _torch()
    lib = load_library()
    k, keep = _as_keys(keys, kind, str_offsets)
    n = int(k.n_keys)
    if out is None:
        if k.on_device:
            out = torch.empty(n, dtype=torch.int64, device=keys.device)
        else:
            out = np.empty(n, dtype=np.uint64)
    if isinstance(out, torch.Tensor):
        ptr, on_dev = out.data_ptr(), int(out.is_cuda)
    else:
        ptr, on_dev = out.ctypes.data, 0
    _check(lib.shk_query(handle, ctypes.byref(k), ptr if n else None, on_dev, _stream_handle(stream)))
    del keep
    return out


def shk_serialize(handle) -> bytes:
    lib = load_library()
    n = ctypes.c_size_t()
    _check(lib.shk_serialize(handle, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.shk_serialize(handle, buf, n.value, ctypes.byref(n)))
    return buf.raw[: n.value]


def shk_deserialize(data: bytes) -> Mphf:
    lib = load_library()
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib.shk_deserialize(buf, len(data), ctypes.byref(out)))
    return Mphf(out.value)


def shk_size_bits(handle) -> int:
    return int(load_library().shk_size_bits(handle))


def shk_release_memory() -> None:
    """Return the library's pooled working memory to the device."""
    load_library().shk_release_memory()


def shk_int_issue_rate(mix: int, iters: int = 4096, stream=None) -> tuple[float, float]:
    """Integer-issue microbenchmark: (lane operations per second -- for mix 3
    key-seed evaluations per second --, ms of the best launch)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().shk_int_issue_rate(mix, iters, ctypes.byref(rate), ctypes.byref(ms),
                                             _stream_handle(stream)))
    return rate.value, ms.value


def shk_free(handle) -> None:
    load_library().shk_free(handle)


def shk_version() -> str:
    return load_library().shk_version().decode()


def shk_leaf_search(leaf_keys, leaf_off, seed_start: int = 0, want_f: bool = True, stream=None,
                    seeds_out=None, f_out=None):
    """Batched leaf search on device tensors: leaf_keys (int64/uint64 bits,
    the 64-bit leaf inputs), leaf_off (int32, n_leaves + 1 offsets).  Returns
    (seeds, f_masks) as device int64 tensors (f_masks None if not wanted).
    Passing the same tensors again (seeds_out / f_out included) replays the
    library's captured CUDA graph."""
    torch = _torch()
    lib = load_library()
    if not (leaf_keys.is_cuda and leaf_off.is_cuda):
        raise ValueError("shk_leaf_search takes device tensors")
    kk = leaf_keys if leaf_keys.is_contiguous() else leaf_keys.contiguous()
    off = leaf_off if leaf_off.is_contiguous() else leaf_off.contiguous()
    nl = off.numel() - 1
    seeds = seeds_out if seeds_out is not None else torch.empty(max(nl, 1), dtype=torch.int64, device=kk.device)
    if f_out is not None:
        f = f_out
    else:
        f = torch.empty(max(nl, 1), dtype=torch.int64, device=kk.device) if want_f else None
    _check(lib.shk_leaf_search(kk.data_ptr(), off.data_ptr(), nl, seed_start, seeds.data_ptr(),
                               f.data_ptr() if f is not None else None, _stream_handle(stream)))
    return seeds[:nl], (f[:nl] if f is not None else None)


def _noalloc_check(leaf_keys, leaf_off, seeds_out, f_out):
    """Argument checks of shk_leaf_search_noalloc, made before anything reaches
    the library: the library writes n_leaves 8-byte words into seeds_out (and
    f_out) on the device, so a short or narrow output would be written out of
    bounds there."""
    import torch

    if leaf_off.dtype != torch.int32:
        raise ValueError("leaf_off must be an int32 tensor of n_leaves + 1 offsets")
    if leaf_off.dim() != 1 or leaf_off.numel() < 1:
        raise ValueError("leaf_off must be a 1-D tensor of n_leaves + 1 offsets")
    nl = leaf_off.numel() - 1
    if leaf_keys.element_size() != 8:
        raise ValueError("leaf_keys must hold 8-byte (64-bit) elements")
    outs = [("seeds_out", seeds_out)] + ([("f_out", f_out)] if f_out is not None else [])
    for name, t in outs:
        if t.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
            raise ValueError(f"{name} must be an int64 tensor")
        if t.numel() < nl:
            raise ValueError(f"{name} holds {t.numel()} elements, fewer than the {nl} leaves")
    tensors = [leaf_keys, leaf_off, seeds_out] + ([f_out] if f_out is not None else [])
    for t in tensors:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("shk_leaf_search_noalloc takes contiguous device tensors")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in tensors):
        raise ValueError("every tensor must be on the current CUDA device")
    return nl


def shk_leaf_search_noalloc(leaf_keys, leaf_off, seeds_out, f_out=None, seed_start: int = 0, stream=None):
    """shk_leaf_search for callers that cannot allocate device memory while
    they run: the caller passes the output tensors (seeds_out, and f_out or
    None; int64 device tensors of at least n_leaves elements) and the library
    takes its working memory from a fixed array in its device image, so at
    most 65536 leaves per call.  Calls that overlap on the GPU race on that
    array; each call synchronises its stream."""
    nl = _noalloc_check(leaf_keys, leaf_off, seeds_out, f_out)
    lib = load_library()
    _check(lib.shk_leaf_search_noalloc(leaf_keys.data_ptr(), leaf_off.data_ptr(), nl, seed_start,
                                       seeds_out.data_ptr(), f_out.data_ptr() if f_out is not None else None,
                                       _stream_handle(stream)))
    return seeds_out, f_out


def shk_leaf_configs() -> list[tuple[int, int, int]]:
    """Supported leaf kernel configurations (seeds per lane, warps per block, unroll)."""
    lib = load_library()
    buf = (ctypes.c_uint32 * 256)()
    n = lib.shk_leaf_configs(buf, 64)
    return [(buf[4 * i], buf[4 * i + 1], buf[4 * i + 2]) for i in range(n)]


def shk_leaf_tune(leaf_size: int, probe_all: bool = False) -> dict:
    """The autotuner's leaf kernel configuration for leaf_size on the current
    device, its measured key-seed evaluations/s, and (probe_all) every
    configuration's rate."""
    lib = load_library()
    cfg = (ctypes.c_uint32 * 4)()
    rate = ctypes.c_double()
    n = len(shk_leaf_configs())
    allr = (ctypes.c_double * max(n, 1))()
    _check(lib.shk_leaf_tune(leaf_size, cfg, ctypes.byref(rate), int(probe_all), allr))
    out = {"seeds_per_lane": cfg[0], "warps_per_block": cfg[1], "key_unroll": cfg[2], "passes": cfg[3],
           "evals_per_s": rate.value}
    if probe_all:
        out["all"] = [{"cfg": c, "evals_per_s": allr[i]} for i, c in enumerate(shk_leaf_configs())]
    return out


def shk_leaf_graph_replays() -> int:
    return int(load_library().shk_leaf_graph_replays())


# --- serving -------------------------------------------------------------------
def shk_server_create(hbm_budget_bytes: int = 0, workers: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load_library().shk_server_create(hbm_budget_bytes, workers, ctypes.byref(out)))
    return out.value


def shk_server_submit(server: int, keys, leaf_size: int, bucket_size: int, *, kind: int = SHK_KEYS_U64,
                      str_offsets=None, **opt) -> int:
    k, keep = _as_keys(keys, kind, str_offsets)
    o = _opts(leaf_size, bucket_size, **opt)
    rid = ctypes.c_uint64()
    _check(load_library().shk_server_submit(server, ctypes.byref(k), ctypes.byref(o), ctypes.byref(rid)))
    del keep
    return rid.value


def _info_dict(info):
    return {name: getattr(info, name) for name, _ in _ReqInfo._fields_}


def shk_server_poll(server: int, req_id: int):
    """(Mphf or None, info dict); None while pending (info['done'] == 0)."""
    out = ctypes.c_void_p()
    info = _ReqInfo()
    _check(load_library().shk_server_poll(server, req_id, ctypes.byref(out), ctypes.byref(info)))
    return (Mphf(out.value) if out.value else None), _info_dict(info)


def shk_server_wait(server: int, req_id: int):
    out = ctypes.c_void_p()
    info = _ReqInfo()
    _check(load_library().shk_server_wait(server, req_id, ctypes.byref(out), ctypes.byref(info)))
    return (Mphf(out.value) if out.value else None), _info_dict(info)


def shk_server_get_stats(server: int) -> dict:
    s = _SrvStats()
    _check(load_library().shk_server_get_stats(server, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in _SrvStats._fields_}


def shk_server_cancel(server: int, req_id: int) -> None:
    _check(load_library().shk_server_cancel(server, req_id))


def shk_build_footprint(keys, leaf_size: int, bucket_size: int, *, kind: int = SHK_KEYS_U64, str_offsets=None,
                        **opt) -> int:
    """The server's device-memory estimate for a build of these keys."""
    k, keep = _as_keys(keys, kind, str_offsets)
    o = _opts(leaf_size, bucket_size, **opt)
    out = ctypes.c_uint64()
    _check(load_library().shk_build_footprint(ctypes.byref(k), ctypes.byref(o), ctypes.byref(out)))
    del keep
    return out.value


def shk_server_destroy(server: int) -> None:
    load_library().shk_server_destroy(server)


def shk_leaf_search_rf(leaf_keys, leaf_off, want_f: bool = True, stream=None):
    """Batched leaf search with rotation fitting: (values v = s*m + r, f masks)."""
    torch = _torch()
    lib = load_library()
    if not (leaf_keys.is_cuda and leaf_off.is_cuda):
        raise ValueError("shk_leaf_search_rf takes device tensors")
    kk = leaf_keys.contiguous()
    off = leaf_off.contiguous()
    nl = off.numel() - 1
    vals = torch.empty(max(nl, 1), dtype=torch.int64, device=kk.device)
    f = torch.empty(max(nl, 1), dtype=torch.int64, device=kk.device) if want_f else None
    _check(lib.shk_leaf_search_rf(kk.data_ptr(), off.data_ptr(), nl, vals.data_ptr(),
                                  f.data_ptr() if f is not None else None, _stream_handle(stream)))
    return vals[:nl], (f[:nl] if f is not None else None)
