"""Benchmark: MPHF construction of 10^8 random strings (lengths 10..50, bytes
1..127, splitmix64 stream seed 4), leaf size 64, bucket size 2000, rotation
fitting with partial hash calculation, retrieval overhead 1.5 %, on one GB300
per rank.

A step is one whole build (string fingerprints, bucket partition, splitting
trees, leaf search, orientation, Golomb-Rice/Elias-Fano encoding, retrieval
solve) from the strings resident in HBM to the encoded MPHF in HBM.  Prints one
JSON line (rank 0) with the 10^6-key, leaf-48 build as a sub-record.  Ranks
build independent key sets (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# headline workload: 10^8 strings, leaf 64, bucket 2000, rotation fitting
# (retrieval overhead: the library's default for 128-bit rows, eps = 164 / 2^16)
STR_KEYS, STR_LEAF, STR_BUCKET, STR_SEED, STR_EPS = 100_000_000, 64, 2000, 4, 0
WORKLOAD = "mphf_build_1e8_strings_leaf64_bucket2000"
METRIC = ("MPHF build keys/s (10^8 random strings, leaf 64, bucket 2000, rotation fitting), "
          "leaf seeds tested/s, % integer-issue roofline")
# sub-record workload: 10^6 distinct u64 keys, leaf 48, bucket 2000
N_KEYS, LEAF, BUCKET, KEY_SEED = 1_000_000, 48, 2000, 2
# integer lane-operations of one key-seed evaluation of the leaf hash + filter:
# xor 1, multiply-add 1, widening multiply by m 1, multiply-high by m-1 1,
# h1 adjust 2 (compare, add), two candidate bits into the mask: 8 when the mask
# is two 32-bit words (2 subtracts, 4 shifts, 2 ors; m > 32), 3 for m <= 32
OPS_PER_EVAL_WIDE = 14
OPS_PER_EVAL_NARROW = 9
# rotation fitting: one (seed, missed cell) step of the bit-parallel rotation
# filter = rotate the reflected 64-bit B mask (two 32-bit funnel shifts) and
# AND it into the seed's rotation set (one op, a three-input AND taking two
# cells per word)
OPS_PER_RF_CELL = 3
LEAF_TRAFFIC_PER_LEAF = 926_208 / 2_100  # DRAM bytes per leaf of the plain leaf kernel, ncu


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_key_seed(rank: int) -> int:
    """Each rank builds its own independent key set (weak scaling)."""
    return KEY_SEED + 1000 * rank


def max_over_ranks(seconds: float, dist, device) -> float:
    """The job's time is the slowest rank's time (no data-path collective:
    only this scalar is reduced)."""
    if dist is None:
        return seconds
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_leaf_step(step: int, leaves: int = 16):
    """One bounded step of the oracle on the headline workload's leaves: the
    strings [2000 step, 2000 (step + 1)) of the same stream taken as one
    bucket (leaf 64), its splitting tree by the oracle, then the oracle's
    rotation-fitting leaf search (OpenMP over leaves) on `leaves` of its leaves
    drawn at random.  Returns (keys searched, seconds of the leaf search,
    threads).  The leaf search is the oracle's dominant cost at leaf size 64
    (splits, encoding and retrieval are well under 1 % of it)."""
    import oracle
    import shk_inputs

    oracle.build()
    data, offs = shk_inputs.ascii_strings(STR_BUCKET * (step + 1), STR_SEED)
    a = STR_BUCKET * step
    sub = data[int(offs[a]):int(offs[-1])]
    so = offs[a:] - offs[a]
    lo, hi = oracle.fingerprints_str(sub, so)
    order = np.lexsort((lo, hi))
    _, _, llo, _, loff, lm = oracle.bucket_splits(lo[order], hi[order], STR_LEAF)
    pick = np.sort(np.random.default_rng(1000 + step).choice(lm.size, min(leaves, lm.size), replace=False))
    packed = np.concatenate([llo[loff[j]:loff[j] + lm[j]] for j in pick])
    po = np.zeros(pick.size + 1, np.uint32)
    po[1:] = np.cumsum(lm[pick])
    threads = min(os.cpu_count() or 1, int(pick.size))
    t = time.perf_counter()
    oracle.leaf_search_batch(packed, po, 0, nthreads=threads, rf=True)
    return int(po[-1]), time.perf_counter() - t, threads


def run_reference(args):
    """The oracle as it stands on the host cores, on a bounded sample of the
    headline workload per step (see _oracle_leaf_step)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    keys = secs = 0.0
    threads = 1
    t0 = time.perf_counter()
    for step in range(args.steps):
        k, dt, threads = _oracle_leaf_step(step, args.ref_leaves)
        keys += k
        secs += dt
    wall = time.perf_counter() - t0
    value = keys / secs
    line = {"metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "keys": STR_KEYS, "leaf_size": STR_LEAF, "bucket_size": STR_BUCKET,
                       "leaf_mode": "rotation fitting", "eps_num": STR_EPS or "library default",
                       "sample": f"{args.ref_leaves} leaves per step"},
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": threads, "kind": "oracle",
                             "sample": f"per step: the rotation-fitting leaf search of {args.ref_leaves} leaves of "
                                       f"a 2,000-string bucket of the same stream (step i: strings 2000 i .. "
                                       f"2000 (i+1) - 1), OpenMP over leaves; keys/s = leaf keys / search time; "
                                       f"{args.steps} steps, {wall:.0f} s wall"},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _bits_parts(blob: bytes, count: int) -> dict:
    """bits/key by section, from the serialized header (16 u64 words: N, n, b,
    B, shard buckets, eps_num, shards, Rice bits, Elias-Fano widths and high
    bits, retrieval bits, leaf mode, retrieval row width)."""
    h = np.frombuffer(blob[:128], dtype="<u8").astype(np.int64)
    B = int(h[4])
    ef = (B + 1) * int(h[9]) + int(h[10]) + (B + 1) * int(h[11]) + int(h[12])
    return {"rice_codes": int(h[8]) / count, "elias_fano": ef / count, "shard_seeds": 8 * int(h[7]) / count,
            "retrieval": int(h[13]) / count, "header_and_padding": (8 * len(blob) - int(h[8]) - ef - 8 * int(h[7])
                                                                    - int(h[13])) / count,
            "retrieval_row_bits": int(h[15]), "retrieval_eps_num": int(h[6]), "shard_buckets": int(h[5])}


def _int_issue(pkg):
    """Integer-issue microbenchmark (the library's shk_int_issue_rate)."""
    out = {}
    for mix, name in ((0, "alu_lop3_shf"), (1, "fma_imad"), (2, "imad_plus_lop3"), (3, "leaf_hash_evals")):
        rate, ms = pkg.shk_int_issue_rate(mix, 4096 if mix < 3 else 256)
        out[name] = rate / (1e12 if mix < 3 else 1.0)
    out["unit"] = "T lane-ops/s (leaf_hash_evals: key-seed evaluations/s)"
    return out


def _radix_rec(stats, count):
    """The radix partition phase alone: two passes that each read and write
    the 16-byte fingerprint record of every key (32 B per key per pass
    counted once read and once written) against the measured copy
    bandwidth."""
    ms = float(np.mean([s["ms_partition"] for s in stats]))
    gbs = 2 * 32 * count / (ms / 1e3) / 1e9
    peak = float(_peaks().get("hbm_gbs", 6800.0))
    return {"ms": ms, "passes": 2, "algorithmic_bytes": 2 * 32 * count, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "note": "phase time includes the host's check of the histogram and the "
                                        "launch gaps; ncu per-pass figures in profiles/"}


def u64_subrecord(pkg, args, flush, stream, peak_tops, cfg):
    """The 10^6 distinct u64 keys (stream seed 2), leaf 48, bucket 2000 build:
    plain leaves (with the plain leaf kernel's roofline), the same keys with
    rotation fitting, the leaf schedules compared, and queries."""
    import torch

    import shk_inputs

    keys = shk_inputs.distinct_u64(N_KEYS, KEY_SEED)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    for _ in range(2):
        pkg.shk_build(dkeys, LEAF, BUCKET, **cfg).close()
    stats, ms = [], []
    for i in range(3):
        flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m = pkg.shk_build(dkeys, LEAF, BUCKET, profile=True, **cfg)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        stats.append(m.stats())
        blob_bytes = len(m.serialize())
        m.close()
    leaf_ms = float(np.mean([s["ms_leaf"] for s in stats]))
    evals = stats[-1]["leaf_key_evals"]
    ach = evals * OPS_PER_EVAL_WIDE / (leaf_ms / 1e3) / 1e12
    rec = {"workload": "mphf_build_1M_u64_keys_leaf48_bucket2000", "keys": N_KEYS,
           "keys_per_s": N_KEYS / (float(np.mean(ms)) / 1e3), "ms_per_build": float(np.mean(ms)),
           "bits_per_key": 8 * blob_bytes / N_KEYS,
           "leaf_seeds_per_s": stats[-1]["leaf_seeds_min"] / (leaf_ms / 1e3),
           "key_seed_evals_per_s": evals / (leaf_ms / 1e3),
           "leaf_kernel_cfg": stats[-1]["leaf_cfg"],
           "phase_ms": {k: float(np.mean([s[k] for s in stats])) for k in
                        ("ms_fingerprint", "ms_partition", "ms_split", "ms_leaf", "ms_orient", "ms_encode",
                         "ms_ribbon", "ms_total")},
           "roofline": {"bound": "alu", "kernel": "k_leaf_persistent", "achieved": ach, "peak": peak_tops,
                        "unit": "T int-lane-ops/s", "frac": ach / peak_tops,
                        "traffic": LEAF_TRAFFIC_PER_LEAF * stats[-1]["n_leaves"],
                        "traffic_note": "scaled by leaves from an ncu capture of the 10^5-key build",
                        "ops_per_launch": evals * OPS_PER_EVAL_WIDE}}
    core = pkg.shk_int_issue_rate(3, 256)[0]
    rec["roofline"]["frac_of_hash_core"] = evals / (leaf_ms / 1e3) / core
    rec["roofline"]["hash_core_evals_per_s"] = core
    # rotation fitting with partial hash calculation on the same keys
    rf = []
    for _ in range(3):
        m = pkg.shk_build(dkeys, LEAF, BUCKET, leaf_mode=pkg.SHK_LEAF_ROTATION, profile=True)
        rf.append(m.stats())
        m.close()
    rf_ms = float(np.median([s["ms_total"] for s in rf]))
    rec["rotation_fitting"] = {"keys_per_s": N_KEYS / (rf_ms / 1e3), "ms_total": rf_ms,
                               "ms_leaf": float(np.median([s["ms_leaf"] for s in rf]))}
    # leaf schedules: the persistent work-stealing launch, one launch over all
    # leaves with one warp per leaf (no work sharing), and one launch per
    # bucket; the per-bucket form on 10^5 keys (the whole set with
    # --compare-per-bucket), the others on all 10^6
    sched = {}
    for name, sc, nk in (("persistent", pkg.SHK_SCHED_PERSISTENT, N_KEYS),
                         ("single_launch_one_warp_per_leaf", pkg.SHK_SCHED_SINGLE_LAUNCH, N_KEYS),
                         ("persistent_100k", pkg.SHK_SCHED_PERSISTENT, 100_000),
                         ("per_bucket_100k", pkg.SHK_SCHED_PER_BUCKET, N_KEYS if args.compare_per_bucket
                          else 100_000)):
        m = pkg.shk_build(dkeys[:nk], LEAF, BUCKET, sched=sc, profile=True, **cfg)
        st = m.stats()
        m.close()
        sched[name] = {"keys": nk, "ms_leaf": st["ms_leaf"], "leaf_launches": st["leaf_launches"]}
    sched["speedup_persistent_vs_single_launch"] = (sched["single_launch_one_warp_per_leaf"]["ms_leaf"]
                                                    / sched["persistent"]["ms_leaf"])
    sched["speedup_persistent_vs_per_bucket"] = (sched["per_bucket_100k"]["ms_leaf"]
                                                 / sched["persistent_100k"]["ms_leaf"])
    rec["leaf_schedules"] = sched
    # queries: every key, device in and out, L2 flushed before each pass
    mq = pkg.shk_build(dkeys, LEAF, BUCKET, **cfg)
    mq.query(dkeys)
    q_ms = []
    for i in range(5):
        flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mq.query(dkeys)
        b.record(stream)
        torch.cuda.synchronize()
        q_ms.append(a.elapsed_time(b))
    mq.close()
    rec["query_keys_per_s"] = N_KEYS / (float(np.median(q_ms)) / 1e3)
    return rec, int(sum(s["kernel_launches"] for s in stats))


def paper_config_run(pkg, ddata, doffs, flush, stream):
    """The one configuration the paper publishes numbers for that runs here
    as printed: ShockHash-RS with rotation fitting, n = 58, b = 2000, 10^7
    keys (the paper's queries table).  The keys are the first 10^7 strings of
    the headline stream (random strings, the paper's key recipe)."""
    import torch

    count = min(10_000_000, doffs.numel() - 1)
    offs = doffs[:count + 1].contiguous()
    data = ddata[:int(offs[-1].item())]
    opts = dict(kind=pkg.SHK_KEYS_STR, str_offsets=offs, leaf_mode=pkg.SHK_LEAF_ROTATION)
    pkg.shk_build(data, 58, 2000, **opts).close()
    ms, stats = [], []
    for i in range(2):
        flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m = pkg.shk_build(data, 58, 2000, profile=True, **opts)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        stats.append(m.stats())
        nbytes = len(m.serialize())
        m.close()
    t = float(np.mean(ms)) / 1e3
    return {"workload": "mphf_build_1e7_strings_leaf58_bucket2000_rf", "keys": count,
            "keys_per_s": count / t, "ns_per_key": 1e9 * t / count, "ms_per_build": 1e3 * t,
            "bits_per_key": 8 * nbytes / count, "ms_leaf": float(np.mean([s["ms_leaf"] for s in stats])),
            "ms_ribbon": float(np.mean([s["ms_ribbon"] for s in stats])),
            "paper": {"bits_per_key": 1.523, "ns_per_key": 111_593, "keys_per_s": 8_961,
                      "setting": "one core of an Intel i7-11700 (AVX-512), rotation fitting, BuRR retrieval; "
                                 "context only, not this hardware",
                      "source": "queries table, ShockHash-RS n = 58, b = 2000, N = 10^7"}}


def run_ours(args):
    """The headline: builds of the 10^8-string workload (see the module
    docstring), then its checks, the end-to-end number, sub-records and the
    oracle leg."""
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2308_09561_gb300 as pkg
    import shk_inputs

    pkg.load_library()
    count = args.keys or STR_KEYS
    t = time.perf_counter()
    ddata, doffs = shk_inputs.ascii_strings_torch(count, STR_SEED + 1000 * rank, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t
    hdata = ddata.cpu().pin_memory()
    hoffs = doffs.cpu().pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    mode = pkg.SHK_LEAF_ROTATION if args.leaf_mode == "rf" else pkg.SHK_LEAF_PLAIN
    opts = dict(kind=pkg.SHK_KEYS_STR, leaf_mode=mode, eps_num=args.eps_num)

    def build(data, offs, profile=True):
        return pkg.shk_build(data, STR_LEAF, STR_BUCKET, str_offsets=offs, profile=profile, **opts)

    for _ in range(max(args.warmup, 0)):
        build(ddata, doffs).close()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats, last = [], None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            m = build(ddata, doffs)
            ev[i][1].record(stream)
            stats.append(m.stats())
            if last is not None:
                last.close()
            last = m
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_sum = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    value = count * ws * args.steps / t_sum
    clocks = clk.summary()
    st = stats[-1]

    # every key ranks bijectively (the last timed build)
    blob = last.serialize()
    torch.cuda.synchronize()
    tq = time.perf_counter()
    ranks = last.query(ddata, kind=pkg.SHK_KEYS_STR, str_offsets=doffs)
    torch.cuda.synchronize()
    query_s = time.perf_counter() - tq
    srt, _ = torch.sort(ranks)
    bijection = bool(torch.equal(srt, torch.arange(count, device="cuda", dtype=torch.int64)))
    del srt, ranks
    last.close()

    # end to end through the public API: pinned host strings in, serialized MPHF out
    # (one untimed build first, as for the device-resident steps: the pool grows
    # once for the staged copy of the strings)
    build(hdata, hoffs, profile=False).close()
    torch.cuda.synchronize()
    t = time.perf_counter()
    m = build(hdata, hoffs, profile=False)
    e2e_blob = m.serialize()
    e2e_s = time.perf_counter() - t
    m.close()
    e2e_same = e2e_blob == blob

    # roofline of the rotation-fitting leaf kernel (or the plain one)
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tops = sms * 4 * 32 * sm_max_mhz * 1e6 / 1e12
    leaf_ms = float(np.mean([s["ms_leaf"] for s in stats]))
    if mode == pkg.SHK_LEAF_ROTATION:
        ops = st["leaf_hash_evals"] * OPS_PER_EVAL_WIDE + st["leaf_rf_cells"] * OPS_PER_RF_CELL
        kernel = "k_leaf_rf_persistent"
        ops_note = (f"{OPS_PER_EVAL_WIDE} per key hash evaluation (a sequential search's: |B| T + |A| ceil(T/8) "
                    f"per leaf, T = seeds tested) + {OPS_PER_RF_CELL} per (seed, missed cell) step of the "
                    f"bit-parallel rotation filter (expected steps given |A|)")
    else:
        ops = st["leaf_key_evals"] * OPS_PER_EVAL_WIDE
        kernel = "k_leaf_persistent"
        ops_note = f"{OPS_PER_EVAL_WIDE} per key-seed evaluation, sum over leaves of (seed + 1) m"
    achieved = ops / (leaf_ms / 1e3) / 1e12
    ints = _int_issue(pkg)
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_tops,
                "unit": "T int-lane-ops/s", "frac": achieved / peak_tops, "traffic": None,
                "traffic_note": "no DRAM traffic to speak of: each leaf's keys are read once into "
                                "shared memory (ncu capture summarised in profiles/)",
                "ops_per_launch": ops, "ops_note": ops_note,
                "peak_note": f"{sms} SMs x 4 schedulers x 32 lanes x {sm_max_mhz:.0f} MHz (max SM clock); "
                             f"measured achievable on this GPU (1:1 multiply-add + logic): "
                             f"{ints['imad_plus_lop3']:.1f}",
                "frac_of_measured_achievable": achieved / ints["imad_plus_lop3"],
                "hash_evals_per_s": st["leaf_hash_evals"] / (leaf_ms / 1e3),
                "frac_of_hash_core": st["leaf_hash_evals"] / (leaf_ms / 1e3) / ints["leaf_hash_evals"],
                "hash_core_note": "hash evaluations/s over the bare leaf hash core's (keys in registers, "
                                  "int_issue_microbench.leaf_hash_evals): the rate the hash alone allows"}
    cfg = {}
    if args.leaf_cfg:
        u, w, r = (int(v) for v in args.leaf_cfg.split(","))
        cfg = {"seeds_per_lane": u, "warps_per_block": w, "key_unroll": r, "chunk_passes": 8}
    u64rec, u64_launches = ({}, 0) if args.no_subrecords else u64_subrecord(pkg, args, flush, stream, peak_tops, cfg)
    part_bytes = int(hdata.numel()) + 8 * (count + 1) + 16 * count + 32 * count
    part_ms = float(np.mean([s["ms_fingerprint"] + s["ms_partition"] for s in stats]))
    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "keys": count, "string_bytes": int(hdata.numel()),
                   "leaf_size": STR_LEAF, "bucket_size": STR_BUCKET, "leaf_mode": args.leaf_mode,
                   "eps_num": args.eps_num, "key_stream_seed": STR_SEED, "schedule": "persistent",
                   "l2": "inputs larger than L2 (string bytes + offsets); also 256 MB written between timed "
                         "steps, outside the step events",
                   "parallelism": f"replicas x{ws}"},
        "bits_per_key": 8 * len(blob) / count,
        "bits_per_key_parts": _bits_parts(blob, count),
        "bijection_all_keys": bijection,
        "leaf_seeds_per_s": st["leaf_seeds_tested"] / (leaf_ms / 1e3),
        "leaf_candidates_per_s": st["leaf_seeds_min"] / (leaf_ms / 1e3),
        "leaf_hash_evals_per_s": st["leaf_hash_evals"] / (leaf_ms / 1e3),
        "leaf_seeds_executed_over_tested": st["leaf_seeds_executed"] / max(st["leaf_seeds_tested"], 1),
        "leaf_note": "seeds tested = sum over leaves of floor(v/m) + 1 (rotation fitting; seed + 1 plain); "
                     "candidates = sum of (v + 1), v = seed m + rotation; executed / tested = the work "
                     "stealing's overshoot (seeds past a leaf's solution searched by helper warps)",
        "phase_ms": {k: float(np.mean([s[k] for s in stats])) for k in
                     ("ms_fingerprint", "ms_partition", "ms_split", "ms_leaf", "ms_orient", "ms_encode",
                      "ms_ribbon", "ms_total")},
        "partition_gbs": part_bytes / (part_ms / 1e3) / 1e9,
        "radix_partition": _radix_rec(stats, count),
        "roofline": roofline,
        "int_issue_microbench": ints,
        "e2e": {"value": count * ws / e2e_s, "unit": "keys/s", "h2d_bytes_per_step":
                int(hdata.numel()) + 8 * (count + 1), "d2h_bytes_per_step": len(e2e_blob),
                "same_bytes_as_device_build": e2e_same},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "query_s_all_keys": query_s,
        "input_generation_s": gen_s,
        "wall_s_timed": wall,
        "u64_1M_leaf48": u64rec,
        "served_builds": {} if args.no_subrecords else serve_run(pkg, args.serve_requests, args.serve_max_keys,
                                                                  True, rank),
        "served_builds_burst": {} if args.no_subrecords else serve_run(pkg, args.serve_requests,
                                                                        args.serve_max_keys, True, rank,
                                                                        burst=True),
        "paper_table_config": {} if args.no_subrecords else paper_config_run(pkg, ddata, doffs, flush, stream),
    }
    if clocks:
        line["clocks"] = clocks
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle.sampled import sampled_parity

        oracle.build()
        data = hdata.numpy()
        offs = hoffs.numpy().view(np.uint64)
        lo, hi = oracle.fingerprints_str(data, offs)
        cores = os.cpu_count() or 1
        par = sampled_parity(blob, lo, hi, STR_LEAF, mode == pkg.SHK_LEAF_ROTATION, n_buckets=args.parity_buckets,
                             n_leaves=args.parity_leaves, nthreads=cores)
        line["oracle_parity_sampled"] = par
        line["cpu_baseline"] = {"value": par["oracle_leaf_keys"] / par["oracle_leaf_s"], "unit": "keys/s",
                                "cores": min(cores, par["sampled_leaves"]), "kind": "oracle",
                                "sample": f"extrapolated per key from the oracle's leaf search of "
                                          f"{par['sampled_leaves']} leaves drawn from {par['sampled_buckets']} "
                                          f"random buckets of this build ({par['oracle_leaf_s']:.1f} s, OpenMP "
                                          f"over leaves); the leaf search is the oracle's dominant cost at "
                                          f"leaf size 64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_leafbatch(args):
    """65,536 independent leaves, sizes uniform in [40, 64], uniform 64-bit
    keys (stream seed 3), seed start 0: one graph-captured persistent launch
    per step (replayed), first passing seed and orientation per leaf."""
    import torch

    import paper_2308_09561_gb300 as pkg
    import shk_inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pkg.load_library()
    count = args.keys or 65536
    keys, offs = shk_inputs.leaf_instances(count, 3 + 1000 * rank)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    off = torch.from_numpy(offs.view(np.int32)).cuda()
    seeds = torch.empty(count, dtype=torch.int64, device="cuda")
    fm = torch.empty(count, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rf = args.leaf_mode == "rf" and args.workload_leafbatch_rf
    for _ in range(max(args.warmup, 0)):
        if rf:
            pkg.shk_leaf_search_rf(dk, off)
        else:
            pkg.shk_leaf_search(dk, off, 0, seeds_out=seeds, f_out=fm)
    torch.cuda.synchronize()
    r0 = pkg.shk_leaf_graph_replays()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            if rf:
                seeds, fm = pkg.shk_leaf_search_rf(dk, off)
            else:
                pkg.shk_leaf_search(dk, off, 0, seeds_out=seeds, f_out=fm)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    s = seeds.cpu().numpy().view(np.uint64).astype(np.float64)
    sizes = np.diff(offs.astype(np.int64))
    seeds_min = float((s + 1).sum())  # with rotation fitting: candidates v + 1
    evals = float(((s + 1) * sizes).sum())
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 4 * 32 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    if rf:
        # rotation fitting: seeds s = 0 .. floor(v / m) are tested; each seed
        # hashes the keys of set B (m / 2 expected) and, once per 8 seeds,
        # those of set A.  Only the hash evaluations are counted (the rotation
        # intersection is left out), so this is a lower bound on the work.
        tested = np.floor(s / sizes) + 1
        hashes = float((tested * sizes * (0.5 + 0.5 / 8)).sum())
        ach = hashes * OPS_PER_EVAL_WIDE / (t / args.steps) / 1e12
        kernel = "k_leaf_rf_persistent"
    else:
        ach = evals * OPS_PER_EVAL_WIDE / (t / args.steps) / 1e12
        kernel = "k_leaf_persistent"
    line = {"metric": "batched leaf search: leaf seeds (rotation fitting: candidates) tested/s "
                      "(65,536 leaves, m in [40,64])",
            "leaf_mode": "rf" if rf else "plain",
            "value": seeds_min * args.steps / t, "unit": "seeds/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "leaf_batch_65536_leaves_m40_64", "leaves": count, "seed_stream": 3},
            "key_seed_evals_per_s": evals * args.steps / t, "mean_seed": float(s.mean()),
            "graph_replays": pkg.shk_leaf_graph_replays() - r0,
            "roofline": {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak,
                         "unit": "T int-lane-ops/s", "frac": ach / peak,
                         "ops_note": ("hash evaluations only (expected |B| per seed, |A| per 8 seeds); the "
                                      "rotation filter's work is not counted, so a lower bound (the build "
                                      "record counts it)") if rf else
                                     f"{OPS_PER_EVAL_WIDE} per key-seed evaluation, sum over leaves of (seed + 1) m"}}
    if not rf:
        line["tuned_cfg"] = pkg.shk_leaf_tune(64)
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serve_run(pkg, requests: int, max_keys: float, rf: bool, rank: int = 0, check_alone: bool = True,
              clk=None, burst: bool = False) -> dict:
    """Served builds: a Poisson stream of MPHF build requests (uniform u64
    keys generated on the device, sizes log-uniform in [1e3, max_keys], leaf
    size 48 or 58 by coin, bucket 2000, stream seed 5, request i from sub-seed
    5 + 7919 i) submitted as device tensors into one server with 4 builds in
    flight; plain or rotation-fitting leaves.  The arrival rate is set for
    ~80 % offered load from calibration builds of each leaf size (a build's
    time alone fitted as fixed + per-key cost).  Reports
    p50/p99 build latency (submit to finish), aggregate keys/s, how the
    requests' leaf-search kernels overlapped on the device (device-time
    intervals), and whether every result equals the same build alone.  With
    burst, every request arrives at once (a backlog: the server's throughput
    and its builds' overlap on the device)."""
    import torch

    import shk_inputs

    R = requests
    u = shk_inputs.uniform01(5 + 1000 * rank, 3 * R)
    sizes = np.floor(10 ** (3 + np.log10(max_keys / 1e3) * u[0::3])).astype(np.int64)
    mode = pkg.SHK_LEAF_ROTATION if rf else pkg.SHK_LEAF_PLAIN
    leafs = np.where(u[1::3] < 0.5, 48, 58)
    reqs = [(shk_inputs.splitmix64_stream_torch(5 + 7919 * i + 1000003 * rank, int(sz), device="cuda"), int(n))
            for i, (sz, n) in enumerate(zip(sizes, leafs))]
    torch.cuda.synchronize()
    # calibration: a build's time alone as fixed + per-key cost at each leaf
    # size, fitted to builds of 6*10^4 and 6*10^5 keys (small builds are
    # dominated by fixed costs such as the retrieval solve's serial chain)
    fixed, per_key = {}, {}
    for n in (48, 58):
        ts = []
        for cnt in (60_000, 600_000):
            k = shk_inputs.distinct_u64(cnt, 77 + n)
            pkg.shk_build(k, n, BUCKET, leaf_mode=mode).close()  # tuning / warm-up
            t = time.perf_counter()
            pkg.shk_build(k, n, BUCKET, leaf_mode=mode).close()
            ts.append(time.perf_counter() - t)
        per_key[n] = max((ts[1] - ts[0]) / 540_000, 1e-12)
        fixed[n] = max(ts[0] - 60_000 * per_key[n], 0.0)
    service = float(np.mean([fixed[n] + k.numel() * per_key[n] for k, n in reqs]))
    rate = 0.8 / service
    gaps = -np.log(1.0 - shk_inputs.uniform01(55 + 1000 * rank, R)) / rate
    if burst:
        gaps = np.zeros(R)
    srv = pkg.shk_server_create(0, 4)
    pending, infos, blobs, spans = {}, {}, {}, []

    def collect(rid, m, info):
        i = pending.pop(rid)
        infos[i] = info
        if m is not None:
            st = m.stats()
            spans.append((st["leaf_t0_ns"], st["leaf_t1_ns"]))
            if check_alone:
                blobs[i] = m.serialize()
            m.close()

    t0 = time.perf_counter()
    arrivals = t0 + np.cumsum(gaps)
    for i, (keys, n) in enumerate(reqs):
        while time.perf_counter() < arrivals[i]:
            for rid in list(pending):
                m, info = pkg.shk_server_poll(srv, rid)
                if info["done"]:
                    collect(rid, m, info)
            time.sleep(0.0005)
        pending[pkg.shk_server_submit(srv, keys, n, BUCKET, leaf_mode=mode)] = i
    for rid in list(pending):
        m, info = pkg.shk_server_wait(srv, rid)
        collect(rid, m, info)
    st = pkg.shk_server_get_stats(srv)
    pkg.shk_server_destroy(srv)
    lat = np.array([(infos[i]["finish_ns"] - infos[i]["submit_ns"]) / 1e6 for i in range(R)])
    ok = all(infos[i]["status"] == 0 for i in range(R))
    span = (max(i["finish_ns"] for i in infos.values()) - min(i["submit_ns"] for i in infos.values())) / 1e9
    total = int(sum(k.numel() for k, _ in reqs))
    spans = sorted(x for x in spans if x[1] > x[0])
    busy = sum(b - a for a, b in spans)
    overlapping = sum(1 for j, (a, b) in enumerate(spans) if any(a < d and c < b for c, d in spans[:j]))
    rec = {"workload": "served_builds_poisson", "requests": R, "sizes": f"log-uniform [1e3, {max_keys:.0e}]",
           "leaf_sizes": [48, 58], "leaf_mode": "rf" if rf else "plain", "bucket_size": BUCKET,
           "offered_load": "all at once" if burst else 0.8, "workers": 4,
           "keys_submitted_as": "device tensors (kept on the device)",
           "keys_per_s": total / span, "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "all_ok": ok,
           "total_keys": total, "makespan_s": span, "arrival_rate_per_s": rate,
           "calibration_s_per_key": per_key, "calibration_fixed_s": fixed,
           "peak_reserved_bytes": st["peak_in_use_bytes"],
           "leaf_kernels": {"requests_overlapping_an_earlier_one": overlapping,
                            "busy_s_summed": busy / 1e9,
                            "first_start_to_last_end_s": (spans[-1][1] - spans[0][0]) / 1e9 if spans else 0.0}}
    if check_alone:
        same = all(pkg.shk_build(k, n, BUCKET, leaf_mode=mode).serialize() == blobs[i]
                   for i, (k, n) in enumerate(reqs))
        rec["all_equal_to_alone"] = bool(same)
    return rec


def run_serve(args):
    """The served-builds workload alone (serve_run) as one JSON line."""
    import torch

    import paper_2308_09561_gb300 as pkg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pkg.load_library()
    with ClockSampler(local) as clk:
        rec = serve_run(pkg, args.requests, args.max_keys, args.serve_rf, rank)
    line = {"metric": "served MPHF builds: aggregate keys/s, p50/p99 latency", "value": rec["keys_per_s"],
            "unit": "keys/s", "n_gpus": ws, "steps": 1, "warmup": 2, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic", "config": {"workload": rec["workload"]}, **rec}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_u64(args):
    """The 10^6-key, leaf-48 build alone (its sub-record as one JSON line), for
    profiling runs of the plain leaf kernel."""
    import torch

    import paper_2308_09561_gb300 as pkg

    torch.cuda.set_device(_dist()[2])
    pkg.load_library()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * 32 * float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    cfg = {}
    if args.leaf_cfg:
        u, w, r = (int(v) for v in args.leaf_cfg.split(","))
        cfg = {"seeds_per_lane": u, "warps_per_block": w, "key_unroll": r, "chunk_passes": 8}
    global N_KEYS
    N_KEYS = args.keys or N_KEYS
    rec, _ = u64_subrecord(pkg, args, flush, torch.cuda.current_stream(), peak, cfg)
    if args.oracle_full:
        # cpu_baseline leg: the oracle's whole build of the same keys on every
        # host core, and its bytes against the GPU build's
        import shk_inputs

        import oracle

        keys = shk_inputs.distinct_u64(N_KEYS, KEY_SEED)
        gpu_blob = pkg.shk_build(keys, LEAF, BUCKET).serialize()
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        orc_blob = oracle.build_mphf(keys, n=LEAF, b=BUCKET, nthreads=cores)
        orc_s = time.perf_counter() - t
        rec["cpu_baseline_full"] = {"value": N_KEYS / orc_s, "unit": "keys/s", "cores": cores, "kind": "oracle",
                                    "seconds": orc_s, "sample": "the whole workload (all keys, all leaves)",
                                    "bytes_equal_to_gpu_build": orc_blob == gpu_blob}
    print(json.dumps(rec), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (sampled parity and cpu_baseline)")
    ap.add_argument("--no-subrecords", action="store_true", help="skip the 10^6-key sub-record")
    ap.add_argument("--ref-leaves", type=int, default=16,
                    help="reference arm: leaves of the workload the oracle searches per step")
    ap.add_argument("--parity-buckets", type=int, default=50, help="oracle leg: buckets compared")
    ap.add_argument("--parity-leaves", type=int, default=64, help="oracle leg: leaves compared")
    ap.add_argument("--keys", type=int, default=None,
                    help="key (leafbatch: leaf) count other than the workload's own, for profiling runs")
    ap.add_argument("--oracle-full", action="store_true",
                    help="workload u64: also time the oracle's whole build of the same keys on all host cores")
    ap.add_argument("--compare-per-bucket", action="store_true",
                    help="time the one-launch-per-bucket form on all 10^6 keys (slow)")
    ap.add_argument("--leaf-cfg", default="",
                    help="plain builds: fix the leaf kernel configuration 'U,W,R' (seeds per lane, warps "
                         "per block, key unroll) instead of the autotuner's (for profiling runs)")
    ap.add_argument("--requests", type=int, default=100, help="serve: number of requests")
    ap.add_argument("--max-keys", type=float, default=3e5,
                    help="serve: largest request (sizes log-uniform from 1e3; 1e7 in the full stream)")
    ap.add_argument("--serve-rf", action="store_true", help="serve: rotation-fitting leaves")
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="headline run: requests of its served-builds sub-record (rotation fitting)")
    ap.add_argument("--serve-max-keys", type=float, default=1e6,
                    help="headline run: largest request of its served-builds sub-record")
    ap.add_argument("--eps-num", type=int, default=STR_EPS,
                    help="headline: retrieval overhead eps = eps_num / 65536 (0: the library default, "
                         "164 (0.25 %%) for the 128-bit rows of leaf size 64)")
    ap.add_argument("--leafbatch-rf", dest="workload_leafbatch_rf", action="store_true",
                    help="leafbatch: rotation fitting (shk_leaf_search_rf)")
    ap.add_argument("--leaf-mode", default="rf", choices=["rf", "plain"],
                    help="headline / leafbatch workloads: rotation fitting or plain leaves")
    ap.add_argument("--workload", default="build", choices=["build", "u64", "leafbatch", "serve"],
                    help="build: the 10^8-string headline; u64: the 10^6-key leaf-48 build alone; "
                         "leafbatch: 65,536 independent leaves of 40..64 keys; serve: served builds")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "leafbatch":
        return run_leafbatch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "u64":
        return run_u64(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
