"""Benchmark: MPHF builds of 10^6 uniform 64-bit keys (splitmix64 stream seed 2),
leaf size 48, bucket size 2000, on one GB300 per rank.

A step is one whole build (fingerprints, bucket partition, splitting trees,
leaf seed search, orientation, Golomb-Rice/Elias-Fano encoding, retrieval
solve) from keys resident in HBM to the encoded MPHF in HBM.  Prints one JSON
line (rank 0).  Ranks build independent key sets (weak scaling, no collective
on the data path).

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

N_KEYS, LEAF, BUCKET, KEY_SEED = 1_000_000, 48, 2000, 2
WORKLOAD = "mphf_build_1M_u64_keys_leaf48_bucket2000"
METRIC = "MPHF build keys/s (1M u64 keys, leaf 48, bucket 2000), leaf seeds tested/s, % integer-issue roofline"
# integer lane-operations of one key-seed evaluation of the leaf hash + filter:
# xor 1, multiply-add 1, widening multiply by m 1, multiply-high by m-1 1,
# h1 adjust 2 (compare, add), two candidate bits into the mask: 8 when the mask
# is two 32-bit words (2 subtracts, 4 shifts, 2 ors; m > 32), 3 for m <= 32
OPS_PER_EVAL_WIDE = 14
LEAF_TRAFFIC_PER_LEAF = 920_576 / 2_100  # DRAM bytes per leaf of the leaf kernel, measured with ncu
OPS_PER_EVAL_NARROW = 9


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


def _cpu_baseline(sample_keys: int, reps: int = 1, single_keys: int = 0):
    """The oracle as it stands on the host cores, on the first sample_keys keys
    of the same stream (same leaf and bucket size).  With single_keys > 0 it is
    also timed on one thread over the first single_keys keys."""
    import oracle

    oracle.build()
    import shk_inputs

    keys = shk_inputs.distinct_u64(max(sample_keys, single_keys), KEY_SEED)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    for _ in range(reps):
        oracle.build_mphf(keys[:sample_keys], n=LEAF, b=BUCKET, nthreads=cores)
    dt = time.perf_counter() - t
    out = {"value": sample_keys * reps / dt, "unit": "keys/s", "cores": cores, "kind": "oracle",
           "sample": f"first {sample_keys} keys of the same stream ({(sample_keys + BUCKET - 1) // BUCKET} buckets), "
                     f"leaf 48, bucket 2000, OpenMP over buckets, {reps} build(s), {dt:.1f} s"}
    if single_keys:
        t = time.perf_counter()
        oracle.build_mphf(keys[:single_keys], n=LEAF, b=BUCKET, nthreads=1)
        dt1 = time.perf_counter() - t
        out["single_thread"] = {"value": single_keys / dt1, "unit": "keys/s",
                                "sample": f"first {single_keys} keys, one thread, {dt1:.1f} s"}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    sample = args.ref_sample_keys
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps would only add minutes
    t = time.perf_counter()
    base = None
    for _ in range(args.steps):
        base = _cpu_baseline(sample)
    dt = time.perf_counter() - t
    value = sample * args.steps / dt
    base["value"] = value
    line = {"metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "keys": N_KEYS, "leaf_size": LEAF, "bucket_size": BUCKET,
                       "sample_keys": sample},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    global N_KEYS
    N_KEYS = args.keys or N_KEYS
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2308_09561_gb300 as pkg
    import shk_inputs

    pkg.load_library()
    keys = shk_inputs.distinct_u64(N_KEYS, rank_key_seed(rank))
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    host_keys = torch.from_numpy(keys.view(np.int64)).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    cfg = {}
    if args.leaf_cfg:
        u, w, r = (int(v) for v in args.leaf_cfg.split(","))
        cfg = {"seeds_per_lane": u, "warps_per_block": w, "key_unroll": r, "chunk_passes": 8}

    def step(profile=True):
        m = pkg.shk_build(dkeys, LEAF, BUCKET, profile=profile, **cfg)
        st = m.stats()
        m.close()
        return st

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    stats = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            stats.append(step())
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_sum = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    value = N_KEYS * ws * args.steps / t_sum

    # end to end through the public API: pinned host keys in, serialized MPHF out
    e2e_ms = []
    blob_bytes = 0
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        m = pkg.shk_build(host_keys, LEAF, BUCKET, **cfg)
        blob = m.serialize()
        e2e_ms.append(1e3 * (time.perf_counter() - t))
        blob_bytes = len(blob)
        m.close()
    e2e_value = N_KEYS * ws / (np.mean(e2e_ms) / 1e3)

    leaf_ms = np.mean([s["ms_leaf"] for s in stats])
    seeds_min = stats[-1]["leaf_seeds_min"]
    evals = stats[-1]["leaf_key_evals"]
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tops = sms * 4 * 32 * sm_max_mhz * 1e6 / 1e12
    achieved_tops = evals * OPS_PER_EVAL_WIDE / (leaf_ms / 1e3) / 1e12
    clocks = clk.summary()
    # the plain form: one leaf-search launch per bucket, one warp per leaf, on a
    # prefix of the same keys (the whole workload with --compare-per-bucket)
    cmp_keys = N_KEYS if args.compare_per_bucket else min(N_KEYS, 100_000)
    ck = dkeys[:cmp_keys]
    t_cmp = {}
    for name, sched in (("persistent", pkg.SHK_SCHED_PERSISTENT), ("per_bucket", pkg.SHK_SCHED_PER_BUCKET)):
        m = pkg.shk_build(ck, LEAF, BUCKET, sched=sched, profile=True, **cfg)
        st = m.stats()
        t_cmp[name] = st
        m.close()
    # rotation fitting with partial hash calculation (leaf mode 1) on the same keys
    rf_stats = []
    for _ in range(3):
        m = pkg.shk_build(dkeys, LEAF, BUCKET, leaf_mode=pkg.SHK_LEAF_ROTATION, profile=True)
        rf_stats.append(m.stats())
        rf_bytes = len(m.serialize())
        m.close()
    rf_ms = float(np.median([s["ms_total"] for s in rf_stats]))
    rotation = {"keys_per_s": N_KEYS / (rf_ms / 1e3), "ms_total": rf_ms,
                "ms_leaf": float(np.median([s["ms_leaf"] for s in rf_stats])),
                "leaf_candidates_per_s": rf_stats[-1]["leaf_seeds_min"] / (rf_stats[-1]["ms_leaf"] / 1e3),
                "bits_per_key": 8 * rf_bytes / N_KEYS,
                "note": "candidates = sum over leaves of (v+1), v = seed*m + rotation"}
    # queries: every key of the workload, device in and out, L2 flushed before each pass
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
    query = {"keys_per_s": N_KEYS / (float(np.median(q_ms)) / 1e3), "ms": float(np.median(q_ms)),
             "note": "shk_query over all keys (fingerprint, bucket, tree descent through the query "
                     "index built by the first query, retrieval parity)"}
    per_bucket = {"keys": cmp_keys, "persistent_ms_leaf": t_cmp["persistent"]["ms_leaf"],
                  "per_bucket_ms_leaf": t_cmp["per_bucket"]["ms_leaf"],
                  "per_bucket_leaf_launches": t_cmp["per_bucket"]["leaf_launches"],
                  "speedup_leaf": t_cmp["per_bucket"]["ms_leaf"] / t_cmp["persistent"]["ms_leaf"],
                  "speedup_build": t_cmp["per_bucket"]["ms_total"] / t_cmp["persistent"]["ms_total"]}
    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "keys": N_KEYS, "leaf_size": LEAF, "bucket_size": BUCKET,
                   "key_stream_seed": KEY_SEED, "schedule": "persistent",
                   "l2": "256 MB buffer written between timed steps (flush), outside the step events",
                   "parallelism": f"replicas x{ws}"},
        "leaf_seeds_per_s": seeds_min / (leaf_ms / 1e3),
        "leaf_seeds_per_s_build": seeds_min * ws * args.steps / t_sum,
        "key_seed_evals_per_s": evals / (leaf_ms / 1e3),
        "bits_per_key": 8 * blob_bytes / N_KEYS,
        "phase_ms": {k: float(np.mean([s[k] for s in stats])) for k in
                     ("ms_fingerprint", "ms_partition", "ms_split", "ms_leaf", "ms_orient", "ms_encode",
                      "ms_ribbon", "ms_total")},
        "roofline": {"bound": "alu", "kernel": "k_leaf_persistent", "achieved": achieved_tops,
                     "peak": peak_tops, "unit": "T int-lane-ops/s", "frac": achieved_tops / peak_tops,
                     # ncu dram read + write of k_leaf_persistent<4,8,4> on the 10^5-key build
                     # (920.6 KB over 2,100 leaves), scaled by the leaves of this launch
                     "traffic": LEAF_TRAFFIC_PER_LEAF * stats[-1]["n_leaves"],
                     "traffic_note": "scaled by leaves from an ncu capture of the 10^5-key build",
                     "ops_per_launch": evals * OPS_PER_EVAL_WIDE,
                     "peak_note": f"{sms} SMs x 4 schedulers x 32 lanes x {sm_max_mhz:.0f} MHz (max SM clock)"},
        "e2e": {"value": e2e_value, "unit": "keys/s", "h2d_bytes_per_step": N_KEYS * 8,
                "d2h_bytes_per_step": blob_bytes},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "leaf_kernel_cfg": stats[-1]["leaf_cfg"],
        "persistent_vs_per_bucket": per_bucket,
        "rotation_fitting": rotation,
        "query": query,
        "wall_s_timed": wall,
    }
    if clocks:
        line["clocks"] = clocks
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(24000, single_keys=4000)
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
                         "unit": "T int-lane-ops/s", "frac": ach / peak}}
    if not rf:
        line["tuned_cfg"] = pkg.shk_leaf_tune(64)
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Served builds: a Poisson stream of MPHF build requests (uniform u64
    keys, sizes log-uniform in [1e3, max_keys], leaf size 48 or 58 by coin,
    bucket 2000, stream seed 5, request i from sub-seed 5 + 7919 i) into one
    server with 4 builds in flight; plain or rotation-fitting leaves.  The
    arrival rate is set for ~80 % offered load from a calibration build of
    each leaf size.  Reports p50/p99 build latency (submit to finish) and
    aggregate keys/s."""
    import torch

    import paper_2308_09561_gb300 as pkg
    import shk_inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pkg.load_library()
    R = args.requests
    u = shk_inputs.uniform01(5 + 1000 * rank, 3 * R)
    sizes = np.floor(10 ** (3 + np.log10(args.max_keys / 1e3) * u[0::3])).astype(np.int64)
    mode = pkg.SHK_LEAF_ROTATION if args.serve_rf else pkg.SHK_LEAF_PLAIN
    leafs = np.where(u[1::3] < 0.5, 48, 58)
    # request keys are generated on the device (the same keys as distinct_u64)
    reqs = [(shk_inputs.splitmix64_stream_torch(5 + 7919 * i + 1000003 * rank, int(sz), device="cuda"), int(n))
            for i, (sz, n) in enumerate(zip(sizes, leafs))]
    torch.cuda.synchronize()
    # calibration: seconds per key of a build at each leaf size
    per_key = {}
    for n in (48, 58):
        k = shk_inputs.distinct_u64(60000, 77 + n)
        pkg.shk_build(k, n, BUCKET, leaf_mode=mode).close()  # tuning / warm-up
        t = time.perf_counter()
        pkg.shk_build(k, n, BUCKET, leaf_mode=mode).close()
        per_key[n] = (time.perf_counter() - t) / k.size
    service = float(np.mean([k.numel() * per_key[n] for k, n in reqs]))
    rate = 0.8 / service
    gaps = -np.log(1.0 - shk_inputs.uniform01(55 + 1000 * rank, R)) / rate
    srv = pkg.shk_server_create(0, 4)
    pending, infos = {}, []
    t0 = time.perf_counter()
    arrivals = t0 + np.cumsum(gaps)
    with ClockSampler(local) as clk:
        for i, (keys, n) in enumerate(reqs):
            while time.perf_counter() < arrivals[i]:
                for rid in list(pending):
                    m, info = pkg.shk_server_poll(srv, rid)
                    if info["done"]:
                        infos.append(info)
                        pending.pop(rid)
                        if m is not None:
                            m.close()
                time.sleep(0.0005)
            pending[pkg.shk_server_submit(srv, keys, n, BUCKET, leaf_mode=mode)] = i
        for rid in list(pending):
            m, info = pkg.shk_server_wait(srv, rid)
            infos.append(info)
            if m is not None:
                m.close()
    st = pkg.shk_server_get_stats(srv)
    pkg.shk_server_destroy(srv)
    lat = np.array([(i["finish_ns"] - i["submit_ns"]) / 1e6 for i in infos])
    ok = all(i["status"] == 0 for i in infos)
    span = (max(i["finish_ns"] for i in infos) - min(i["submit_ns"] for i in infos)) / 1e9
    total = int(sum(k.numel() for k, _ in reqs))
    line = {"metric": "served MPHF builds: aggregate keys/s, p50/p99 latency", "value": total / span,
            "unit": "keys/s", "n_gpus": ws, "steps": 1, "warmup": 2, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "served_builds_poisson", "requests": R,
                       "sizes": f"log-uniform [1e3, {args.max_keys:.0e}]", "leaf_sizes": [48, 58],
                       "leaf_mode": "rf" if args.serve_rf else "plain", "bucket_size": BUCKET,
                       "offered_load": 0.8, "workers": 4},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "all_ok": ok, "total_keys": total, "makespan_s": span,
            "arrival_rate_per_s": rate, "calibration_s_per_key": per_key,
            "peak_reserved_bytes": st["peak_in_use_bytes"]}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_strings(args):
    """10^8 random strings (length uniform in [10, 50], bytes uniform in
    [1, 127], stream seed 4) hashed to 128-bit fingerprints, leaf size 64,
    bucket size 2000, rotation fitting with partial hash calculation.  One
    timed build (after a warm-up build of the first 10^6 strings), then every
    key is queried and the ranks checked to be a permutation of [0, N)."""
    import torch

    import paper_2308_09561_gb300 as pkg
    import shk_inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pkg.load_library()
    count = args.keys or 100_000_000
    t = time.perf_counter()
    data, offs = shk_inputs.ascii_strings(count, 4 + 1000 * rank)
    gen_s = time.perf_counter() - t
    ddata = torch.from_numpy(data).cuda()
    doffs = torch.from_numpy(offs.view(np.int64)).cuda()
    leaf, mode = 64, (pkg.SHK_LEAF_ROTATION if args.leaf_mode == "rf" else pkg.SHK_LEAF_PLAIN)
    w = min(count, 1_000_000)
    eps = args.eps_num
    pkg.shk_build(ddata, leaf, BUCKET, kind=pkg.SHK_KEYS_STR, str_offsets=doffs[:w + 1], leaf_mode=mode,
                  eps_num=eps).close()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        m = pkg.shk_build(ddata, leaf, BUCKET, kind=pkg.SHK_KEYS_STR, str_offsets=doffs, leaf_mode=mode,
                          eps_num=eps, profile=True)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = m.stats()
    blob = m.serialize()
    tq = time.perf_counter()
    ranks = m.query(ddata, kind=pkg.SHK_KEYS_STR, str_offsets=doffs)
    torch.cuda.synchronize()
    query_s = time.perf_counter() - tq
    srt, _ = torch.sort(ranks)
    bij = bool(torch.equal(srt, torch.arange(count, device="cuda", dtype=torch.int64)))
    del srt, ranks
    m.close()
    # fingerprint + radix partition bytes: read the strings and their
    # offsets, write one 16-byte fingerprint per key; the scatter reads it
    # and writes it into its bucket
    part_bytes = data.size + 8 * (count + 1) + 16 * count + 32 * count
    part_ms = st["ms_fingerprint"] + st["ms_partition"]
    line = {"metric": "MPHF build keys/s, 10^8 string keys, leaf 64", "value": count / (ms / 1e3),
            "unit": "keys/s", "n_gpus": ws, "steps": 1, "warmup": 1, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "mphf_build_1e8_strings_leaf64_bucket2000", "keys": count,
                       "string_bytes": int(data.size), "leaf_size": leaf, "bucket_size": BUCKET,
                       "leaf_mode": args.leaf_mode, "eps_num": eps or "default"},
            "bits_per_key": 8 * len(blob) / count, "bijection": bij, "query_s_all_keys": query_s,
            "phase_ms": {k: st[k] for k in ("ms_fingerprint", "ms_partition", "ms_split", "ms_leaf",
                                            "ms_orient", "ms_encode", "ms_ribbon", "ms_total")},
            "partition_gbs": part_bytes / (part_ms / 1e3) / 1e9,
            "leaf_candidates_per_s": st["leaf_seeds_min"] / (st["ms_leaf"] / 1e3),
            "leaves": st["n_leaves"], "input_generation_s": gen_s}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample-keys", type=int, default=24000,
                    help="reference arm: keys of the workload's stream the oracle builds per step")
    ap.add_argument("--keys", type=int, default=None,
                    help="key (leafbatch: leaf) count other than the workload's own, for profiling runs")
    ap.add_argument("--compare-per-bucket", action="store_true",
                    help="time the one-launch-per-bucket form on the whole workload (slow)")
    ap.add_argument("--leaf-cfg", default="",
                    help="build: fix the leaf kernel configuration 'U,W,R' (seeds per lane, warps per "
                         "block, key unroll) instead of the autotuner's (for profiling runs)")
    ap.add_argument("--requests", type=int, default=100, help="serve: number of requests")
    ap.add_argument("--max-keys", type=float, default=3e5,
                    help="serve: largest request (sizes log-uniform from 1e3; 1e7 in the full stream)")
    ap.add_argument("--serve-rf", action="store_true", help="serve: rotation-fitting leaves")
    ap.add_argument("--eps-num", type=int, default=983,
                    help="strings: retrieval overhead eps = eps_num / 65536 (default 983, ~1.5 %%, "
                         "for ~1.54 bits/key; 0: the library default, 3277)")
    ap.add_argument("--leafbatch-rf", dest="workload_leafbatch_rf", action="store_true",
                    help="leafbatch: rotation fitting (shk_leaf_search_rf)")
    ap.add_argument("--leaf-mode", default="rf", choices=["rf", "plain"],
                    help="strings / leafbatch workloads: rotation fitting or plain leaves")
    ap.add_argument("--workload", default="build", choices=["build", "leafbatch", "serve", "strings"],
                    help="leafbatch: 65,536 independent leaves of 40..64 keys, one graph-replayed launch")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "leafbatch":
        return run_leafbatch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "strings":
        return run_strings(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
