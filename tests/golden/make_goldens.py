"""Write the stored expected values of the full-size parity tests.

Every value here comes from the CPU oracle (oracle/) on inputs from the seeded
generators (shk_inputs); nothing is read from the CUDA library.  Run from the
repository root:  python tests/golden/make_goldens.py  (about 10 minutes on 8
cores).

  config2_build_digest.txt  SHA-256 of the oracle's serialized MPHF of the
                            10^6-key, leaf-48, bucket-2000 workload (plain and
                            rotation-fitting leaves)
  config3_leaf_sample.txt   256 leaves drawn uniformly from the 65,536-leaf
                            batch: the oracle's first passing seed and
                            orientation mask, plain and rotation fitting
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import shk_inputs as inp  # noqa: E402

CONFIG3_SAMPLE_SEED = 2308
CONFIG3_SAMPLE = 256


def config3_sample_indices() -> np.ndarray:
    return np.sort(np.random.default_rng(CONFIG3_SAMPLE_SEED).choice(65536, CONFIG3_SAMPLE, replace=False))


def write_config2(threads: int):
    keys = inp.distinct_u64(1_000_000, 2)
    lines = ["# Oracle build of the 10^6-key workload: distinct u64 keys of the splitmix64 stream from",
             "# seed 2, leaf size 48, bucket size 2000, default retrieval overhead (eps_num 3277).",
             "# Written by tests/golden/make_goldens.py from oracle/ only.",
             "# leaf_mode bytes sha256"]
    for mode in (0, 1):
        t = time.time()
        blob = oracle.build_mphf(keys, n=48, b=2000, nthreads=threads, leaf_mode=mode)
        lines.append(f"{mode} {len(blob)} {hashlib.sha256(blob).hexdigest()}")
        print(f"config 2 leaf mode {mode}: {len(blob)} bytes, {time.time() - t:.0f} s", flush=True)
    with open(os.path.join(HERE, "config2_build_digest.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def write_config3(threads: int):
    keys, offs = inp.leaf_instances(65536, 3)
    idx = config3_sample_indices()
    sizes = np.diff(offs.astype(np.int64))
    packed = np.concatenate([keys[offs[i]:offs[i + 1]] for i in idx])
    po = np.zeros(idx.size + 1, np.uint32)
    po[1:] = np.cumsum(sizes[idx])
    t = time.time()
    s, f = oracle.leaf_search_batch(packed, po, 0, nthreads=threads)
    print(f"config 3 plain: {time.time() - t:.0f} s", flush=True)
    t = time.time()
    v, fr = oracle.leaf_search_batch(packed, po, 0, nthreads=threads, rf=True)
    print(f"config 3 rotation fitting: {time.time() - t:.0f} s", flush=True)
    lines = ["# 256 leaves drawn uniformly from the 65,536-leaf batch (shk_inputs.leaf_instances(65536, 3):",
             f"# sizes 40..64), indices numpy default_rng({CONFIG3_SAMPLE_SEED}).choice(65536, 256, replace=False),",
             "# seed start 0.  Oracle values: first passing seed and orientation mask (plain leaves),",
             "# smallest v = s*m + r and its mask (rotation fitting).  Written by tests/golden/make_goldens.py.",
             "# index m seed fmask rf_value rf_fmask"]
    for j, i in enumerate(idx):
        lines.append(f"{i} {sizes[i]} {s[j]} {f[j]:x} {v[j]} {fr[j]:x}")
    with open(os.path.join(HERE, "config3_leaf_sample.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    oracle.build()
    n = os.cpu_count() or 1
    which = sys.argv[1:] or ["config3", "config2"]
    if "config3" in which:
        write_config3(n)
    if "config2" in which:
        write_config2(n)
