"""The C-ABI library loads and exports every function include/*.h declares
(no compute calls: these run without a GPU)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(shk_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2308_09561_gb300 import build_ext

    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("shk_build", "shk_query", "shk_serialize", "shk_deserialize", "shk_size_bits",
                 "shk_free", "shk_last_error", "shk_leaf_search", "shk_build_stats"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_the_abi(lib):
    import paper_2308_09561_gb300 as pkg

    pkg.load_library()
    for name in _declared():
        assert callable(getattr(pkg, name)), name
    assert pkg.shk_version() == "SHKRS002"


def test_host_side_argument_errors_without_gpu(lib):
    """Argument checks happen before any device call."""
    import paper_2308_09561_gb300 as pkg

    pkg.load_library()
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_deserialize(b"\0" * 64)
    assert e.value.status in (pkg.SHK_EFORMAT,)
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_deserialize(b"\0" * 130)
    assert e.value.status == pkg.SHK_EFORMAT


def test_binding_rejects_keys_of_the_wrong_element_size():
    """The binding describes keys by their bytes; an array of another element
    size is refused rather than reinterpreted."""
    import numpy as np

    import paper_2308_09561_gb300 as pkg

    with pytest.raises(ValueError):
        pkg._as_keys(np.zeros(4, np.uint32), pkg.SHK_KEYS_U64)
    with pytest.raises(ValueError):
        pkg._as_keys(np.zeros(3, np.uint64), pkg.SHK_KEYS_FP128)
    with pytest.raises(ValueError):
        pkg._as_keys(np.zeros(8, np.uint64), pkg.SHK_KEYS_STR, np.array([0, 8], np.uint64))
    with pytest.raises(ValueError):
        pkg._as_keys(np.zeros(2, np.uint64), 7)
    k, _ = pkg._as_keys(np.zeros(6, np.uint64), pkg.SHK_KEYS_FP128)
    assert k.n_keys == 3 and k.on_device == 0
    k, _ = pkg._as_keys(np.zeros(10, np.uint8), pkg.SHK_KEYS_STR, np.array([0, 4, 10], np.uint64))
    assert k.n_keys == 2


def test_missing_library_raises():
    """Without the built library every call raises: there is no fallback."""
    import subprocess
    import sys

    code = ("import paper_2308_09561_gb300 as p\n"
            "try:\n"
            "    p.load_library('/nonexistent/libshk_gpu.so')\n"
            "except p.ShkError as e:\n"
            "    print('raised', e.status)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "raised 4"


def test_compute_calls_fail_loudly_without_a_device(lib):
    """On a machine without a CUDA device a build raises (the stream lookup or
    the library reports the missing device) instead of computing anything
    elsewhere; with an explicit stream handle the library itself reports
    SHK_ECUDA."""
    import numpy as np
    import torch

    import paper_2308_09561_gb300 as pkg

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    pkg.load_library()
    keys = np.arange(1, 1001, dtype=np.uint64)
    with pytest.raises(RuntimeError):
        pkg.shk_build(keys, 16, 100)
    with pytest.raises(pkg.ShkError) as e:
        pkg.shk_build(keys, 16, 100, stream=0)
    assert e.value.status == pkg.SHK_ECUDA


def test_leaf_configuration_table_without_gpu(lib):
    """The autotuner's configuration table is host data: every entry is a
    supported shape (seeds per lane 1-4, warps per block a power of two up
    to 16, key unroll 1-4), and the configuration the tuner picks on GB300
    for 48-key leaves (4 seeds, 8 warps, unroll 4) is one of them."""
    import paper_2308_09561_gb300 as pkg

    pkg.load_library()
    cfgs = pkg.shk_leaf_configs()
    assert len(cfgs) == len(set(cfgs)) >= 4
    for u, w, r in cfgs:
        assert 1 <= u <= 4 and w in (4, 8, 16) and 1 <= r <= 4
    assert (4, 8, 4) in cfgs


def test_oracle_and_cuda_path_share_no_code():
    """The oracle and the CUDA library are independent: neither side imports,
    includes or builds the other's sources."""
    import glob as _glob

    pkg_dir = os.path.join(ROOT, "paper_2308_09561_gb300")
    oracle_dir = os.path.join(ROOT, "oracle")
    for path in _glob.glob(os.path.join(pkg_dir, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".c")) and "_build" not in path:
            text = open(path).read()
            assert "oracle" not in text.lower(), path
    for path in _glob.glob(os.path.join(oracle_dir, "*.*")):
        if path.endswith((".py", ".c", ".h")):
            text = open(path).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2308_09561_gb300", text, flags=re.M), path
            assert not re.search(r'#\s*include\s*"[^"]*(csrc|shk_internal|kernels|shk\.h)', text), path


def test_noalloc_binding_rejects_short_or_narrow_outputs_before_any_launch():
    """shk_leaf_search_noalloc writes n_leaves 8-byte words into its outputs on
    the device: the binding refuses outputs that are too short or too narrow,
    and offsets of the wrong type, before the library is called (CPU tensors
    here, so any call that got through would fail on the device check last)."""
    import torch

    import paper_2308_09561_gb300 as pkg

    keys = torch.zeros(40, dtype=torch.int64)
    off = torch.tensor([0, 10, 20, 30, 40], dtype=torch.int32)
    with pytest.raises(ValueError, match="fewer than the 4 leaves"):
        pkg.shk_leaf_search_noalloc(keys, off, torch.empty(3, dtype=torch.int64))
    with pytest.raises(ValueError, match="int64"):
        pkg.shk_leaf_search_noalloc(keys, off, torch.empty(4, dtype=torch.int32))
    with pytest.raises(ValueError, match="f_out holds"):
        pkg.shk_leaf_search_noalloc(keys, off, torch.empty(4, dtype=torch.int64),
                                    f_out=torch.empty(2, dtype=torch.int64))
    with pytest.raises(ValueError, match="int32"):
        pkg.shk_leaf_search_noalloc(keys, off.to(torch.int64), torch.empty(4, dtype=torch.int64))
    with pytest.raises(ValueError, match="8-byte"):
        pkg.shk_leaf_search_noalloc(keys.to(torch.int32), off, torch.empty(4, dtype=torch.int64))
    with pytest.raises(ValueError, match="device tensors"):
        pkg.shk_leaf_search_noalloc(keys, off, torch.empty(4, dtype=torch.int64))


def test_binding_status_and_enum_constants_match_the_header():
    """Every SHK_ constant the header's enums define has the same value in the
    binding."""
    import paper_2308_09561_gb300 as pkg

    text = open(os.path.join(ROOT, "include", "shk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = 0
    for m in re.finditer(r"typedef enum \{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(SHK_\w+)\s*=\s*(\d+)", m.group(1)):
            assert getattr(pkg, name) == int(val), name
            found += 1
    assert found >= 17
