"""The device-side input stream equals the host stream (same keys on both)."""
from __future__ import annotations

import numpy as np
import pytest

import shk_inputs as inp


@pytest.mark.parametrize("seed", [2, 5, 77, 2**64 - 7])
def test_torch_stream_equals_host_stream(seed):
    want = inp.distinct_u64(50000, seed)
    got = inp.splitmix64_stream_torch(seed, 50000, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(got, want)
    tail = inp.splitmix64_stream(seed, 1000, start=123456)
    got2 = inp.splitmix64_stream_torch(seed, 1000, start=123456, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(got2, tail)


@pytest.mark.gpu
def test_torch_stream_on_the_gpu_equals_host_stream():
    import torch

    assert torch.cuda.is_available()
    got = inp.splitmix64_stream_torch(5 + 7919, 200000, device="cuda").cpu().numpy().view(np.uint64)
    assert np.array_equal(got, inp.distinct_u64(200000, 5 + 7919))
