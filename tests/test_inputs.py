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


def test_torch_string_generator_equals_numpy():
    """The device generator of the string workload gives the numpy bytes and
    offsets bit for bit (run here on torch's CPU device, small chunks so the
    chunk seams are crossed)."""
    import numpy as np

    for count, seed in [(1, 4), (1000, 4), (3333, 9)]:
        data, offs = inp.ascii_strings(count, seed)
        td, to = inp.ascii_strings_torch(count, seed, device="cpu", chunk=4096)
        assert np.array_equal(td.numpy(), data)
        assert np.array_equal(to.numpy().view(np.uint64), offs)


@pytest.mark.gpu
def test_torch_string_generator_on_the_gpu_equals_numpy():
    import torch

    assert torch.cuda.is_available()
    data, offs = inp.ascii_strings(200000, 4)
    td, to = inp.ascii_strings_torch(200000, 4, device="cuda", chunk=1 << 20)
    assert np.array_equal(td.cpu().numpy(), data)
    assert np.array_equal(to.cpu().numpy().view(np.uint64), offs)
