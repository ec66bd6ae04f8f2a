"""Pins of the oracle's closed forms for the Blackwell instruction probes:
brute-force enumeration of what each thread loads from tensor memory, and
the accumulation of n MMAs of all-ones operands done step by step in FP32."""
import numpy as np
import pytest

import oracle as O


def _brute_tmem(iters, store):
    # lane l, column c hold l * 512 + c (after a store pass p: + p); thread t
    # of warp w reads lane 32 (w % 4) + t % 32, columns 256 (w // 4) .. + 255
    out = np.zeros(256, dtype=np.uint64)
    for t in range(256):
        w = t // 32
        lane = 32 * (w % 4) + t % 32
        cols = range(256 * (w // 4), 256 * (w // 4) + 256)
        if store:
            s = sum(lane * 512 + c + (iters - 1) for c in cols)
        else:
            s = iters * sum(lane * 512 + c for c in cols)
        out[t] = s % (1 << 32)
    return out.astype(np.uint32)


@pytest.mark.parametrize("iters,store", [(1, False), (7, False), (300, False), (1, True), (5, True), (1 << 20, False)])
def test_tmem_probe_sums_brute_force(iters, store):
    assert np.array_equal(O.tmem_probe_sums(iters, store), _brute_tmem(iters, store))


@pytest.mark.parametrize("dt,k", [(0, 8), (1, 16), (2, 32)])
def test_mma_probe_value_step_by_step(dt, k):
    # n MMAs each adding a K-deep dot product of ones into an FP32 accumulator
    for n in (1, 3, 1000, 1 << 15):
        acc = np.float32(0)
        step = np.float32(sum(np.float32(1) * np.float32(1) for _ in range(k)))
        for _ in range(n):
            acc = np.float32(acc + step)
        assert O.mma_probe_value(n, dt) == acc
