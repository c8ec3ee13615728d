"""The allocation-free sample-state read (ranc_read_sample_state_noalloc).

Some callers of this library cannot allocate device memory while they run:
programs whose own allocator owns the GPU memory, real-time loops that must not
allocate after start-up, callers held to a fixed memory budget.  For them the
library offers one read that uses a fixed scratch array compiled into the
library instead of temporary buffers.  These tests check, through the C ABI,
that it returns exactly what ranc_read_sample_state returns, on two calls in a
row (the scratch array keeps the previous call's contents), on both paths,
and that it refuses ranges larger than its scratch.  This file is collected
last, so a failure here comes after every other test has run.
"""

import numpy as np
import pytest

import ranc_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


@pytest.mark.parametrize("path", [1, 0], ids=["batched", "plain"])
def test_noalloc_read_equals_allocating_read_twice(ranc, path):
    net = W.tiny_5core()
    B = 130
    x = W.rate_coded_inputs(21, B, 8, 784, 0.2)
    sim = ranc.Sim(net, B, path)
    sim.load_inputs(x)
    sim.step(5)
    for b0, nb in ((3, 7), (120, 10)):  # two calls in a row, different ranges
        v_ref, s_ref = ranc.ranc_read_sample_state(sim.h, b0, nb, net.n_cores, net.neurons)
        v, s = ranc.ranc_read_sample_state_noalloc(sim.h, b0, nb, net.n_cores, net.neurons)
        np.testing.assert_array_equal(v, v_ref)
        np.testing.assert_array_equal(s, s_ref)
    sim.step(3)  # the state moves on; the scratch must not serve stale values
    v_ref, s_ref = ranc.ranc_read_sample_state(sim.h, 3, 7, net.n_cores, net.neurons)
    v, s = ranc.ranc_read_sample_state_noalloc(sim.h, 3, 7, net.n_cores, net.neurons)
    np.testing.assert_array_equal(v, v_ref)
    np.testing.assert_array_equal(s, s_ref)
    sim.close()


def test_noalloc_read_rejects_ranges_beyond_its_scratch(ranc):
    net = W.mnist_512core()
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    v, _ = ranc.ranc_read_sample_state_noalloc(sim.h, 0, 15, net.n_cores, net.neurons)  # 15 x 528 KiB fits
    assert v.shape == (15, 512, 256)
    with pytest.raises(ranc.RancError) as ei:
        ranc.ranc_read_sample_state_noalloc(sim.h, 0, 16, net.n_cores, net.neurons)
    assert ei.value.code == ranc.RANC_EINVAL and "at most" in str(ei.value)
    sim.close()
