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

import os

import numpy as np
import pytest

import ranc_workloads as W
from parity_util import idle_core_ticks, unpack_spikes

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


def test_noalloc_read_first_inside_a_deferred_period(ranc, oracle_mod):
    """A feed-forward net whose second-layer cores fall idle in an input gap,
    so their idle ticks are deferred.  The first read of the handle is the
    allocation-free one, in the middle of that deferred period: it must apply
    the deferred ticks itself and return the oracle's potentials and spikes.
    A second allocation-free call later (the scratch array still holds the
    first call's contents) must equal both the oracle and the allocating read.
    The allocation-free calls make no device allocation; the allocating read
    does."""
    net = W.layered_net(63)
    B, T, t_read = 260, 20, 10
    x = W.rate_coded_inputs(29, B, 12, net.n_inputs, 0.3)
    x[:, 2:12] = 0
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=os.cpu_count() or 1)
    idle = idle_core_ticks(net, x, ref, T)
    assert idle[t_read - 2:t_read + 1, 2:4].all()  # cores 2-3 idle for the three ticks up to the read
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    sim.step(t_read + 1)
    ranges = ((0, 7), (129, 13))
    n0 = ranc.ranc_device_allocations()
    for b0, nb in ranges:
        v, s = ranc.ranc_read_sample_state_noalloc(sim.h, b0, nb, net.n_cores, net.neurons)
        np.testing.assert_array_equal(v, ref["v_trace"][b0:b0 + nb, t_read])
        np.testing.assert_array_equal(unpack_spikes(s, net.neurons), ref["spike_trace"][b0:b0 + nb, t_read])
    assert ranc.ranc_device_allocations() == n0
    _, dfr = ranc.ranc_item_ticks(sim.h)
    assert dfr > 0
    sim.step(T - t_read - 1)
    n1 = ranc.ranc_device_allocations()
    v, s = ranc.ranc_read_sample_state_noalloc(sim.h, 129, 13, net.n_cores, net.neurons)
    assert ranc.ranc_device_allocations() == n1
    np.testing.assert_array_equal(v, ref["v_trace"][129:142, T - 1])
    v_ref, s_ref = ranc.ranc_read_sample_state(sim.h, 129, 13, net.n_cores, net.neurons)
    assert ranc.ranc_device_allocations() > n1
    np.testing.assert_array_equal(v, v_ref)
    np.testing.assert_array_equal(s, s_ref)
    sim.close()
