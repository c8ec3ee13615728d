"""Plain path (one thread per neuron) against the CPU oracle, bit for bit:
every potential, every spike and every output count, per tick on small
networks and on the 512-core workload's sampled samples."""

import os

import numpy as np
import pytest

import ranc_workloads as W
from parity_util import digest, gpu_trace, unpack_spikes

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def per_tick_parity(ranc, oracle_mod, net, x, T, path, batch=None):
    B = x.shape[0] if batch is None else batch
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, B, path)
    sim.load_inputs(x)
    v, s, d = gpu_trace(sim, T)
    np.testing.assert_array_equal(v, ref["v_trace"])
    np.testing.assert_array_equal(s, ref["spike_trace"])
    for t in range(T):
        assert d[t] == digest(ref["v_trace"][:, t]), t
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    cnt = sim.counters()
    np.testing.assert_array_equal(cnt[:4], ref["counters"][:, :4].sum(0))
    assert cnt[4] == B * T and sim.tick() == T
    sim.close()
    return ref


def test_tiny_workload_every_tick(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(net.meta["seed"], 64, 8, 784, 0.15)
    ref = per_tick_parity(ranc, oracle_mod, net, x, 9, ranc.RANC_PATH_PLAIN)
    assert ref["counters"][:, 2].sum() > 0  # the output bus saw events


SHAPES = [
    # grid, axons, neurons, types, neg_mode, delay_max, holes, v0
    ((2, 1), 32, 32, 1, 0, 1, (), (0, 0)),
    ((3, 2), 64, 96, 3, 1, 15, ((1, 1),), (-3, 3)),
    ((4, 4), 128, 64, 8, 0, 15, ((0, 3), (2, 2)), (-5, 5)),
    ((1, 3), 96, 160, 4, 1, 7, (), (0, 2)),
]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[1]}x{s[2]}k{s[3]}" for s in SHAPES])
def test_random_nets_every_tick(ranc, oracle_mod, shape):
    (gw, gh), A, N, K, neg, dmax, holes, v0 = shape
    net = W.random_net(100 + A + N, gw, gh, axons=A, neurons=N, n_types=K, neg_mode=neg, delay_max=dmax,
                       holes=holes, v0=v0, n_inputs=70, fanout_per_line=3, p_core=0.6, p_out=0.2)
    x = W.rate_coded_inputs(7, 5, 12, net.n_inputs, 0.35)
    per_tick_parity(ranc, oracle_mod, net, x, 20, ranc.RANC_PATH_PLAIN)


def test_mnist512_sampled_every_tick(ranc, oracle_mod):
    net = W.mnist_512core()
    x = W.rate_coded_inputs(net.meta["seed"], 3, 16, 784, 0.15, first_sample=4093)
    per_tick_parity(ranc, oracle_mod, net, x, 24, ranc.RANC_PATH_PLAIN)


def test_run_samples_batch1_like_the_benchmark(ranc, oracle_mod):
    """Batch 1, samples back to back through ranc_run_samples (host and
    device buffers): per-sample output counts and summed counters."""
    import torch
    net = W.mnist_512core()
    S = 6
    x = W.rate_coded_inputs(net.meta["seed"], S, 16, 784, 0.15)
    ref = oracle_mod.run(net, x, 24, n_threads=NPROC)
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    np.testing.assert_array_equal(sim.run_samples(x, 24), ref["out"])
    cnt = sim.counters()
    sim.reset()
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((S, 10), dtype=torch.int32, device="cuda")
    ranc.ranc_run_samples(sim.h, dx.data_ptr(), S, 16, 24, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref["out"])
    cnt2 = sim.counters()
    np.testing.assert_array_equal(cnt[:4], ref["counters"][:, :4].sum(0))
    np.testing.assert_array_equal(cnt2, cnt)
    sim.close()


def test_run_samples_without_the_shared_memory_shortcuts(ranc, oracle_mod):
    """The persistent window kernel's two shared-memory shortcuts both off:
    16 cores of 64 neurons per CTA with 7 sorted words each (3584 sorted
    positions: more than two per thread, so the gather reads the permutation
    every tick) and about 28 000 input-line entries per core group (more than
    shared memory holds, so the entries are read from global memory)."""
    net = W.random_net(91, 8, 4, axons=128, neurons=64, n_types=4, n_inputs=2000, fanout_per_line=28,
                       delay_max=5, p_core=0.5, p_out=0.3, n_outputs=6)
    x = W.rate_coded_inputs(91, 6, 10, net.n_inputs, 0.1)
    ref = oracle_mod.run(net, x, 14, n_threads=NPROC)
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    l0 = ranc.ranc_launch_count(sim.h)
    np.testing.assert_array_equal(sim.run_samples(x, 14), ref["out"])
    assert ranc.ranc_launch_count(sim.h) - l0 <= 3  # the persistent kernel, not per-tick launches
    assert ref["out"].sum() > 0
    sim.close()


def test_run_samples_ragged_groups(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(3, 11, 8, 784, 0.15)
    ref = oracle_mod.run(net, x, 9)
    sim = ranc.Sim(net, 4, ranc.RANC_PATH_PLAIN)
    np.testing.assert_array_equal(sim.run_samples(x, 9), ref["out"])
    np.testing.assert_array_equal(sim.counters()[:4], ref["counters"][:, :4].sum(0))
    sim.close()


def test_edge_cases_zero_ticks_no_inputs_short_inputs(ranc, oracle_mod):
    net = W.random_net(77, 2, 2, axons=32, neurons=64, n_inputs=20, leak=(-1, 2), pthr=(3, 9), v0=(-2, 2))
    sim = ranc.Sim(net, 3, ranc.RANC_PATH_PLAIN)
    sim.step(0)
    assert sim.tick() == 0
    v, s, _ = sim.state()
    np.testing.assert_array_equal(v, np.broadcast_to(net.v0, v.shape))
    # no inputs loaded: leak and v0 alone drive the net
    sim.step(7)
    ref = oracle_mod.run(net, np.zeros((3, 0, net.in_words), np.uint32), 7)
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    # inputs shorter than the window
    sim.reset()
    x = W.rate_coded_inputs(8, 3, 2, net.n_inputs, 0.5)
    sim.load_inputs(x)
    sim.step(11)
    ref = oracle_mod.run(net, x, 11)
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    sim.close()


def test_net_without_inputs_and_largest_core(ranc, oracle_mod):
    net = W.random_net(78, 1, 1, axons=1024, neurons=1024, n_inputs=0, fanout_per_line=0, leak=(-2, 3),
                       pthr=(2, 40), v0=(-4, 30), w_lim=7, p_core=0.5, delay_max=3)
    ref = oracle_mod.run(net, np.zeros((2, 0, 0), np.uint32), 6, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    v, s, _ = gpu_trace(sim, 6)
    np.testing.assert_array_equal(v, ref["v_trace"])
    np.testing.assert_array_equal(s, ref["spike_trace"])
    assert ref["counters"][:, 1].sum() > 0
    sim.close()


def test_checkpoint_round_trip(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(11, 4, 8, 784, 0.2)
    ref = oracle_mod.run(net, x, 12)
    a = ranc.Sim(net, 4, ranc.RANC_PATH_PLAIN)
    a.load_inputs(x)
    a.step(5)
    buf = a.save()
    a.step(7)
    b = ranc.Sim(net, 4, ranc.RANC_PATH_PLAIN)
    b.load_inputs(x)
    b.load(buf)
    assert b.tick() == 5
    b.step(7)
    for s in (a, b):
        np.testing.assert_array_equal(s.state()[0], ref["v"])
        np.testing.assert_array_equal(s.outputs(), ref["out"])
        np.testing.assert_array_equal(s.counters()[:4], ref["counters"][:, :4].sum(0))
    a.close()
    b.close()


def test_reset_and_rerun_are_deterministic(ranc):
    net = W.mnist_512core()
    x = W.rate_coded_inputs(net.meta["seed"], 2, 16, 784, 0.15)
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    digs = []
    for _ in range(2):
        sim.load_inputs(x)
        sim.step(24)
        digs.append((sim.state()[2], sim.outputs().tobytes(), sim.counters().tobytes()))
        sim.reset()
    assert digs[0] == digs[1]
    sim.close()


def test_kernel_timing_and_launch_count(ranc):
    net = W.tiny_5core()
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    n0 = ranc.ranc_launch_count(sim.h)
    ranc.ranc_set_kernel_timing(sim.h, True)
    sim.step(10)  # one persistent launch for the 10 ticks
    ms, n = ranc.ranc_read_kernel_timing(sim.h)
    assert n == 10 and ms > 0
    assert ranc.ranc_launch_count(sim.h) - n0 == 1
    for _ in range(3):
        sim.step(1)  # one per-tick launch each
    ms, n = ranc.ranc_read_kernel_timing(sim.h)
    assert n == 13 and ranc.ranc_launch_count(sim.h) - n0 == 4
    # one persistent launch for 5 samples in windows of 9 ticks (3 windows of batch 2)
    ranc.ranc_set_kernel_timing(sim.h, True)
    sim.run_samples(W.rate_coded_inputs(1, 5, 8, 784, 0.15), 9)
    ms, n = ranc.ranc_read_kernel_timing(sim.h)
    assert n == 27 and ms > 0
    sim.close()


def _persistent_steps_case(ranc, oracle_mod, net, B, T, seed):
    """ranc_step(k) in one persistent launch (checked by the launch count)
    against the oracle's trace and against per-tick launches, with state
    reads between the calls."""
    x = W.rate_coded_inputs(seed, B, 10, net.n_inputs, 0.3)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    a = ranc.Sim(net, B, ranc.RANC_PATH_PLAIN)
    b = ranc.Sim(net, B, ranc.RANC_PATH_PLAIN)
    for s in (a, b):
        s.load_inputs(x)
    t = 0
    for k in (5, 2, 7):
        l0 = ranc.ranc_launch_count(a.h)
        a.step(k)
        assert ranc.ranc_launch_count(a.h) - l0 == 1, "one persistent launch"
        for _ in range(k):
            b.step(1)
        t += k
        va, sa, da = a.state()
        np.testing.assert_array_equal(va, ref["v_trace"][:, t - 1], err_msg=f"tick {t - 1}")
        np.testing.assert_array_equal(unpack_spikes(sa, net.neurons), ref["spike_trace"][:, t - 1])
        assert da == b.state()[2]
    np.testing.assert_array_equal(a.outputs(), ref["out"])
    np.testing.assert_array_equal(a.counters()[:4], ref["counters"][:, :4].sum(0))
    np.testing.assert_array_equal(a.counters(), b.counters())
    assert ref["counters"][:, 1].sum() > 0
    a.close()
    b.close()


def test_persistent_steps_with_more_units_than_ctas(ranc, oracle_mod):
    """ranc_step(n) on the plain path runs n ticks in one persistent launch
    whose CTAs serve several (sample, core) units each: a 64 x 32 grid of
    32 x 32 cores, 4 samples (8192 units, 54 per CTA; potentials and
    parameters resident in shared memory)."""
    net = W.random_net(77, 64, 32, axons=32, neurons=32, n_types=4, delay_max=6, n_inputs=300,
                       fanout_per_line=8, p_core=0.6, p_out=0.2, w_lim=7, weight_bits=4, pthr=(1, 12),
                       nthr=(-12, -1), leak=(-2, 1), v0=(-2, 2))
    _persistent_steps_case(ranc, oracle_mod, net, 4, 14, 5)


def test_persistent_steps_potentials_in_global_memory(ranc, oracle_mod):
    """The same with 1024-neuron cores (1600 cores, batch 1, 11 units per
    CTA): the units' potentials and parameters do not fit shared memory, so
    the launch reads and writes them in global memory every tick."""
    net = W.random_net(78, 40, 40, axons=32, neurons=1024, n_types=4, delay_max=6, n_inputs=300,
                       fanout_per_line=8, p_core=0.6, p_out=0.2, w_lim=7, weight_bits=4, pthr=(1, 12),
                       nthr=(-12, -1), leak=(-2, 1), v0=(-2, 2))
    _persistent_steps_case(ranc, oracle_mod, net, 1, 14, 6)
