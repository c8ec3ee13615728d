"""Streaming runs (one new input frame per tick, the shape of the paper's
MNIST and CIFAR-10 runs in Table I) against the CPU oracle, bit for bit: the
output-bus log of every tick, the potentials after the run and the counters,
on both paths, in the persistent and the per-tick launch forms, host and
device memory."""

import os

import numpy as np
import pytest

import ranc_workloads as W

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def stream_parity(ranc, oracle_mod, net, x, T, path, runs=1, launches=None):
    """x [B, n_in, words]: every batch slot is one stream.  launches:
    "persistent" (the whole stream in one tick-kernel launch, besides the
    reset) or "per_tick" (at least one launch per tick)."""
    B = x.shape[0]
    ref = oracle_mod.run(net, x, T, n_threads=NPROC, out_trace=True)
    sim = ranc.Sim(net, B, path)
    for r in range(runs):  # a run resets the state, so every run matches the oracle again
        l0 = ranc.ranc_launch_count(sim.h)
        log = sim.run_stream(x, T)
        n = ranc.ranc_launch_count(sim.h) - l0
        if launches == "persistent":
            assert n <= 3, n
        elif launches == "per_tick":
            assert n >= T, n
        np.testing.assert_array_equal(log, ref["out_trace"], err_msg=f"run {r}")
        np.testing.assert_array_equal(sim.outputs(), ref["out"])
        v, _, _ = sim.state()
        np.testing.assert_array_equal(v, ref["v"])
        assert sim.tick() == T
    cnt = sim.counters()  # counters accumulate over the runs
    np.testing.assert_array_equal(cnt[:4], runs * ref["counters"][:, :4].sum(0))
    assert cnt[4] == runs * B * T
    sim.close()
    return ref


def random_stream_net(seed):
    return W.random_net(seed, 3, 2, axons=64, neurons=128, n_types=3, n_inputs=50, fanout_per_line=4,
                        delay_max=5, p_core=0.5, p_out=0.3, n_outputs=7, v0=(-2, 2))


def test_plain_persistent_single_stream(ranc, oracle_mod):
    net = random_stream_net(41)
    x = W.rate_coded_inputs(41, 1, 40, net.n_inputs, 0.3)
    ref = stream_parity(ranc, oracle_mod, net, x, 48, ranc.RANC_PATH_PLAIN, runs=2, launches="persistent")
    assert ref["out_trace"].sum() > 0


def test_plain_persistent_three_streams(ranc, oracle_mod):
    net = random_stream_net(42)
    x = W.rate_coded_inputs(42, 3, 30, net.n_inputs, 0.3)
    stream_parity(ranc, oracle_mod, net, x, 37, ranc.RANC_PATH_PLAIN, launches="persistent")


def test_plain_per_tick_launches_when_the_grid_does_not_fit(ranc, oracle_mod):
    """200 streams of the 5-core net need more CTAs than can be resident, so
    the per-tick launches run (with the log slot of each tick)."""
    net = W.tiny_5core()
    x = W.rate_coded_inputs(43, 200, 20, 784, 0.15)
    ref = stream_parity(ranc, oracle_mod, net, x, 24, ranc.RANC_PATH_PLAIN, launches="per_tick")
    assert ref["out_trace"].sum() > 0


def test_batched_ragged_streams(ranc, oracle_mod):
    net = random_stream_net(44)
    x = W.rate_coded_inputs(44, 130, 25, net.n_inputs, 0.3)
    stream_parity(ranc, oracle_mod, net, x, 30, ranc.RANC_PATH_BATCHED, runs=2)


def test_stream_longer_than_the_scheduler_and_inputs(ranc, oracle_mod):
    """More ticks than input frames and than scheduler rows: frames stop, the
    pipeline drains, the rows wrap many times."""
    net = random_stream_net(45)
    x = W.rate_coded_inputs(45, 2, 9, net.n_inputs, 0.4)
    stream_parity(ranc, oracle_mod, net, x, 70, ranc.RANC_PATH_PLAIN)
    stream_parity(ranc, oracle_mod, net, x, 70, ranc.RANC_PATH_BATCHED)


def test_mnist512_stream_device_memory(ranc, oracle_mod):
    """The 512-core workload streamed one frame per tick (64 frames, 72
    ticks), inputs and log in device memory, plain persistent path."""
    torch = pytest.importorskip("torch")
    net = W.mnist_512core()
    x = W.rate_coded_inputs(net.meta["seed"], 1, 64, 784, 0.15)
    T = 72
    ref = oracle_mod.run(net, x, T, n_threads=NPROC, out_trace=True)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dlog = torch.zeros((1, T, net.n_outputs), dtype=torch.int32, device="cuda")
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    l0 = ranc.ranc_launch_count(sim.h)
    ranc.ranc_run_stream(sim.h, dx.data_ptr(), 64, T, dlog.data_ptr(), ranc.RANC_MEM_DEVICE)
    torch.cuda.synchronize()
    assert ranc.ranc_launch_count(sim.h) - l0 <= 3  # the 72 ticks in one persistent launch
    np.testing.assert_array_equal(dlog.cpu().numpy().view(np.uint32), ref["out_trace"])
    assert ref["out_trace"].sum() > 0
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    sim.close()


def test_run_stream_rejects_bad_arguments(ranc):
    net = W.tiny_5core()
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    out = np.zeros((1, 4, net.n_outputs), np.uint32)
    with pytest.raises(ranc.RancError):
        ranc.ranc_run_stream(sim.h, None, 3, 4, out)  # frames promised, no array
    with pytest.raises(ranc.RancError):
        ranc.ranc_run_stream(sim.h, None, 0, -1, out)
    sim.reset()
    ranc.ranc_run_stream(sim.h, None, 0, 4, out)  # no frames: a valid run without input
    sim.close()
