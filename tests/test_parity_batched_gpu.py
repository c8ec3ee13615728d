"""Batched tensor-core path against the CPU oracle, bit for bit: potentials,
spikes and output counts per tick on small networks and ragged batches, and
sampled samples of the 4096-sample, 512-core configuration that the benchmark
times (same handle shape and launch configuration)."""

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


def expected_format(ranc, net):
    """The storage the header promises: the reachable range [lo, hi] of every
    neuron decides between fp16, int16 and int32."""
    pt, nt = net.pos_thr.astype(np.int64), net.neg_thr.astype(np.int64)
    r, v0, lk = net.reset.astype(np.int64), net.v0.astype(np.int64), net.leak.astype(np.int64)
    hi = np.maximum.reduce([pt - 1, nt, r, v0])
    lo = np.minimum.reduce([nt, r, v0])
    half = (lo >= -2048) & (hi <= 2048) & (lo + lk >= -2048) & (hi + lk <= 2048) & (np.abs(lk) <= 2048) & \
        (pt >= -2047) & (pt <= 2048) & (nt >= -2047) & (nt <= 2048)
    if half.all():
        return ranc.RANC_POTENTIAL_FP16
    if (hi <= 32767).all() and (lo >= -32768).all():
        return ranc.RANC_POTENTIAL_INT16
    return ranc.RANC_POTENTIAL_INT32


def per_tick_parity(ranc, oracle_mod, net, x, T, fmt=None):
    B = x.shape[0]
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    if fmt is not None:
        assert sim.potential_format() == fmt
    sim.load_inputs(x)
    v, s, d = gpu_trace(sim, T)
    for t in range(T):
        np.testing.assert_array_equal(v[:, t], ref["v_trace"][:, t], err_msg=f"tick {t}")
        np.testing.assert_array_equal(s[:, t], ref["spike_trace"][:, t], err_msg=f"tick {t}")
        assert d[t] == digest(ref["v_trace"][:, t]), t
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    cnt = sim.counters()
    np.testing.assert_array_equal(cnt[:4], ref["counters"][:, :4].sum(0))
    assert cnt[4] == B * T
    sim.close()
    return ref


def test_tiny_workload_one_padded_tile(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(net.meta["seed"], 64, 8, 784, 0.15)
    per_tick_parity(ranc, oracle_mod, net, x, 9, fmt=ranc.RANC_POTENTIAL_FP16)


SHAPES = [
    # grid, axons, neurons, types, neg_mode, delay_max, batch, v0, weight limit / bits
    ((2, 2), 64, 128, 2, 0, 15, 128, (0, 0), (7, 4)),
    ((3, 1), 128, 256, 4, 1, 5, 130, (-3, 3), (255, 9)),
    ((2, 2), 192, 128, 8, 0, 9, 257, (-5, 5), (2047, 12)),
    ((1, 3), 256, 256, 3, 1, 15, 40, (0, 4), (100, 8)),
]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[1]}x{s[2]}b{s[6]}" for s in SHAPES])
def test_random_nets_every_tick(ranc, oracle_mod, shape):
    (gw, gh), A, N, K, neg, dmax, B, v0, (wl, wb) = shape
    net = W.random_net(200 + A + N, gw, gh, axons=A, neurons=N, n_types=K, neg_mode=neg, delay_max=dmax,
                       v0=v0, n_inputs=90, fanout_per_line=4, p_core=0.6, p_out=0.2, w_lim=wl,
                       weight_bits=wb, pthr=(1, 3 * wl), nthr=(-3 * wl, -1), leak=(-2, 2))
    x = W.rate_coded_inputs(9, B, 10, net.n_inputs, 0.3)
    ref = per_tick_parity(ranc, oracle_mod, net, x, 18, fmt=expected_format(ranc, net))
    assert ref["counters"][:, 1].sum() > 0


def test_int32_potentials_when_int16_cannot_hold_them(ranc, oracle_mod):
    net = W.random_net(301, 2, 1, axons=64, neurons=128, w_lim=2047, weight_bits=12, pthr=(30000, 60000),
                       nthr=(-60000, -30000), leak=(-5, 5), n_inputs=40, fanout_per_line=6)
    x = W.rate_coded_inputs(10, 150, 8, net.n_inputs, 0.5)
    per_tick_parity(ranc, oracle_mod, net, x, 12, fmt=ranc.RANC_POTENTIAL_INT32)


def fp16_edge_net(seed, neg_mode, pthr_hi=2048):
    """Thresholds and values at the edges of the fp16 format's conditions:
    theta+ up to 2048, theta- down to -2047, leak in [-1, 1] so that V + leak
    reaches +-2048, weights of 12 bits so that V + dV overflows fp16 (to
    +-inf) when many axons are active; a few neurons carry reset / v0 at
    +-2048 with zero leak."""
    net = W.random_net(seed, 2, 2, axons=128, neurons=128, n_types=4, density=0.6, w_lim=2047, weight_bits=12,
                       pthr=(1900, pthr_hi), nthr=(-2047, -1900), leak=(-1, 1), reset=(-2047, 2047),
                       neg_mode=neg_mode, v0=(-1500, 1500), n_inputs=64, fanout_per_line=16, p_core=0.6,
                       p_out=0.2, delay_max=3)
    net.leak[:, :8] = 0
    net.reset[:, 0], net.reset[:, 1] = 2048, -2048
    net.v0[:, 2], net.v0[:, 3] = 2048, -2048
    net.pos_thr[:, 4], net.neg_thr[:, 4] = 2048, -2047
    net.pos_thr[:, 5], net.neg_thr[:, 5] = -2047, -2047   # theta+ <= theta-: fires at any x >= -2047
    return net


@pytest.mark.parametrize("neg_mode", [0, 1])
def test_fp16_potentials_at_the_edges_of_their_range(ranc, oracle_mod, neg_mode):
    net = fp16_edge_net(311 + neg_mode, neg_mode)
    x = W.rate_coded_inputs(12, 140, 10, net.n_inputs, 0.5)
    ref = per_tick_parity(ranc, oracle_mod, net, x, 14, fmt=ranc.RANC_POTENTIAL_FP16)
    v = ref["v_trace"]
    assert v.max() >= 2000 and v.min() <= -2000          # the extremes are reached
    assert ref["counters"][:, 0].sum() > 0


def test_int16_potentials_one_past_the_fp16_range(ranc, oracle_mod):
    net = fp16_edge_net(313, 0, pthr_hi=2049)
    assert net.pos_thr.max() == 2049
    x = W.rate_coded_inputs(13, 130, 10, net.n_inputs, 0.5)
    per_tick_parity(ranc, oracle_mod, net, x, 12, fmt=ranc.RANC_POTENTIAL_INT16)


SAMPLED = [0, 1, 127, 128, 1000, 2047, 2048, 3001, 4094, 4095]


def test_mnist512_full_batch_sampled(ranc, oracle_mod):
    """The benchmark's handle: 512 cores, 4096 samples in 32 tiles, 24 ticks.
    Sampled samples are compared with the oracle in full (every potential and
    spike of the last tick, output counts); the digest of every potential of
    the sampled samples is compared after every tick."""
    net = W.mnist_512core()
    B = 4096
    x = W.rate_coded_inputs(net.meta["seed"], B, 16, 784, 0.15)
    xs = x[SAMPLED]
    ref = oracle_mod.run(net, xs, 24, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    for t in range(24):
        sim.step(1)
        for k, b in enumerate(SAMPLED):
            v, s = sim.sample_state(b, 1)
            np.testing.assert_array_equal(v[0], ref["v_trace"][k, t], err_msg=f"sample {b} tick {t}")
            np.testing.assert_array_equal(unpack_spikes(s[0], 256), ref["spike_trace"][k, t])
    out = sim.outputs()
    np.testing.assert_array_equal(out[SAMPLED], ref["out"])
    cnt = sim.counters()
    assert cnt[4] == B * 24
    # every sample: output events and spikes are consistent with the counters
    assert int(out.sum()) == int(cnt[2])
    sim.close()


def test_mnist512_window_graph_as_benchmarked(ranc, oracle_mod):
    """The benchmark's exact launch sequence: a 4096-sample handle, the inputs
    and counts in device memory, ranc_run_samples recorded as a window graph
    and replayed (deferred idle ticks included, no state read in between),
    with and without the timing events the benchmark records.  64 samples
    spread over all 32 tiles (two per tile, at varying positions) are compared
    with the oracle: every output count, and every potential (and its digest)
    after the window."""
    import torch
    net = W.mnist_512core()
    B, t_in, window = 4096, 16, 24
    x = W.rate_coded_inputs(net.meta["seed"], B, t_in, 784, 0.15)
    picked = np.array([64 * k + (37 * k + 5) % 64 for k in range(64)])
    assert len(set(picked // 128)) == 32
    ref = oracle_mod.run(net, x[picked], window, n_threads=NPROC)
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((B, net.n_outputs), dtype=torch.int32, device="cuda")
    run = lambda: ranc.ranc_run_samples(sim.h, dx.data_ptr(), B, t_in, window, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
    for timed in (False, True):
        ranc.ranc_set_kernel_timing(sim.h, timed)
        for k in range(3):  # a recording, then replays
            dout.zero_()
            run()
            out = dout.cpu().numpy().view(np.uint32)
            np.testing.assert_array_equal(out[picked], ref["out"], err_msg=f"timed {timed}, call {k}")
            v = np.stack([sim.sample_state(int(b), 1)[0][0] for b in picked])
            np.testing.assert_array_equal(v, ref["v"], err_msg=f"timed {timed}, call {k}")
            assert digest(v) == digest(ref["v"])
        if timed:  # the replays timed their own tick kernels: 24 per call
            ms, n = ranc.ranc_read_kernel_timing(sim.h)
            assert n == 3 * window and ms > 0
    assert ranc.ranc_graph_stats(sim.h) == (2, 4)  # one recording per timing setting
    upd, dfr = ranc.ranc_item_ticks(sim.h)
    act, idle, dfr2 = ranc.ranc_item_classes(sim.h)
    assert act + idle == upd and dfr2 == dfr and dfr > 0  # the window defers idle ticks
    sim.close()


def test_batched_equals_plain_on_every_sample_of_a_large_batch(ranc, oracle_mod):
    """All 1000 samples (8 tiles, ragged) through both paths; the plain path
    is pinned to the oracle separately, and both are compared with the oracle
    on a sampled subset here."""
    net = W.mnist_512core()
    B = 1000
    x = W.rate_coded_inputs(net.meta["seed"], B, 16, 784, 0.15, first_sample=5000)
    res = {}
    for path in (ranc.RANC_PATH_PLAIN, ranc.RANC_PATH_BATCHED):
        sim = ranc.Sim(net, B, path)
        sim.load_inputs(x)
        sim.step(24)
        res[path] = (sim.outputs(), sim.state()[2], sim.counters())
        sim.close()
    a, b = res[ranc.RANC_PATH_PLAIN], res[ranc.RANC_PATH_BATCHED]
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])
    sel = [0, 511, 999]
    ref = oracle_mod.run(net, x[sel], 24, n_threads=NPROC)
    np.testing.assert_array_equal(b[0][sel], ref["out"])


def test_run_samples_ragged_groups_batched(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(4, 300, 8, 784, 0.15)
    ref = oracle_mod.run(net, x, 9, n_threads=NPROC)
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    np.testing.assert_array_equal(sim.run_samples(x, 9), ref["out"])
    np.testing.assert_array_equal(sim.counters()[:4], ref["counters"][:, :4].sum(0))
    sim.close()


def test_checkpoint_round_trip_batched(ranc, oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(12, 130, 8, 784, 0.2)
    ref = oracle_mod.run(net, x, 12, n_threads=NPROC)
    a = ranc.Sim(net, 130, ranc.RANC_PATH_BATCHED)
    a.load_inputs(x)
    a.step(4)
    buf = a.save()
    b = ranc.Sim(net, 130, ranc.RANC_PATH_BATCHED)
    b.load_inputs(x)
    b.load(buf)
    for s in (a, b):
        s.step(8)
        np.testing.assert_array_equal(s.state()[0], ref["v"])
        np.testing.assert_array_equal(s.outputs(), ref["out"])
        np.testing.assert_array_equal(s.counters()[:4], ref["counters"][:, :4].sum(0))
    # a plain-path checkpoint has the same canonical content but another path tag
    a.close()
    b.close()


def test_batched_rejects_unsupported_shapes(ranc):
    net = W.random_net(5, 2, 1, axons=32, neurons=32)
    with pytest.raises(ranc.RancError) as ei:
        ranc.ranc_create(net, 128, ranc.RANC_PATH_BATCHED)
    assert ei.value.code == ranc.RANC_EINVAL
