"""Work classes of the batched tick kernel against the CPU oracle, bit for bit.

A (core, tile) item whose scheduler row is empty and whose core no input line
drives in the tick has no synaptic input: it is updated without an MMA
("idle"), or, when every neuron of the core has leak <= 0, theta- < theta+,
reset < theta+ and v0 < theta+ with a saturating negative threshold, its idle
ticks are only counted and applied later as V <- max(V + k * leak, theta-)
("lazy").  These tests drive networks through input gaps so that cores fall
idle and wake up again, read the state in the middle of deferred periods
(which applies the deferred ticks first), mix eligible and ineligible cores,
and cross checkpoints, resets and window graphs."""

import os

import numpy as np
import pytest

import ranc_workloads as W
from parity_util import digest, idle_core_ticks, unpack_spikes

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def lazy_net(seed, w_lim=60, pthr=(1, 150), nthr=(-150, -1), hot_cores=()):
    """Feed-forward net (2 + 2 + 2 cores) whose cores all qualify for deferred
    idle ticks, except the cores in ``hot_cores``, which get a leak of +1 on
    every 17th neuron."""
    net = W.layered_net(seed, layers=(2, 2, 2), w_lim=w_lim, pthr=pthr, nthr=nthr)
    for c in hot_cores:
        net.leak[c, ::17] = 1
    return net


def with_gap(x, g0, g1):
    x = x.copy()
    x[:, g0:g1] = 0
    return x


def check_state(sim, ref, t, msg=""):
    v, s, d = sim.state()
    np.testing.assert_array_equal(v, ref["v_trace"][:, t], err_msg=f"V after tick {t} {msg}")
    np.testing.assert_array_equal(unpack_spikes(s, sim.net.neurons), ref["spike_trace"][:, t],
                                  err_msg=f"spikes after tick {t} {msg}")
    assert d == digest(ref["v_trace"][:, t]), t


FORMATS = [  # w_lim, pthr, nthr -> fp16, int16, int32 potentials
    (60, (1, 150), (-150, -1)),
    (900, (1000, 3000), (-3000, -1)),
    (2047, (20000, 40000), (-40000, -1)),
]


@pytest.mark.parametrize("fmt", range(3), ids=["fp16", "int16", "int32"])
def test_idle_and_deferred_ticks_read_in_chunks(ranc, oracle_mod, fmt):
    w_lim, pthr, nthr = FORMATS[fmt]
    net = lazy_net(41 + fmt, w_lim=w_lim, pthr=pthr, nthr=nthr, hot_cores=(4,))
    B, T = 300, 30
    x = with_gap(W.rate_coded_inputs(17 + fmt, B, 16, net.n_inputs, 0.35), 4, 11)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    idle = idle_core_ticks(net, x, ref, T)
    # the workload really has idle cores that wake up again
    assert idle.any() and (idle[:-1] & ~idle[1:]).any()
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    assert sim.potential_format() == [ranc.RANC_POTENTIAL_FP16, ranc.RANC_POTENTIAL_INT16,
                                      ranc.RANC_POTENTIAL_INT32][fmt]
    sim.load_inputs(x)
    t = 0
    for k in (1, 2, 5, 3, 1, 6, 4, 8):
        sim.step(k)
        t += k
        check_state(sim, ref, t - 1, f"(chunks, format {fmt})")
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    np.testing.assert_array_equal(sim.counters()[:4], ref["counters"][:, :4].sum(0))
    # every (core, 128-sample tile) item is either updated or deferred in every tick,
    # and this workload defers some
    upd, dfr = ranc.ranc_item_ticks(sim.h)
    assert upd + dfr == -(-B // 128) * net.n_cores * T and dfr > 0
    sim.close()


def test_deferred_ticks_with_a_leak_near_the_int32_limit(ranc, oracle_mod):
    """int32 potentials, every other neuron of the first two layers leaking
    -1e9 per tick down to theta- = -1e9: k deferred idle ticks apply k * leak,
    which leaves 32 bits after three ticks; the result must still be
    max(V + k * leak, theta-) as in the oracle's tick-by-tick int64
    arithmetic, both when a state read applies the deferred ticks (layer 1 in
    the input gap, layer 0 after the inputs) and when a core wakes up (layer 1
    when the inputs resume)."""
    w_lim, pthr, nthr = FORMATS[2]
    net = lazy_net(47, w_lim=w_lim, pthr=pthr, nthr=nthr)
    big = -10**9
    for c in range(4):
        net.leak[c, ::2] = big
        net.neg_thr[c, ::2] = big
    B, T = 140, 30
    x = with_gap(W.rate_coded_inputs(19, B, 24, net.n_inputs, 0.35), 3, 20)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    assert (ref["v_trace"][:, :, :2, ::2] == big).any()  # the saturated neurons are there
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    assert sim.potential_format() == ranc.RANC_POTENTIAL_INT32
    sim.load_inputs(x)
    t = 0
    for k in (2, 12, 8, 8):  # reads inside the input gap, after the wake-up, after the inputs
        sim.step(k)
        t += k
        check_state(sim, ref, t - 1, "(leak -1e9)")
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    upd, dfr = ranc.ranc_item_ticks(sim.h)
    assert dfr > 0
    sim.close()


def test_item_ticks_without_deferral_and_on_the_plain_path(ranc, oracle_mod):
    net = lazy_net(96, hot_cores=range(6))  # every core has a positive leak somewhere: nothing defers
    x = with_gap(W.rate_coded_inputs(41, 130, 10, net.n_inputs, 0.3), 2, 8)
    ref = oracle_mod.run(net, x, 16, n_threads=NPROC)
    sim = ranc.Sim(net, 130, ranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    sim.step(16)
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    assert ranc.ranc_item_ticks(sim.h) == (2 * net.n_cores * 16, 0)
    sim.close()
    plain = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    with pytest.raises(ranc.RancError):
        ranc.ranc_item_ticks(plain.h)
    plain.close()


def test_state_read_every_tick_through_idle_periods(ranc, oracle_mod):
    net = lazy_net(52, hot_cores=(1, 5))
    B, T = 140, 22
    x = with_gap(W.rate_coded_inputs(23, B, 14, net.n_inputs, 0.3), 3, 9)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    for t in range(T):
        sim.step(1)
        check_state(sim, ref, t, "(every tick)")
    sim.close()


def test_sample_state_reads_in_a_deferred_period(ranc, oracle_mod):
    net = lazy_net(63)
    B, T = 260, 20
    x = with_gap(W.rate_coded_inputs(29, B, 12, net.n_inputs, 0.3), 2, 12)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    sim = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    sim.step(9)
    for b in (0, 129, 259):
        v, s = sim.sample_state(b, 1)
        np.testing.assert_array_equal(v[0], ref["v_trace"][b, 8])
    sim.step(T - 9)
    check_state(sim, ref, T - 1, "(after sample reads)")
    sim.close()


def test_checkpoint_and_reset_inside_a_deferred_period(ranc, oracle_mod):
    net = lazy_net(74, hot_cores=(2,))
    B, T = 200, 24
    x = with_gap(W.rate_coded_inputs(31, B, 16, net.n_inputs, 0.3), 3, 12)
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    a = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    a.load_inputs(x)
    a.step(7)
    buf = a.save()
    b = ranc.Sim(net, B, ranc.RANC_PATH_BATCHED)
    b.load_inputs(x)
    b.load(buf)
    for s, name in ((a, "original"), (b, "restored")):
        s.step(5)
        check_state(s, ref, 11, name)
        s.step(T - 12)
        check_state(s, ref, T - 1, name)
        np.testing.assert_array_equal(s.outputs(), ref["out"])
    # a reset in the middle of a deferred period starts from v0 again
    a.reset()
    a.load_inputs(x)
    a.step(6)
    a.reset()
    a.load_inputs(x)
    a.step(T)
    check_state(a, ref, T - 1, "(after resets)")
    np.testing.assert_array_equal(a.outputs(), ref["out"])
    a.close()
    b.close()


def test_window_graph_replays_on_a_deferring_net(ranc, oracle_mod):
    import torch
    net = lazy_net(85, hot_cores=(3,))
    S, t_in, window = 300, 12, 22
    x = with_gap(W.rate_coded_inputs(37, S, t_in, net.n_inputs, 0.3), 3, 8)
    ref = oracle_mod.run(net, x, window, n_threads=NPROC)
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((S, net.n_outputs), dtype=torch.int32, device="cuda")
    ref_last = oracle_mod.run(net, x[256:], window + 3, trace=True, n_threads=NPROC)  # the last group: 44 samples
    for k in range(3):
        dout.zero_()
        ranc.ranc_run_samples(sim.h, dx.data_ptr(), S, t_in, window, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
        np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref["out"], err_msg=f"call {k}")
        # the state after the window is readable and exact, and stepping on
        # from it keeps the deliveries still in flight
        v, _, _ = sim.state(want_spikes=False, want_digest=False)
        np.testing.assert_array_equal(v[:S - 256], ref_last["v_trace"][:, window - 1], err_msg=f"call {k}")
        sim.step(3)
        v, _, _ = sim.state(want_spikes=False, want_digest=False)
        np.testing.assert_array_equal(v[:S - 256], ref_last["v_trace"][:, window + 2], err_msg=f"call {k}, +3")
    assert ranc.ranc_graph_stats(sim.h) == (1, 2)
    sim.close()
