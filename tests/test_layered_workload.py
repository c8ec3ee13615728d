"""The feed-forward workload behind the batched path's item-class tests
(`ranc_workloads.layered_net`), checked on the CPU: its structure, and, under
the oracle, that cores fall idle once the inputs stop and wake up when they
resume (the property that makes the GPU tests exercise idle and deferred
items)."""

import os

import numpy as np

import ranc_workloads as W

NPROC = os.cpu_count() or 1


def _dest_cores(net):
    pos = {(int(x), int(y)): k for k, (x, y) in enumerate(net.core_xy)}
    d = net.dest
    out = np.full(d.shape, -1)
    for c in range(net.n_cores):
        for n in range(net.neurons):
            if d["kind"][c, n] == W.KIND_CORE:
                out[c, n] = pos[(int(net.core_xy[c, 0] + d["dx"][c, n]), int(net.core_xy[c, 1] + d["dy"][c, n]))]
    return out


def test_layered_net_is_feed_forward():
    layers = (3, 2, 2)
    net = W.layered_net(11, layers=layers, axons=64, neurons=64)
    start = np.concatenate([[0], np.cumsum(layers)])
    layer_of = np.repeat(np.arange(len(layers)), layers)
    dc = _dest_cores(net)
    kinds = net.dest["kind"]
    for c in range(net.n_cores):
        k = layer_of[c]
        targets = dc[c][kinds[c] == W.KIND_CORE]
        if k + 1 < len(layers):
            assert len(targets) > 0 and np.all(layer_of[targets] == k + 1)
            assert not np.any(kinds[c] == W.KIND_OUTPUT)
        else:
            assert len(targets) == 0 and np.any(kinds[c] == W.KIND_OUTPUT)
    assert np.all(np.asarray(net.in_core) < start[1])  # inputs drive layer 0 only
    d = net.dest["delay"][kinds == W.KIND_CORE]
    assert d.min() >= 1 and d.max() <= 6
    # the deferral conditions hold for every neuron (leak <= 0, reset, theta- and v0 below theta+)
    assert np.all(net.leak <= 0) and np.all(net.reset < net.pos_thr) and np.all(net.neg_thr < net.pos_thr)
    assert np.all(net.v0 < net.pos_thr) and net.neg_mode == W.NEG_SATURATE


def test_layered_net_cores_fall_idle_and_wake_up(oracle_mod):
    net = W.layered_net(41, layers=(2, 2, 2), w_lim=60, pthr=(1, 150), nthr=(-150, -1))
    T = 30
    x = W.rate_coded_inputs(17, 64, 16, net.n_inputs, 0.35)
    x[:, 4:11] = 0  # an input gap
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    # per (tick, core): some packet or input arrives in some sample
    dc = _dest_cores(net)
    fired = ref["spike_trace"].any(0)
    active = np.zeros((T, net.n_cores), bool)
    for t in range(T):
        for c, n in zip(*np.nonzero(fired[t])):
            if dc[c, n] >= 0 and t + int(net.dest["delay"][c, n]) < T:
                active[t + int(net.dest["delay"][c, n]), dc[c, n]] = True
    driven = np.zeros(net.n_cores, bool)
    driven[np.asarray(net.in_core)] = True
    for t in range(T):
        if x[:, min(t, x.shape[1] - 1)].any() and t < x.shape[1]:
            active[t] |= driven
    idle = ~active
    assert idle.sum() > 0.2 * idle.size  # a good share of core-ticks is idle
    wakeups = idle[:-1] & ~idle[1:]
    assert wakeups.sum() >= 2  # and idle cores receive input again


def test_idle_ticks_of_eligible_cores_compose_in_closed_form(oracle_mod):
    """The identity behind the batched path's deferred ticks, checked on the
    oracle's trace: over a run of ticks in which a core receives no packet and
    no input, every neuron of a core with leak <= 0, reset, theta- and v0
    below theta+ and a saturating negative threshold does not fire, and its
    potential after k such ticks is max(V + k * leak, theta-)."""
    net = W.layered_net(57, layers=(2, 2, 2), w_lim=60, pthr=(1, 150), nthr=(-150, -1))
    T = 34
    x = W.rate_coded_inputs(23, 48, 20, net.n_inputs, 0.35)
    x[:, 3:14] = 0  # a long input gap
    ref = oracle_mod.run(net, x, T, trace=True, n_threads=NPROC)
    v, sp = ref["v_trace"], ref["spike_trace"]  # [S, T, C, N]
    dc = _dest_cores(net)
    # per (sample, tick, core): a packet or an input arrives
    S = x.shape[0]
    recv = np.zeros((S, T, net.n_cores), bool)
    for t in range(T):
        for s, c, n in zip(*np.nonzero(sp[:, t])):
            if dc[c, n] >= 0 and t + int(net.dest["delay"][c, n]) < T:
                recv[s, t + int(net.dest["delay"][c, n]), dc[c, n]] = True
    bits = np.unpackbits(x.view(np.uint8), axis=-1, bitorder="little")[..., :net.n_inputs]  # [S, T_in, L]
    offs = np.asarray(net.in_offsets)
    for line in range(net.n_inputs):
        for e in range(offs[line], offs[line + 1]):
            recv[:, :x.shape[1], net.in_core[e]] |= bits[:, :, line].astype(bool)
    lam = net.leak.astype(np.int64)
    checked = 0
    for s in range(S):
        for c in range(net.n_cores):
            t = 1
            while t < T:
                if recv[s, t, c]:
                    t += 1
                    continue
                t1 = t  # ticks t1 .. t2 - 1 receive nothing
                while t < T and not recv[s, t, c]:
                    t += 1
                k = t - t1
                assert not sp[s, t1:t, c].any()
                expect = np.maximum(v[s, t1 - 1, c].astype(np.int64) + k * lam[c], net.neg_thr[c])
                np.testing.assert_array_equal(v[s, t - 1, c], expect, err_msg=f"sample {s} core {c} ticks {t1}..{t - 1}")
                checked += k
    assert checked > 500  # idle ticks covered
