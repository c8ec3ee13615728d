"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test checks the oracle against something it does not compute itself:
hand-worked golden trajectories, closed forms, the delay/row timing of the
scheduler, OR merging, packet conservation, a per-tick matrix-product identity
and brute force against an independent hop-by-hop restatement.
"""

import itertools
import math
import os

import numpy as np
import pytest

import ranc_workloads as W
from ranc_workloads import rng

from hop_router import simulate as hop_simulate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BIG = 1 << 20


# ---------------------------------------------------------------------------
# helpers that build tiny nets (inputs only; no simulation arithmetic)
# ---------------------------------------------------------------------------

def single_neuron_net(w, leak, pos_thr, neg_thr, reset, neg_mode):
    C, A, N, K = 1, 32, 32, 4
    syn = np.zeros((C, A, N), np.uint8)
    syn[0, 0, 0] = 1
    weight = np.zeros((C, K, N), np.int16)
    weight[0, 0, 0] = w
    lk = np.zeros((C, N), np.int32)
    lk[0, 0] = leak
    pt = np.full((C, N), BIG, np.int32)
    pt[0, 0] = pos_thr
    nt = np.full((C, N), -BIG, np.int32)
    nt[0, 0] = neg_thr
    rs = np.zeros((C, N), np.int32)
    rs[0, 0] = reset
    dest = W.empty_dest(C, N)
    dest[0, 0] = (0, 0, 0, 1, W.KIND_OUTPUT)
    return W.make_net("single", 1, 1, [(0, 0)], syn, np.zeros((C, A)), weight, lk, pt, nt, rs, dest,
                      1, 1, [(0, 0, 0)], neg_mode=neg_mode, weight_bits=16)


def bits_inputs(pattern):
    """[1, T, 1] uint32 with line 0 set at the ticks where pattern is 1."""
    return np.array(pattern, dtype=np.uint32).reshape(1, -1, 1)


def chain_net(delay, n_sources=1, w_b=1, thr_b=1):
    """Core 0 neurons 0..n_sources-1 each fire on input line 0 and send to
    core 1 axon 0 with the given delay; core 1 neuron 0 integrates axon 0."""
    C, A, N, K = 2, 32, 32, 4
    syn = np.zeros((C, A, N), np.uint8)
    syn[0, 0, :n_sources] = 1
    syn[1, 0, 0] = 1
    weight = np.zeros((C, K, N), np.int16)
    weight[0, 0, :n_sources] = 1
    weight[1, 0, 0] = w_b
    pt = np.full((C, N), BIG, np.int32)
    pt[0, :n_sources] = 1
    pt[1, 0] = thr_b
    dest = W.empty_dest(C, N)
    for i in range(n_sources):
        dest[0, i] = (1, 0, 0, delay, W.KIND_CORE)
    dest[1, 0] = (-1, 0, 5, 1, W.KIND_CORE)  # back to core 0, axon 5 (unconnected)
    return W.make_net("chain", 2, 1, [(0, 0), (1, 0)], syn, np.zeros((C, A)), weight, 0, pt, -BIG, 0,
                      dest, 1, 1, [(0, 0, 0)], weight_bits=16)


def parse_golden_cases(path):
    cases, cur = [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "case":
            cur = {"name": vals[0]}
            cases.append(cur)
        elif key in ("input", "v", "spike"):
            cur[key] = [int(x) for x in vals]
        else:
            cur[key] = int(vals[0])
    return cases


GOLDEN_CASES = parse_golden_cases(os.path.join(GOLDEN, "single_neuron.txt"))


# ---------------------------------------------------------------------------
# generator (the shared input module) against the published SplitMix64 outputs
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    g = np.uint64(0x9E3779B97F4A7C15)
    assert int(rng.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    assert int(rng.splitmix64(g)) == 0x6E789E6AA1B965F4
    with np.errstate(over="ignore"):
        assert int(rng.splitmix64(g * np.uint64(2))) == 0x06C45D188009454F


def test_generator_shapes_and_ranges():
    net = W.tiny_5core()
    assert net.crossbar.shape == (5, 256, 8) and net.weight.shape == (5, 4, 256)
    assert net.weight.min() >= -64 and net.weight.max() <= 64
    m = W.mnist_512core()
    assert m.n_cores == 512 and m.in_offsets[-1] == 384 * 256
    assert set(np.unique(m.dest["delay"][m.dest["kind"] == W.KIND_CORE])) <= {1, 2, 3, 4}
    x = W.rate_coded_inputs(7, 6, 4, 784, 0.15)
    y = W.rate_coded_inputs(7, 3, 4, 784, 0.15, first_sample=3)
    assert (x[3:] == y).all()
    dens = np.unpackbits(x.view(np.uint8), bitorder="little").mean()
    assert 0.12 < dens * (800 / 784) < 0.18


# ---------------------------------------------------------------------------
# single-neuron pins
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLDEN_CASES, ids=[c["name"] for c in GOLDEN_CASES])
def test_golden_single_neuron(oracle_mod, case):
    net = single_neuron_net(case["w"], case["leak"], case["pos_thr"], case["neg_thr"], case["reset"],
                            case["neg_mode"])
    T = len(case["input"])
    r = oracle_mod.run(net, bits_inputs(case["input"]), T, trace=True)
    assert r["v_trace"][0, :, 0, 0].tolist() == case["v"]
    assert r["spike_trace"][0, :, 0, 0].tolist() == case["spike"]
    assert int(r["out"][0, 0]) == sum(case["spike"])


CLOSED = [(w, lk, th) for w in (1, 3, 7, 16) for lk in (-2, 0, 1) for th in (1, 5, 8, 12, 16)]


@pytest.mark.parametrize("w,leak,thr", CLOSED)
def test_closed_form_constant_drive(oracle_mod, w, leak, thr):
    """One axon active every tick: u = w + leak.  u > 0: period p = ceil(thr/u),
    V_t = (t mod p) u, floor(T/p) spikes in T ticks.  u <= 0: never fires and
    V_t = max(neg_thr, t u)."""
    T, nthr = 40, -9
    net = single_neuron_net(w, leak, thr, nthr, 0, W.NEG_SATURATE)
    r = oracle_mod.run(net, bits_inputs([1] * T), T, trace=True)
    v = r["v_trace"][0, :, 0, 0]
    u = w + leak
    if u > 0:
        p = -(-thr // u)
        assert v.tolist() == [(t % p) * u for t in range(1, T + 1)]
        assert int(r["out"][0, 0]) == T // p
    else:
        assert v.tolist() == [max(nthr, t * u) for t in range(1, T + 1)]
        assert int(r["out"][0, 0]) == 0


@pytest.mark.parametrize("u,nthr", [(-1, -1), (-1, -4), (-3, -10), (-5, -10), (-4, -4), (-7, -20)])
def test_closed_form_negative_reset_mode(oracle_mod, u, nthr):
    """Reset mode with u < 0 and reset 0: V_t = (t mod q) u with
    q = floor(|neg_thr| / |u|) + 1 (strict comparison)."""
    T = 30
    net = single_neuron_net(u, 0, 100, nthr, 0, W.NEG_RESET)
    r = oracle_mod.run(net, bits_inputs([1] * T), T, trace=True)
    q = abs(nthr) // abs(u) + 1
    assert r["v_trace"][0, :, 0, 0].tolist() == [(t % q) * u for t in range(1, T + 1)]


# ---------------------------------------------------------------------------
# scheduler row timing, OR merge
# ---------------------------------------------------------------------------

def _delay_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "delay_chain.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    return rows


@pytest.mark.parametrize("t0,d,fire", _delay_rows())
def test_golden_delay_chain(oracle_mod, t0, d, fire):
    net = chain_net(d)
    T = 32
    pattern = [1 if t == t0 else 0 for t in range(T)]
    r = oracle_mod.run(net, bits_inputs(pattern), T, trace=True)
    st = r["spike_trace"][0]
    assert np.flatnonzero(st[:, 0, 0]).tolist() == [t0]
    assert np.flatnonzero(st[:, 1, 0]).tolist() == [fire]


@pytest.mark.parametrize("d", range(1, 16))
def test_every_delay(oracle_mod, d):
    net = chain_net(d)
    r = oracle_mod.run(net, bits_inputs([1] + [0] * 19), 20, trace=True)
    assert np.flatnonzero(r["spike_trace"][0, :, 1, 0]).tolist() == [d]
    assert int(r["counters"][0, 1]) == 2  # core 0 neuron 0 and core 1 neuron 0 both send a packet


def test_or_merge_of_duplicate_packets(oracle_mod):
    """Three packets to the same (core, axon, tick) are one axon spike: with
    weight 1 and pos_thr 2 the target must not fire, and V ends at 1."""
    net = chain_net(2, n_sources=3, w_b=1, thr_b=2)
    r = oracle_mod.run(net, bits_inputs([1, 0, 0, 0]), 4, trace=True)
    assert r["spike_trace"][0, :, 1, 0].sum() == 0
    assert r["v_trace"][0, 2, 1, 0] == 1
    assert int(r["counters"][0, 1]) == 3  # packets count packets, not bits


# ---------------------------------------------------------------------------
# invariants and the per-tick matrix identity on random and workload nets
# ---------------------------------------------------------------------------

def _dest_core_index(net):
    """[C, N] destination core id for kind-core neurons (-1 otherwise)."""
    pos = {(int(x), int(y)): c for c, (x, y) in enumerate(net.core_xy)}
    out = np.full((net.n_cores, net.neurons), -1, np.int64)
    for c in range(net.n_cores):
        for n in np.flatnonzero(net.dest["kind"][c] == W.KIND_CORE):
            d = net.dest[c, n]
            out[c, n] = pos[(int(net.core_xy[c, 0]) + int(d["dx"]), int(net.core_xy[c, 1]) + int(d["dy"]))]
    return out


def check_matrix_identity(net, inputs, res, n_ticks):
    """Rebuild each tick's active-axon matrix S_t from the inputs and the
    oracle's own earlier spikes, then require
    V_t = rule(V_{t-1} + sum_k w_k * ((S_t masked to type k) @ C) + leak)
    with numpy int64 matrix products, and spikes == (pre >= pos_thr)."""
    Cn, A, N, K = net.n_cores, net.axons, net.neurons, net.n_types
    syn = np.unpackbits(net.crossbar.view(np.uint8), axis=-1, bitorder="little").reshape(Cn, A, N).astype(np.int64)
    dst = _dest_core_index(net)
    S_all = res["spike_trace"].shape[0]
    for s in range(S_all):
        pending = np.zeros((n_ticks + 16, Cn, A), np.int64)
        v_prev = net.v0.astype(np.int64)
        syn_events = 0
        for t in range(n_ticks):
            S = pending[t].copy()
            if t < inputs.shape[1]:
                lines = np.unpackbits(inputs[s, t].view(np.uint8), bitorder="little")[:net.n_inputs]
                for i in np.flatnonzero(lines):
                    for k in range(net.in_offsets[i], net.in_offsets[i + 1]):
                        S[net.in_core[k], net.in_axon[k]] = 1
            dv = np.zeros((Cn, N), np.int64)
            for c in range(Cn):
                for k in range(K):
                    Sk = S[c] * (net.axon_type[c] == k)
                    dv[c] += net.weight[c, k].astype(np.int64) * (Sk @ syn[c])
                syn_events += int((S[c] @ syn[c]).sum())
            pre = v_prev + dv + net.leak
            fire = pre >= net.pos_thr
            low = np.where(net.neg_mode == 0, net.neg_thr, net.reset)
            v = np.where(fire, net.reset, np.where(pre < net.neg_thr, low, pre))
            assert (res["spike_trace"][s, t] == fire).all(), (s, t)
            assert (res["v_trace"][s, t] == v).all(), (s, t)
            for c, n in zip(*np.nonzero(fire & (dst >= 0))):
                d = net.dest[c, n]
                pending[t + int(d["delay"]), dst[c, n], int(d["axon"])] = 1
            v_prev = v
        assert int(res["counters"][s, 3]) == syn_events


def check_conservation(net, res):
    st = res["spike_trace"].astype(np.int64)
    kind = net.dest["kind"]
    per_sample = st.sum(axis=1)  # [S, C, N]
    assert (res["counters"][:, 0] == st.sum(axis=(1, 2, 3))).all()
    assert (res["counters"][:, 1] == (per_sample * (kind == W.KIND_CORE)).sum(axis=(1, 2))).all()
    assert (res["counters"][:, 2] == (per_sample * (kind == W.KIND_OUTPUT)).sum(axis=(1, 2))).all()
    for o in range(net.n_outputs):
        m = (kind == W.KIND_OUTPUT) & (net.dest["axon"] == o)
        assert (res["out"][:, o] == (per_sample * m).sum(axis=(1, 2))).all()


@pytest.mark.parametrize("seed,neg_mode", [(11, 0), (12, 1), (13, 0)])
def test_random_net_matrix_identity_and_conservation(oracle_mod, seed, neg_mode):
    net = W.random_net(seed, 3, 2, axons=32, neurons=64, n_types=3, neg_mode=neg_mode, n_inputs=40,
                       fanout_per_line=3, delay_max=6, v0=(-3, 3))
    x = W.rate_coded_inputs(seed, 4, 8, net.n_inputs, 0.3)
    T = 14
    r = oracle_mod.run(net, x, T, trace=True)
    assert r["counters"][:, 0].sum() > 0
    check_matrix_identity(net, x, r, T)
    check_conservation(net, r)


def test_tiny_workload_matrix_identity_and_conservation(oracle_mod):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(net.meta["seed"], 3, 8, 784, 0.15)
    r = oracle_mod.run(net, x, 9, trace=True)
    check_matrix_identity(net, x, r, 9)
    check_conservation(net, r)


def stream_chain_net(delay):
    """chain_net with core 1 neuron 0 on the output bus (id 0) instead of
    sending back to core 0."""
    net = chain_net(delay)
    net.dest[1, 0] = (0, 0, 0, 1, W.KIND_OUTPUT)
    return net


@pytest.mark.parametrize("d", [1, 3, 15])
def test_stream_output_log_timing(oracle_mod, d):
    """One frame per tick (the streamed runs of Table I): a frame with line 0
    on at tick t drives core 0 at t (input delay 0), core 1 at t + d, and the
    bus logs one event of id 0 at tick t + d; frames at neighbouring ticks
    stay separate in the log.  Derived by hand from the tick rules."""
    frames = [2, 5, 6, 11]
    T = 11 + d + 3
    r = oracle_mod.run(stream_chain_net(d), bits_inputs([1 if t in frames else 0 for t in range(12)]), T,
                       out_trace=True)
    log = r["out_trace"][0, :, 0]
    assert np.flatnonzero(log).tolist() == [t + d for t in frames]
    assert log.sum() == len(frames) == r["out"][0, 0]


@pytest.mark.parametrize("seed", [21, 22])
def test_output_log_equals_output_spikes_of_each_tick(oracle_mod, seed):
    """The per-tick log sums to the window counts and, tick by tick, equals
    the number of spiking output-kind neurons of each id."""
    net = W.random_net(seed, 3, 2, axons=32, neurons=64, n_types=3, n_inputs=40, fanout_per_line=3,
                       delay_max=4, p_out=0.4, n_outputs=6)
    x = W.rate_coded_inputs(seed, 3, 12, net.n_inputs, 0.3)
    T = 16
    r = oracle_mod.run(net, x, T, trace=True, out_trace=True)
    log = r["out_trace"].astype(np.int64)
    assert log.sum() > 0
    assert (log.sum(axis=1) == r["out"]).all()
    st = r["spike_trace"].astype(np.int64)
    kind = net.dest["kind"]
    for o in range(net.n_outputs):
        m = (kind == W.KIND_OUTPUT) & (net.dest["axon"] == o)
        assert (log[:, :, o] == (st * m).sum(axis=(2, 3))).all(), o


def test_zero_spike_special_case(oracle_mod):
    """No input, leak <= 0, positive thresholds, v0 = 0: nothing ever fires
    and V_t = max(neg_thr, t * leak) (the shape of a grid with no mapped
    application)."""
    net = W.random_net(21, 4, 4, axons=32, neurons=32, leak=(-3, 0), pthr=(1, 9), nthr=(-20, -1))
    T = 12
    x = np.zeros((2, T, net.in_words), np.uint32)
    r = oracle_mod.run(net, x, T, trace=True)
    assert r["counters"][:, :3].sum() == 0
    for t in range(T):
        assert (r["v_trace"][:, t] == np.maximum(net.neg_thr, (t + 1) * net.leak)).all()


# ---------------------------------------------------------------------------
# brute force against the independent hop-by-hop restatement
# ---------------------------------------------------------------------------

def _compare_with_hop(oracle_mod, net, x, T):
    r = oracle_mod.run(net, x, T, trace=True)
    for s in range(x.shape[0]):
        vt, stt, out, cnt = hop_simulate(net, x[s], T)
        assert (r["v_trace"][s] == np.array(vt)).all(), s
        assert (r["spike_trace"][s] == np.array(stt)).all(), s
        assert r["out"][s].tolist() == out, s
        assert r["counters"][s].tolist() == cnt, s
    return r


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_bruteforce_two_core_exhaustive_inputs(oracle_mod, seed):
    """2-core nets, 3 input lines, every one of the 2**9 input patterns over 3
    ticks, simulated for 6 ticks, against the hop-by-hop restatement."""
    net = W.random_net(seed, 2, 1, axons=8, neurons=32, n_types=2, density=0.5, n_inputs=3,
                       fanout_per_line=3, delay_max=3, pthr=(1, 6), nthr=(-6, -1), p_core=0.6,
                       neg_mode=seed % 2)
    pats = np.array(list(itertools.product([0, 1], repeat=9)), np.uint32).reshape(-1, 3, 3)
    x = (pats * (1 << np.arange(3, dtype=np.uint32))).sum(axis=2, dtype=np.uint32)[:, :, None]
    r = _compare_with_hop(oracle_mod, net, x, 6)
    assert r["counters"][:, 1].sum() > 0


def test_bruteforce_mesh_with_hole(oracle_mod):
    """A 3 x 2 grid with one empty cell, long delays and multi-hop packets."""
    net = W.random_net(41, 3, 2, axons=32, neurons=32, n_types=4, n_inputs=6, fanout_per_line=4,
                       delay_max=15, holes=((1, 1),), p_core=0.7)
    x = W.rate_coded_inputs(41, 12, 10, net.n_inputs, 0.4)
    _compare_with_hop(oracle_mod, net, x, 24)


# ---------------------------------------------------------------------------
# error behaviour
# ---------------------------------------------------------------------------

def test_packet_to_empty_cell_is_an_error(oracle_mod):
    net = chain_net(1)
    net.dest[0, 0] = (1, 1, 0, 1, W.KIND_CORE)  # (1, 1) is off the 2 x 1 grid
    with pytest.raises(ValueError):
        oracle_mod.run(net, bits_inputs([1, 0]), 2)


def test_potential_outside_int32_is_an_error(oracle_mod):
    net = single_neuron_net(1, 0, 2**31 - 1, -2**31, 0, 0)
    net.v0[0, 0] = 2**31 - 1
    with pytest.raises(ValueError):
        oracle_mod.run(net, bits_inputs([1, 1]), 2)
