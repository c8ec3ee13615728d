"""A second, literal restatement of the RANC tick semantics, used only to pin
the C oracle by brute force on tiny networks.

It is written independently of the oracle and deliberately differently:

* future axon spikes are a set of (absolute tick, core, axon) events instead
  of a ring of scheduler rows;
* a packet travels hop by hop, one east/west step at a time and then one
  north/south step at a time, through the mesh (the serial RANC router of
  Sec. III-D, Fig. 2a), and is dropped into the destination core's event set;
* the neuron block sums weights over the set of active axons with Python
  integers.

The expected agreement with the oracle therefore also shows that direct
(single-step) routing reaches the same core as hop-by-hop routing.
"""


def _bit(words, i):
    return (int(words[i // 32]) >> (i % 32)) & 1


def simulate(net, inputs, n_ticks):
    """Returns (v_trace, spike_trace, out, counters) for one sample.

    ``inputs`` is [t_in][words] for this sample."""
    C, A, N = net.n_cores, net.axons, net.neurons
    pos = {(int(net.core_xy[c, 0]), int(net.core_xy[c, 1])): c for c in range(C)}
    syn = [[[_bit(net.crossbar[c, a], n) for n in range(N)] for a in range(A)] for c in range(C)]
    V = {(c, n): int(net.v0[c, n]) for c in range(C) for n in range(N)}
    events = set()
    out = [0] * net.n_outputs
    spikes = packets = outputs = syn_events = 0
    v_trace, s_trace = [], []
    t_in = len(inputs)
    for t in range(n_ticks):
        active = {c: set() for c in range(C)}
        for (tick, c, a) in list(events):
            if tick == t:
                active[c].add(a)
                events.discard((tick, c, a))
        if t < t_in:
            for line in range(net.n_inputs):
                if _bit(inputs[t], line):
                    for k in range(int(net.in_offsets[line]), int(net.in_offsets[line + 1])):
                        active[int(net.in_core[k])].add(int(net.in_axon[k]))
        fired = []
        for c in range(C):
            for n in range(N):
                total = 0
                for a in sorted(active[c]):
                    if syn[c][a][n]:
                        total += int(net.weight[c, int(net.axon_type[c, a]), n])
                        syn_events += 1
                v = V[(c, n)] + total + int(net.leak[c, n])
                if v >= int(net.pos_thr[c, n]):
                    fired.append((c, n))
                    v = int(net.reset[c, n])
                elif v < int(net.neg_thr[c, n]):
                    v = int(net.neg_thr[c, n]) if net.neg_mode == 0 else int(net.reset[c, n])
                V[(c, n)] = v
        for (c, n) in fired:
            spikes += 1
            d = net.dest[c, n]
            kind = int(d["kind"])
            if kind == 1:
                x, y = int(net.core_xy[c, 0]), int(net.core_xy[c, 1])
                tx, ty = x + int(d["dx"]), y + int(d["dy"])
                while x != tx:
                    x += 1 if tx > x else -1
                    assert 0 <= x < net.grid_w
                while y != ty:
                    y += 1 if ty > y else -1
                    assert 0 <= y < net.grid_h
                events.add((t + int(d["delay"]), pos[(x, y)], int(d["axon"])))
                packets += 1
            elif kind == 2:
                out[int(d["axon"])] += 1
                outputs += 1
        v_trace.append([[V[(c, n)] for n in range(N)] for c in range(C)])
        s_trace.append([[1 if (c, n) in set(fired) else 0 for n in range(N)] for c in range(C)])
    return v_trace, s_trace, out, [spikes, packets, outputs, syn_events, n_ticks]
