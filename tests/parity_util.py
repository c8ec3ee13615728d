"""Helpers shared by the GPU parity tests (comparison side only)."""

import numpy as np


def mix64(z):
    """SplitMix64 output mixing function on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def digest(v):
    """sum_i mix64((i << 32) | uint32(V_i)) mod 2**64 over the flat [B, C, N] index."""
    v = np.ascontiguousarray(v, dtype=np.int32).ravel()
    i = np.arange(v.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(mix64((i << np.uint64(32)) | v.view(np.uint32).astype(np.uint64)).sum(dtype=np.uint64))


def unpack_spikes(words, neurons):
    """[..., N/32] uint32 words -> [..., N] 0/1 uint8."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return b.reshape(*w.shape[:-1], neurons)


def gpu_trace(sim, n_ticks):
    """Step one tick at a time and read V, spikes and digest after each."""
    vs, ss, ds = [], [], []
    for _ in range(n_ticks):
        sim.step(1)
        v, s, d = sim.state()
        vs.append(v)
        ss.append(unpack_spikes(s, sim.net.neurons))
        ds.append(d)
    return np.stack(vs, 1), np.stack(ss, 1), ds


def idle_core_ticks(net, x, ref, n_ticks):
    """[n_ticks, C] True where the core received no packet and no input in any
    sample (computed from the oracle's spike trace)."""
    C, A = net.n_cores, net.axons
    act = np.zeros((n_ticks, C), bool)
    pos = {(int(a), int(b)): k for k, (a, b) in enumerate(net.core_xy)}
    d = net.dest
    fired = ref["spike_trace"].any(0)  # [ticks, C, N]
    for t in range(n_ticks):
        for c, n in zip(*np.nonzero(fired[t])):
            if d["kind"][c, n] == 1:
                tt = t + int(d["delay"][c, n])
                if tt < n_ticks:
                    act[tt, pos[(int(net.core_xy[c, 0] + d["dx"][c, n]), int(net.core_xy[c, 1] + d["dy"][c, n]))]] = True
    driven = np.zeros(C, bool)
    driven[np.asarray(net.in_core)] = True
    for t in range(min(x.shape[1], n_ticks)):
        act[t] |= driven
    return ~act
