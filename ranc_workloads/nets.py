"""Seeded synthetic RANC networks and rate-coded inputs.

A :class:`Net` is the network/core-parameter description that both the CUDA
library (``ranc_create``) and the CPU oracle take.  Its arrays use one
interchange format:

* ``core_xy``   int16  [C, 2]        grid position (x, y) of each core
* ``crossbar``  uint32 [C, A, N/32]  synapse (a, n) is bit n%32 of word n/32
* ``axon_type`` uint8  [C, A]        axon type in [0, K)
* ``weight``    int16  [C, K, N]     one signed weight per (type, neuron)
* ``leak``, ``pos_thr``, ``neg_thr``, ``reset``, ``v0``  int32 [C, N]
* ``dest``      structured [C, N]    (dx int16, dy int16, axon uint16,
  delay uint8, kind uint8); kind 0 = none, 1 = core, 2 = output bus
  (the output id is the ``axon`` field)
* input fan-out CSR: line i feeds (in_core[k], in_axon[k]) for
  k in [in_offsets[i], in_offsets[i+1])
* inputs: uint32 [S, T, ceil(n_inputs/32)], line i of tick t is bit i%32 of
  word i/32.

The builders reproduce the shapes of the paper's MNIST workloads (Section IV,
Table I: 256 axons x 256 neurons per core, 28x28 inputs, 10 classes) with
random parameters, because the trained networks and the dataset are not part
of this project.  Nothing here simulates: the module only lays out inputs.
"""

from dataclasses import dataclass, field

import numpy as np

from . import rng

KIND_NONE, KIND_CORE, KIND_OUTPUT = 0, 1, 2
NEG_SATURATE, NEG_RESET = 0, 1

DEST_DTYPE = np.dtype([("dx", "<i2"), ("dy", "<i2"), ("axon", "<u2"),
                       ("delay", "u1"), ("kind", "u1")])

# stream ids of the fields of one workload
S_XBAR, S_TYPE, S_WEIGHT, S_LEAK, S_POSTHR, S_DELAY, S_INPUT, S_NEGTHR, S_RESET, S_DEST = range(1, 11)


@dataclass
class Net:
    name: str
    grid_w: int
    grid_h: int
    axons: int
    neurons: int
    n_types: int
    weight_bits: int
    neg_mode: int
    core_xy: np.ndarray
    crossbar: np.ndarray
    axon_type: np.ndarray
    weight: np.ndarray
    leak: np.ndarray
    pos_thr: np.ndarray
    neg_thr: np.ndarray
    reset: np.ndarray
    v0: np.ndarray
    dest: np.ndarray
    n_inputs: int
    n_outputs: int
    in_offsets: np.ndarray
    in_core: np.ndarray
    in_axon: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_cores(self):
        return int(self.core_xy.shape[0])

    @property
    def in_words(self):
        return (self.n_inputs + 31) // 32


def pack_bits_lsb(dense):
    """Pack a 0/1 array along its last axis (length multiple of 32) into uint32 words, LSB first."""
    dense = np.asarray(dense, dtype=np.uint8)
    *lead, n = dense.shape
    assert n % 32 == 0
    b = np.packbits(dense.reshape(*lead, n // 32, 32), axis=-1, bitorder="little")
    return b.view("<u4").reshape(*lead, n // 32).astype(np.uint32)


def fanout_csr(n_inputs, pairs):
    """CSR (offsets, core, axon) from a list of (line, core, axon) triples."""
    pairs = sorted(pairs)
    offsets = np.zeros(n_inputs + 1, dtype=np.int32)
    for line, _, _ in pairs:
        offsets[line + 1] += 1
    offsets = np.cumsum(offsets).astype(np.int32)
    core = np.array([p[1] for p in pairs], dtype=np.int32)
    axon = np.array([p[2] for p in pairs], dtype=np.int32)
    return offsets, core, axon


def make_net(name, grid_w, grid_h, core_xy, syn, axon_type, weight, leak, pos_thr,
             neg_thr, reset, dest, n_inputs, n_outputs, fanout, v0=None,
             weight_bits=9, neg_mode=NEG_SATURATE, meta=None):
    """Build a :class:`Net` from dense per-core arrays.

    ``syn`` is the dense 0/1 crossbar [C, A, N]; ``fanout`` a list of
    (line, core, axon) triples.
    """
    if isinstance(syn, tuple) and syn[0] == "packed":  # ("packed", uint32 [C, A, N/32], N)
        packed = np.ascontiguousarray(syn[1], dtype=np.uint32)
        C, A, N = packed.shape[0], packed.shape[1], int(syn[2])
    else:
        syn = np.asarray(syn, dtype=np.uint8)
        C, A, N = syn.shape
        packed = pack_bits_lsb(syn)
    as32 = lambda x: np.array(np.broadcast_to(np.asarray(x, dtype=np.int32), (C, N)), dtype=np.int32)
    if isinstance(fanout, tuple) and fanout[0] == "csr":  # ("csr", offsets, core, axon), already grouped by line
        offs, icore, iaxon = (np.ascontiguousarray(a, dtype=np.int32) for a in fanout[1:])
    else:
        offs, icore, iaxon = fanout_csr(n_inputs, fanout)
    return Net(
        name=name, grid_w=int(grid_w), grid_h=int(grid_h), axons=int(A), neurons=int(N),
        n_types=int(weight.shape[1]), weight_bits=int(weight_bits), neg_mode=int(neg_mode),
        core_xy=np.ascontiguousarray(np.asarray(core_xy, dtype=np.int16).reshape(C, 2)),
        crossbar=packed,
        axon_type=np.ascontiguousarray(np.asarray(axon_type, dtype=np.uint8).reshape(C, A)),
        weight=np.ascontiguousarray(np.asarray(weight, dtype=np.int16)),
        leak=as32(leak), pos_thr=as32(pos_thr), neg_thr=as32(neg_thr), reset=as32(reset),
        v0=as32(0 if v0 is None else v0),
        dest=np.ascontiguousarray(dest, dtype=DEST_DTYPE).reshape(C, N),
        n_inputs=int(n_inputs), n_outputs=int(n_outputs),
        in_offsets=offs, in_core=icore, in_axon=iaxon, meta=dict(meta or {}))


def empty_dest(C, N):
    return np.zeros((C, N), dtype=DEST_DTYPE)


# ---------------------------------------------------------------------------
# Workload 1: tiny 2-layer net, 5 cores (4 -> 1), 256 x 256 cores.
# ---------------------------------------------------------------------------

def tiny_5core(seed=0x5EED0001):
    """Four first-layer cores on x = 0..3 feed core 4; neurons 0-9 of core 4
    drive output-bus ids 0-9.  Pixel p feeds core p // 196, axon p % 196."""
    C, A, N, K = 5, 256, 256, 4
    syn = rng.bernoulli(seed, S_XBAR, (C, A, N), 0.25)
    atype = rng.uniform_int(seed, S_TYPE, (C, A), 0, K - 1)
    w = rng.uniform_int(seed, S_WEIGHT, (C, K, N), -64, 64)
    leak = rng.uniform_int(seed, S_LEAK, (C, N), -2, 0)
    pthr = rng.uniform_int(seed, S_POSTHR, (C, N), 32, 128)
    dest = empty_dest(C, N)
    for x in range(4):
        for n in range(64):
            dest[x, n] = (4 - x, 0, 64 * x + n, 1, KIND_CORE)
    for n in range(10):
        dest[4, n] = (0, 0, n, 1, KIND_OUTPUT)
    fan = [(p, p // 196, p % 196) for p in range(784)]
    xy = [(x, 0) for x in range(5)]
    return make_net("tiny-5core", 5, 1, xy, syn, atype, w, leak, pthr, -128, 0, dest,
                    784, 10, fan, weight_bits=8, meta=dict(seed=seed, t_in=8, window=9, p_in=0.15))


# ---------------------------------------------------------------------------
# Workload 2/3: MNIST-shaped 512-core tiled 3-layer net on a 32 x 16 grid.
# ---------------------------------------------------------------------------

# Leak and thresholds are not fixed by the workload statement; these values were
# chosen once so that every layer fires at 5-30 % per tick (about 20 % in layer 1
# while inputs arrive and about 24 % in layers 2 and 3 at steady state) and are
# frozen here.
MNIST512_PARAMS = dict(density=0.3, w_lo=-255, w_hi=255, leak_lo=-8, leak_hi=0,
                       pthr_lo=512, pthr_hi=2048, neg_thr=-1024, reset=0, delay_lo=1, delay_hi=4)


def mnist_512core(seed=0x5EED0512, **over):
    """Cores k = 0..511 sit at (k % 32, k // 32).

    * Layer 1, cores 0..383 (grid rows 0-11): core c sees the 16x16 patch at
      (4i, 4j), (i, j) = divmod(c % 16, 4), pixel (r, q) of the patch on axon
      16 r + q; c // 16 is the replica index (24 replicas).
    * Layer 2, cores 384..479 (rows 12-14): L1 neuron n < 64 of L1 core c has
      g = 64 c + n and targets L2 core g % 96, axon g // 96.
    * Layer 3, cores 480..511 (row 15): L2 neuron n < 64 of L2 core c has
      g = 64 c + n and targets L3 core g % 32, axon g // 32.
    * L3 neurons 0..9 drive output-bus ids 0..9 (summed over the 32 cores).
    """
    p = dict(MNIST512_PARAMS)
    p.update(over)
    C, A, N, K = 512, 256, 256, 4
    GW = 32
    syn = rng.bernoulli(seed, S_XBAR, (C, A, N), p["density"])
    atype = rng.uniform_int(seed, S_TYPE, (C, A), 0, K - 1)
    w = rng.uniform_int(seed, S_WEIGHT, (C, K, N), p["w_lo"], p["w_hi"])
    leak = rng.uniform_int(seed, S_LEAK, (C, N), p["leak_lo"], p["leak_hi"])
    pthr = rng.uniform_int(seed, S_POSTHR, (C, N), p["pthr_lo"], p["pthr_hi"])
    delay = rng.uniform_int(seed, S_DELAY, (C, N), p["delay_lo"], p["delay_hi"])
    xy = np.array([(k % GW, k // GW) for k in range(C)], dtype=np.int16)
    dest = empty_dest(C, N)
    L1, L2, L3 = 384, 96, 32
    for c in range(L1):
        for n in range(64):
            g = 64 * c + n
            dst = L1 + g % L2
            dest[c, n] = (xy[dst, 0] - xy[c, 0], xy[dst, 1] - xy[c, 1], g // L2, delay[c, n], KIND_CORE)
    for c2 in range(L2):
        c = L1 + c2
        for n in range(64):
            g = 64 * c2 + n
            dst = L1 + L2 + g % L3
            dest[c, n] = (xy[dst, 0] - xy[c, 0], xy[dst, 1] - xy[c, 1], g // L3, delay[c, n], KIND_CORE)
    for c3 in range(L3):
        c = L1 + L2 + c3
        for n in range(10):
            dest[c, n] = (0, 0, n, 1, KIND_OUTPUT)
    fan = []
    for c in range(L1):
        i, j = divmod(c % 16, 4)
        for r in range(16):
            for q in range(16):
                fan.append(((4 * i + r) * 28 + (4 * j + q), c, 16 * r + q))
    return make_net("mnist-512core", GW, 16, xy, syn, atype, w, leak, pthr, p["neg_thr"], p["reset"],
                    dest, 784, 10, fan, weight_bits=9,
                    meta=dict(seed=seed, t_in=16, window=24, p_in=0.15, layers=(L1, L2, L3), params=p))


# ---------------------------------------------------------------------------
# TrueNorth-sized reference grid with no application (Table I, Sec. IV).
# ---------------------------------------------------------------------------

def truenorth_ref(seed=0x5EED4096, grid=64, axons=256, neurons=256, density=0.3):
    """grid x grid cores of axons x neurons, random crossbars, weights and
    destinations, no input lines and non-positive leaks with positive
    thresholds: every tick performs the full update of every core but no
    neuron ever fires (the paper's scaling case with no mapped application).
    Built with array operations so the 4096-core grid takes seconds."""
    C, A, N, K = grid * grid, axons, neurons, 4
    packed = np.zeros((C, A, N // 32), np.uint32)
    step = 128
    for c0 in range(0, C, step):  # same draws as one call over (C, A, N), without the 2 GB temporary
        c1 = min(C, c0 + step)
        packed[c0:c1] = pack_bits_lsb(rng.bernoulli(seed, S_XBAR, (c1 - c0, A, N), density, offset=c0 * A * N))
    syn = ("packed", packed, N)
    atype = rng.uniform_int(seed, S_TYPE, (C, A), 0, K - 1)
    w = rng.uniform_int(seed, S_WEIGHT, (C, K, N), -255, 255)
    leak = rng.uniform_int(seed, S_LEAK, (C, N), -3, 0)
    pthr = rng.uniform_int(seed, S_POSTHR, (C, N), 64, 1024)
    nthr = rng.uniform_int(seed, S_NEGTHR, (C, N), -1024, -64)
    xy = np.stack([np.arange(C) % grid, np.arange(C) // grid], axis=1).astype(np.int16)
    u = rng.uniform_int(seed, S_DEST, (C, N, 4), 0, 2**31 - 1)
    dst = u[..., 0] % C
    dest = empty_dest(C, N)
    dest["dx"] = xy[dst, 0] - xy[:, None, 0]
    dest["dy"] = xy[dst, 1] - xy[:, None, 1]
    dest["axon"] = u[..., 1] % A
    dest["delay"] = 1 + u[..., 2] % 15
    dest["kind"] = KIND_CORE
    return make_net("truenorth-ref", grid, grid, xy, syn, atype, w, leak, pthr, nthr, 0, dest, 0, 10, [],
                    weight_bits=9, meta=dict(seed=seed, ticks=500))


# ---------------------------------------------------------------------------
# Inputs and small random nets for tests.
# ---------------------------------------------------------------------------

def rate_coded_inputs(seed, n_samples, t_in, n_inputs, p, first_sample=0, chunk=256):
    """Bernoulli(p) spikes per (sample, tick, line), packed [S, T, ceil(n/32)].

    Sample s uses draw indices ((s * t_in) + t) * n_inputs + line, so a
    sub-range of samples equals the same rows of a larger set."""
    W = (n_inputs + 31) // 32
    out = np.zeros((n_samples, t_in, W), dtype=np.uint32)
    for s0 in range(0, n_samples, chunk):
        s1 = min(n_samples, s0 + chunk)
        g0 = first_sample + s0
        dense = rng.bernoulli(seed, S_INPUT, ((s1 - s0), t_in, n_inputs), p,
                              offset=g0 * t_in * n_inputs)
        pad = np.zeros((s1 - s0, t_in, W * 32), dtype=np.uint8)
        pad[..., :n_inputs] = dense
        out[s0:s1] = pack_bits_lsb(pad)
    return out


def random_net(seed, grid_w, grid_h, axons=32, neurons=32, n_types=4, density=0.3,
               w_lim=7, weight_bits=4, n_inputs=16, n_outputs=4, fanout_per_line=2,
               delay_max=15, p_core=0.5, p_out=0.2, leak=(-2, 1), pthr=(1, 12),
               nthr=(-12, -1), reset=(-3, 3), neg_mode=NEG_SATURATE, v0=(0, 0), holes=()):
    """A small random net with every core-to-core destination on a real core.

    ``holes`` lists grid cells (x, y) left without a core."""
    cells = [(x, y) for y in range(grid_h) for x in range(grid_w) if (x, y) not in set(holes)]
    C, A, N, K = len(cells), axons, neurons, n_types
    syn = rng.bernoulli(seed, S_XBAR, (C, A, N), density)
    atype = rng.uniform_int(seed, S_TYPE, (C, A), 0, K - 1)
    w = rng.uniform_int(seed, S_WEIGHT, (C, K, N), -w_lim, w_lim)
    lk = rng.uniform_int(seed, S_LEAK, (C, N), *leak)
    pt = rng.uniform_int(seed, S_POSTHR, (C, N), *pthr)
    nt = rng.uniform_int(seed, S_NEGTHR, (C, N), *nthr)
    rs = rng.uniform_int(seed, S_RESET, (C, N), *reset)
    vv = rng.uniform_int(seed, S_RESET, (C, N), v0[0], v0[1], offset=C * N)
    u = rng.uniform_int(seed, S_DEST, (C, N, 4), 0, 2**31 - 1)
    dest = empty_dest(C, N)
    for c in range(C):
        for n in range(N):
            r = u[c, n, 0] % 1000
            if r < p_core * 1000:
                dc = int(u[c, n, 1] % C)
                dest[c, n] = (cells[dc][0] - cells[c][0], cells[dc][1] - cells[c][1],
                              u[c, n, 2] % A, 1 + u[c, n, 3] % delay_max, KIND_CORE)
            elif r < (p_core + p_out) * 1000:
                dest[c, n] = (0, 0, u[c, n, 2] % n_outputs, 1, KIND_OUTPUT)
    fu = rng.uniform_int(seed, S_DEST, (n_inputs, fanout_per_line, 2), 0, 2**31 - 1, offset=C * N * 4)
    fan = set()
    for i in range(n_inputs):
        for j in range(fanout_per_line):
            fan.add((i, int(fu[i, j, 0] % C), int(fu[i, j, 1] % A)))
    return make_net(f"random-{seed}", grid_w, grid_h, cells, syn, atype, w, lk, pt, nt, rs, dest,
                    n_inputs, n_outputs, sorted(fan), v0=vv, weight_bits=weight_bits,
                    neg_mode=neg_mode, meta=dict(seed=seed))


def layered_net(seed, layers=(2, 2, 2), axons=128, neurons=256, n_types=4, density=0.3, w_lim=60,
                weight_bits=12, n_inputs=64, n_outputs=8, fanout_per_line=3, delay_max=6, p_fwd=0.5,
                p_out=0.1, pthr=(1, 150), nthr=(-150, -1), leak=(-3, 0), reset=(-3, 0), v0=(-3, 0),
                neg_mode=NEG_SATURATE):
    """A feed-forward random net on one row of cores: a fraction ``p_fwd`` of
    the neurons of layer k send to a random core, axon and delay of layer
    k + 1, a fraction ``p_out`` of the last layer's neurons drive random
    output-bus ids, and the input lines drive layer 0 only.  Once the inputs
    stop, activity drains layer by layer, so cores fall idle and wake up again
    when the inputs resume."""
    C, A, N, K = int(sum(layers)), axons, neurons, n_types
    start = np.concatenate([[0], np.cumsum(layers)]).astype(int)
    cells = [(x, 0) for x in range(C)]
    syn = rng.bernoulli(seed, S_XBAR, (C, A, N), density)
    atype = rng.uniform_int(seed, S_TYPE, (C, A), 0, K - 1)
    w = rng.uniform_int(seed, S_WEIGHT, (C, K, N), -w_lim, w_lim)
    lk = rng.uniform_int(seed, S_LEAK, (C, N), *leak)
    pt = rng.uniform_int(seed, S_POSTHR, (C, N), *pthr)
    nt = rng.uniform_int(seed, S_NEGTHR, (C, N), *nthr)
    rs = rng.uniform_int(seed, S_RESET, (C, N), *reset)
    vv = rng.uniform_int(seed, S_RESET, (C, N), v0[0], v0[1], offset=C * N)
    u = rng.uniform_int(seed, S_DEST, (C, N, 4), 0, 2**31 - 1)
    dest = empty_dest(C, N)
    for k in range(len(layers)):
        for c in range(start[k], start[k + 1]):
            for n in range(N):
                r = u[c, n, 0] % 1000
                if k + 1 < len(layers):
                    if r < p_fwd * 1000:
                        dc = start[k + 1] + int(u[c, n, 1] % layers[k + 1])
                        dest[c, n] = (dc - c, 0, u[c, n, 2] % A, 1 + u[c, n, 3] % delay_max, KIND_CORE)
                elif r < p_out * 1000:
                    dest[c, n] = (0, 0, u[c, n, 2] % n_outputs, 1, KIND_OUTPUT)
    fu = rng.uniform_int(seed, S_DEST, (n_inputs, fanout_per_line, 2), 0, 2**31 - 1, offset=C * N * 4)
    fan = set()
    for i in range(n_inputs):
        for j in range(fanout_per_line):
            fan.add((i, int(fu[i, j, 0] % layers[0]), int(fu[i, j, 1] % A)))
    return make_net(f"layered-{seed}", C, 1, cells, syn, atype, w, lk, pt, nt, rs, dest, n_inputs, n_outputs,
                    sorted(fan), v0=vv, weight_bits=weight_bits, neg_mode=neg_mode,
                    meta=dict(seed=seed, layers=tuple(layers)))
