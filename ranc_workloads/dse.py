"""Seeded design space of RANC configurations for design-space exploration.

A design point changes the architectural parameters the paper lists as the
reasons for long design sweeps (Sec. I, Sec. V): cores in use, neurons per
core, weight bit width, axon types per core, crossbar density, thresholds,
leak and the largest packet delay.  Every point is derived from one fixed
seeded master network so that two points differ only by those parameters,
and so that their outputs on the same inputs can be compared with a nominal
point.  This module builds inputs only; it simulates nothing.

Master layout (maximum 12 replicas): replica r has 16 patch cores in layer 1
(16 x 16 patches of the 28 x 28 input at offsets (4i, 4j)) and 4 cores in
layer 2; neuron n < 64 of its patch core p feeds its layer-2 core
4r + (64p + n) // 256, axon (64p + n) % 256; layer-2 neurons 0..9 drive output
ids 0..9, summed over the replicas in use (an ensemble).
"""

from dataclasses import dataclass

import numpy as np

from . import nets as NT
from . import rng

R_MAX, PATCHES, A, N_MAX, K_MAX = 12, 16, 256, 256, 4
L2_PER_R = 4
C_MAX = PATCHES * R_MAX + L2_PER_R * R_MAX
WB_CHOICES = (4, 6, 9)
STREAMS = dict(syn=21, typ=22, w=23, thr=24, leak=25, delay=26, cand=27, proto=28, spikes=29)


@dataclass(frozen=True)
class Point:
    replicas: int      # 1..12 -> 20 * replicas cores
    neurons: int       # 128 or 256 neurons per core
    weight_bits: int   # 4, 6 or 9
    n_types: int       # 2 or 4 axon types
    density: float     # crossbar density
    thr_scale: float   # multiplies the thresholds
    leak_max: float    # largest leak magnitude, in units of 1/255 of the weight range
    delay_max: int     # delays drawn from 1..delay_max

    def features(self):
        """Inputs of the surrogate, scaled to about [0, 1]."""
        return np.array([self.replicas / R_MAX, self.neurons == 256, self.weight_bits == 4, self.weight_bits == 6,
                         self.weight_bits == 9, self.n_types == 4, self.density,
                         np.log2(self.thr_scale) / 2 + 0.5, self.leak_max / 8, self.delay_max / 15],
                        dtype=np.float32)


NOMINAL = Point(replicas=12, neurons=256, weight_bits=9, n_types=4, density=0.3, thr_scale=1.0, leak_max=4.0,
                delay_max=4)
N_FEATURES = 10


class Master:
    """Master random fields of the largest network (seeded once)."""

    def __init__(self, seed=0x5EEDD5E):
        self.seed = seed
        C = C_MAX
        self.u_syn = (rng.uniform_int(seed, STREAMS["syn"], (C, A, N_MAX), 0, 255)).astype(np.uint8)
        self.typ = rng.uniform_int(seed, STREAMS["typ"], (C, A), 0, K_MAX - 1).astype(np.uint8)
        self.w = (rng.uniform_int(seed, STREAMS["w"], (C, K_MAX, N_MAX), -1000, 1000) / 1000.0)
        self.thr = 0.25 + 0.75 * rng.uniform_int(seed, STREAMS["thr"], (C, N_MAX), 0, 1000) / 1000.0
        self.leak = rng.uniform_int(seed, STREAMS["leak"], (C, N_MAX), 0, 1000) / 1000.0
        self.delay_u = rng.uniform_int(seed, STREAMS["delay"], (C, N_MAX), 0, 999) / 1000.0


def build(master, p):
    """The network of design point p (a ranc_workloads Net)."""
    R, N, wb, K = p.replicas, p.neurons, p.weight_bits, p.n_types
    l1 = np.arange(PATCHES * R)                       # layer-1 cores in use
    l2 = PATCHES * R_MAX + np.arange(L2_PER_R * R)    # layer-2 cores in use
    cores = np.concatenate([l1, l2])
    C1, C = len(l1), len(cores)
    wmax = (1 << (wb - 1)) - 1
    syn = master.u_syn[cores][:, :, :N] < np.uint8(min(255, int(round(p.density * 256))))
    typ = master.typ[cores] % K
    w = np.rint(master.w[cores][:, :K, :N] * wmax).astype(np.int16)
    pthr = np.maximum(1, np.rint(p.thr_scale * master.thr[cores][:, :N] * wmax * 8)).astype(np.int32)
    leak = -np.rint(master.leak[cores][:, :N] * p.leak_max * wmax / 255.0).astype(np.int32)
    nthr = -4 * wmax
    delay = 1 + np.floor(master.delay_u[cores][:, :N] * p.delay_max).astype(np.int32)
    # grid: layer-1 core (r, patch) at (patch, r); layer-2 core k at (k % 16, 12 + k // 16)
    xy = np.zeros((C, 2), np.int16)
    xy[:C1, 0] = l1 % PATCHES
    xy[:C1, 1] = l1 // PATCHES
    k2 = np.arange(len(l2))
    xy[C1:, 0] = k2 % 16
    xy[C1:, 1] = R_MAX + k2 // 16
    dest = NT.empty_dest(C, N)
    # replica r's patch p, neuron n < 64 -> its own layer-2 core 4r + (64p + n) // 256, axon (64p + n) % 256
    r_of = (l1 // PATCHES)[:, None]
    g = 64 * (l1 % PATCHES)[:, None] + np.arange(64)[None, :]
    dst = C1 + L2_PER_R * r_of + g // 256
    dest["dx"][:C1, :64] = xy[dst, 0] - xy[:C1, None, 0]
    dest["dy"][:C1, :64] = xy[dst, 1] - xy[:C1, None, 1]
    dest["axon"][:C1, :64] = g % 256
    dest["delay"][:C1, :64] = delay[:C1, :64]
    dest["kind"][:C1, :64] = NT.KIND_CORE
    dest["axon"][C1:, :10] = np.arange(10)
    dest["delay"][C1:, :10] = 1
    dest["kind"][C1:, :10] = NT.KIND_OUTPUT
    # input fan-out CSR grouped by line (pixel (r, q) of patch (i, j) on axon 16 r + q)
    c = np.repeat(np.arange(C1), 256)
    pi, pj = np.divmod(c % PATCHES, 4)
    rq = np.tile(np.arange(256), C1)
    lines = (4 * pi + rq // 16) * 28 + (4 * pj + rq % 16)
    order = np.lexsort((rq, c, lines))
    counts = np.bincount(lines, minlength=784)
    offs = np.concatenate([[0], np.cumsum(counts)])
    fan = ("csr", offs, c[order], rq[order])
    return NT.make_net(f"dse-{p}", 16, R_MAX + 3, xy, syn.astype(np.uint8), typ, w, leak, pthr, nthr, 0, dest,
                       784, 10, fan, weight_bits=wb, meta=dict(point=p))


def sample_points(seed, n, offset=0):
    """n seeded design points, uniform over the space."""
    u = rng.uniform_int(seed, STREAMS["cand"], (n, 8), 0, 2**31 - 1, offset=offset * 8)
    pts = []
    for r in u:
        pts.append(Point(replicas=int(1 + r[0] % R_MAX), neurons=(128, 256)[r[1] % 2],
                         weight_bits=WB_CHOICES[r[2] % 3], n_types=(2, 4)[r[3] % 2],
                         density=round(float(0.1 + 0.4 * (r[4] % 1001) / 1000), 3),
                         thr_scale=round(float(2.0 ** (-1 + 2 * (r[5] % 1001) / 1000)), 3),
                         leak_max=round(float(8 * (r[6] % 1001) / 1000), 3), delay_max=int(1 + r[7] % 15)))
    return pts


def prototype_inputs(seed, n_samples, t_in=16, n_proto=10, p_on=0.35, p_off=0.03, frac_on=0.2):
    """Inputs with class structure: prototype k is a seeded set of about
    frac_on of the 784 pixels; sample s rate-codes prototype s % n_proto
    (Bernoulli p_on on its pixels, p_off elsewhere, every tick).  Packed
    [n_samples, t_in, 25] like rate_coded_inputs."""
    proto = rng.bernoulli(seed, STREAMS["proto"], (n_proto, 784), frac_on)
    u = rng.draws(seed, STREAMS["spikes"], n_samples * t_in * 784).reshape(n_samples, t_in, 784)
    p = np.where(proto[np.arange(n_samples) % n_proto][:, None, :] == 1, p_on, p_off)
    thr = np.floor(p * 2.0**32).astype(np.uint64)
    dense = ((u >> np.uint64(32)) < thr).astype(np.uint8)
    pad = np.zeros((n_samples, t_in, 800), np.uint8)
    pad[..., :784] = dense
    return NT.pack_bits_lsb(pad)
