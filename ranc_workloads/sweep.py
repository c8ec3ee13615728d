"""Seeded design sweeps: many independent random RANC networks of ragged shape.

The paper motivates GPU simulation by the cost of exploring RANC's
configuration space (Sec. I, Sec. V: core sizes, weight bit widths, axon types,
thresholds and delays are all parameters).  A sweep here is a list of
networks whose shapes are drawn from that space: core size (axons x neurons)
from a set such as {128, 256, 512}^2, weight bits {4, 6, 9}, 2 or 4 axon
types, crossbar density U[0.1, 0.5], delays U{1..15}, a core count from a
range, and one shared set of input lines (every configuration sees the same
samples).  Each network is a random recurrent graph on a near-square grid:
every neuron sends to a random core and axon (probability p_core), to one of
the output ids (p_out) or nowhere.  This module builds inputs only; it
simulates nothing.
"""

from dataclasses import dataclass

import numpy as np

from . import nets as NT
from . import rng

STREAMS = dict(spec=61, syn=62, typ=63, w=64, leak=65, thr=66, dest=67, fan=68)


@dataclass(frozen=True)
class SweepSpec:
    cores: int
    axons: int
    neurons: int
    weight_bits: int
    n_types: int
    density: float
    delay_max: int
    neg_mode: int


def sweep_specs(seed, n, core_range=(64, 1024), sizes=(128, 256, 512), weight_bits=(4, 6, 9), types=(2, 4),
                density=(0.1, 0.5), delay_max=15, neg_modes=(0,)):
    """n seeded configurations drawn uniformly from the given choices."""
    u = rng.uniform_int(seed, STREAMS["spec"], (n, 8), 0, 2**31 - 1)
    out = []
    for r in u:
        out.append(SweepSpec(cores=int(core_range[0] + r[0] % (core_range[1] - core_range[0] + 1)),
                             axons=int(sizes[r[1] % len(sizes)]), neurons=int(sizes[r[2] % len(sizes)]),
                             weight_bits=int(weight_bits[r[3] % len(weight_bits)]),
                             n_types=int(types[r[4] % len(types)]),
                             density=round(float(density[0] + (density[1] - density[0]) * (r[5] % 1001) / 1000), 3),
                             delay_max=int(1 + r[6] % delay_max), neg_mode=int(neg_modes[r[7] % len(neg_modes)])))
    return out


def sweep_net(seed, index, spec, n_inputs=1024, n_outputs=10, fanout=8, p_core=0.5, p_out=0.05, chunk=16):
    """Network `index` of a sweep with shape `spec` (a :class:`ranc_workloads.Net`).

    Weights U[-wmax, wmax] with wmax = 2^(bits-1) - 1, leak U[-wmax/8, 0],
    theta+ U[wmax, 4 wmax], theta- = -4 wmax, reset 0."""
    C, A, N, K = spec.cores, spec.axons, spec.neurons, spec.n_types
    s = (seed * 1000003 + index) & 0xFFFFFFFF
    wmax = (1 << (spec.weight_bits - 1)) - 1
    gw = int(np.ceil(np.sqrt(C)))
    gh = (C + gw - 1) // gw
    xy = np.stack([np.arange(C) % gw, np.arange(C) // gw], 1).astype(np.int16)
    packed = np.zeros((C, A, N // 32), np.uint32)
    for c0 in range(0, C, chunk):  # bounded temporaries for large cores
        c1 = min(C, c0 + chunk)
        dense = rng.bernoulli(s, STREAMS["syn"], (c1 - c0, A, N), spec.density, offset=c0 * A * N)
        packed[c0:c1] = NT.pack_bits_lsb(dense)
    typ = rng.uniform_int(s, STREAMS["typ"], (C, A), 0, K - 1)
    w = rng.uniform_int(s, STREAMS["w"], (C, K, N), -wmax, wmax)
    leak = -rng.uniform_int(s, STREAMS["leak"], (C, N), 0, max(wmax // 8, 0))
    pthr = rng.uniform_int(s, STREAMS["thr"], (C, N), wmax, 4 * wmax)
    u = rng.uniform_int(s, STREAMS["dest"], (C, N, 4), 0, 2**31 - 1)
    dest = NT.empty_dest(C, N)
    r = u[..., 0] % 1000
    core = r < p_core * 1000
    out = (~core) & (r < (p_core + p_out) * 1000)
    dc = u[..., 1] % C
    dest["dx"] = np.where(core, xy[dc, 0] - xy[:, None, 0], 0)
    dest["dy"] = np.where(core, xy[dc, 1] - xy[:, None, 1], 0)
    dest["axon"] = np.where(core, u[..., 2] % A, np.where(out, u[..., 2] % n_outputs, 0))
    dest["delay"] = np.where(core, 1 + u[..., 3] % spec.delay_max, np.where(out, 1, 0))
    dest["kind"] = np.where(core, NT.KIND_CORE, np.where(out, NT.KIND_OUTPUT, NT.KIND_NONE))
    f = rng.uniform_int(s, STREAMS["fan"], (n_inputs, fanout, 2), 0, 2**31 - 1)
    fc, fa = (f[..., 0] % C).ravel(), (f[..., 1] % A).ravel()
    offs = np.arange(0, n_inputs * fanout + 1, fanout)
    return NT.make_net(f"sweep-{seed}-{index}", gw, gh, xy, ("packed", packed, N), typ, w, leak, pthr, -4 * wmax, 0,
                       dest, n_inputs, n_outputs, ("csr", offs, fc, fa), weight_bits=spec.weight_bits,
                       neg_mode=spec.neg_mode, meta=dict(spec=spec, index=index))


def sweep(seed, n, workers=None, **spec_kw):
    """The n networks of a sweep (list of Net), built on `workers` threads
    (numpy releases the interpreter lock in its array loops)."""
    import concurrent.futures as cf
    import os
    specs = sweep_specs(seed, n, **spec_kw)
    workers = workers or min(8, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda a: sweep_net(seed, a[0], a[1]), enumerate(specs)))
