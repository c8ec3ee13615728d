"""Design sweeps: many independent RANC networks simulated together.

Exploring RANC's configuration space means simulating many variants of a
network (Sec. I, Sec. V).  A sweep is run here with as few launches per tick
as possible.  Plans:

* ``multi`` (the default through ``auto``): every network whose core shape the
  multi-network path takes (axons a multiple of 64 up to 512, neurons a
  multiple of 128 up to 512) joins one multi-network handle
  (``ranc_create_multi``) per negative-threshold mode, so one tick launch
  updates every core of every such network; the rest fall back to ``combined``.
  ``auto`` also tunes that handle: it times every weight-stage depth and a few
  split cost settings (``ranc_set_multi_tuning``) on the first ``probe``
  samples and keeps the fastest (cached by the sweep's signature when
  ``cache`` names a JSON file).
* ``combined``: networks of one *shape class* are merged into one combined
  network (below), one tick launch per class.
* ``separate``: one handle per network.

Combined network of a class (exact: each member's results are those of
simulating it alone):

* cores: member k's cores keep their positions shifted down by the summed grid
  heights of members 0..k-1, so every packet stays inside its own member (the
  destination offsets are unchanged);
* input lines: line i feeds every member that has a line i (a sweep presents
  the same samples to every configuration);
* output bus: member k's ids are shifted by the summed id counts of members
  0..k-1;
* padding (only the axon-type count and, when needed, neurons or axons up to
  the class size): padded axons are never driven (no input line and no packet
  reaches them), padded neurons have no connections, no leak, V = 0 and
  theta+ = 1, so they never fire; every padded value also fits the narrowest
  potential format, which is decided per class.

A class is (path, axons, neurons, negative-threshold mode, potential format):
cores with at most 256 axons and neurons go to the batched (tensor-core) path,
padded to 128 or 256 neurons and a multiple of 64 axons; larger cores go to the
plain path with their own sizes.  Each network's counters are read through
``ranc_read_core_counters``.
"""

import json
import os
import time

import numpy as np

from . import ranc

FORMAT_NAMES = {ranc.RANC_POTENTIAL_INT32: "int32", ranc.RANC_POTENTIAL_INT16: "int16",
                ranc.RANC_POTENTIAL_FP16: "fp16"}


def potential_format(net):
    """The storage the library chooses for this network's potentials on the
    batched path (asked from the library: ranc_desc_potential_format)."""
    return ranc.ranc_desc_potential_format(net, ranc.RANC_PATH_BATCHED)


def multi_ok(net):
    """Whether the multi-network path takes this network's core shape."""
    return net.axons % 64 == 0 and 64 <= net.axons <= 512 and net.neurons % 128 == 0 and 128 <= net.neurons <= 512


def shape_class(net):
    """(path, axons, neurons, neg_mode, format) of the class the network joins."""
    A, N = net.axons, net.neurons
    if A <= 256 and N <= 256:
        return (ranc.RANC_PATH_BATCHED, -(-A // 64) * 64, 128 if N <= 128 else 256, net.neg_mode,
                potential_format(net))
    return (ranc.RANC_PATH_PLAIN, A, N, net.neg_mode, ranc.RANC_POTENTIAL_INT32)


def combine(nets, axons=None, neurons=None):
    """One network holding every member of `nets` (same negative mode),
    padded to `axons` x `neurons` per core.  Returns (net, core_offsets,
    output_offsets)."""
    from ranc_workloads import nets as NT
    A = axons or max(n.axons for n in nets)
    N = neurons or max(n.neurons for n in nets)
    assert N % 32 == 0 and A % 32 == 0 and len({n.neg_mode for n in nets}) == 1
    K = max(n.n_types for n in nets)
    C = sum(n.n_cores for n in nets)
    coff = np.concatenate([[0], np.cumsum([n.n_cores for n in nets])])
    ooff = np.concatenate([[0], np.cumsum([n.n_outputs for n in nets])])
    yoff = np.concatenate([[0], np.cumsum([n.grid_h for n in nets])])
    xy = np.zeros((C, 2), np.int16)
    xbar = np.zeros((C, A, N // 32), np.uint32)
    typ = np.zeros((C, A), np.uint8)
    w = np.zeros((C, K, N), np.int16)
    leak, v0, reset = (np.zeros((C, N), np.int32) for _ in range(3))
    pthr, nthr = np.ones((C, N), np.int32), np.full((C, N), -1, np.int32)
    dest = NT.empty_dest(C, N)
    lines, cores, axs = [], [], []
    for k, n in enumerate(nets):
        c0, c1, nn, na = coff[k], coff[k + 1], n.neurons, n.axons
        xy[c0:c1] = n.core_xy + np.array([0, yoff[k]], np.int16)
        xbar[c0:c1, :na, :nn // 32] = n.crossbar
        typ[c0:c1, :na] = n.axon_type
        w[c0:c1, :n.n_types, :nn] = n.weight
        for dst, src in ((leak, n.leak), (v0, n.v0), (reset, n.reset), (pthr, n.pos_thr), (nthr, n.neg_thr)):
            dst[c0:c1, :nn] = src
        d = n.dest.copy()
        d["axon"] = np.where(d["kind"] == NT.KIND_OUTPUT, d["axon"] + ooff[k], d["axon"])
        dest[c0:c1, :nn] = d
        cnt = np.diff(n.in_offsets)
        lines.append(np.repeat(np.arange(n.n_inputs), cnt))
        cores.append(n.in_core + c0)
        axs.append(n.in_axon)
    lines, cores, axs = np.concatenate(lines), np.concatenate(cores), np.concatenate(axs)
    order = np.argsort(lines, kind="stable")
    n_in = max(n.n_inputs for n in nets)
    offs = np.concatenate([[0], np.cumsum(np.bincount(lines, minlength=n_in))])
    net = NT.make_net("combined", max(n.grid_w for n in nets), int(yoff[-1]), xy, ("packed", xbar, N), typ, w,
                      leak, pthr, nthr, reset, dest, n_in, int(ooff[-1]), ("csr", offs, cores[order], axs[order]),
                      v0=v0, weight_bits=max(n.weight_bits for n in nets), neg_mode=nets[0].neg_mode)
    return net, coff, ooff


class _Group:
    """Members of one class simulated by one combined handle or one handle each."""

    def __init__(self, key, members, nets, batch, plan):
        self.key, self.members, self.plan = key, members, plan
        path, A, N = key[0], key[1], key[2]
        if plan == "combined":
            net, self.coff, self.ooff = combine([nets[i] for i in members], A, N)
            self.sims = [ranc.Sim(net, batch, path)]
        else:
            self.sims = [ranc.Sim(nets[i], batch, path) for i in members]

    def run(self, nets, x, window):
        """Per-member output counts [S, n_out] for x [S, t_in, words]."""
        out = {}
        if self.plan == "combined":
            c = self.sims[0].run_samples(x, window)
            for j, i in enumerate(self.members):
                out[i] = c[:, self.ooff[j]:self.ooff[j + 1]]
        else:
            for s, i in zip(self.sims, self.members):
                out[i] = s.run_samples(x[..., :(nets[i].n_inputs + 31) // 32], window)
        return out

    def counters(self):
        res = {}
        if self.plan == "combined":
            for j, i in enumerate(self.members):
                res[i] = self.sims[0].core_counters(self.coff[j], self.coff[j + 1])
        else:
            for s, i in zip(self.sims, self.members):
                res[i] = s.counters()[:4]
        return res

    def reset(self):
        for s in self.sims:
            s.reset()

    def close(self):
        for s in self.sims:
            s.close()
        self.sims = []


class _MultiGroup:
    """Members simulated by one multi-network handle (one tick launch)."""

    def __init__(self, key, members, nets, batch, tuning=None):
        self.key, self.members, self.plan = key, members, "multi"
        self.sim = ranc.MultiSim([nets[i] for i in members], batch)
        self.sims = [self.sim]
        if tuning is not None:
            self.sim.set_tuning(*tuning)

    def run(self, nets, x, window):
        outs = self.sim.run_samples(x[..., :(self.sim.n_inputs + 31) // 32], window)
        return dict(zip(self.members, outs))

    def counters(self):
        return dict(zip(self.members, self.sim.counters()))

    def reset(self):
        self.sim.reset()

    def close(self):
        self.sim.close()
        self.sims = []


# Split cost settings (cost_item, cost_mma, cost_slice) the tuner tries beside
# every weight-stage depth: the library's default (a fit of the kernel's
# measured per-item, per-slice and per-MMA-group times) and three neighbours.
COST_CANDIDATES = ((4, 1, 3), (2, 1, 3), (6, 1, 3), (4, 1, 2))


class Sweep:
    """Many networks, one call: ``run_samples(inputs, window)`` returns each
    network's output counts; ``counters()`` each network's spikes, packets,
    output events and synaptic events.

    ``plan``: "auto" (the multi-network plan with its pipeline and split
    settings tuned on the first ``probe`` samples of the first run; the
    candidates' times and the choice are kept in ``tuning`` and, when
    ``cache`` names a JSON file, reused for the same sweep signature),
    "multi" (the same with the library's default settings), "combined" (one
    handle per shape class) or "separate" (one handle per network)."""

    def __init__(self, nets, batch, plan="auto", probe=128, cache=None):
        self.nets, self.batch, self.plan, self.probe, self.cache = list(nets), int(batch), plan, probe, cache
        classes = {}
        for i, n in enumerate(self.nets):
            if plan in ("auto", "multi") and multi_ok(n):
                key = ("multi", n.neg_mode)
            else:
                key = shape_class(n)
            classes.setdefault(key, []).append(i)
        self.classes = classes
        self.groups = None
        self.tuning = {}

    def _signature(self, key, members):
        cores = sum(self.nets[i].n_cores for i in members)
        if key[0] == "multi":
            shapes = sorted({(self.nets[i].axons, self.nets[i].neurons) for i in members})
            return f"multi-neg{key[1]}-nets{len(members)}-cores{cores}-shapes{shapes}-b{self.batch}-costs3"
        return f"path{key[0]}-A{key[1]}-N{key[2]}-neg{key[3]}-fmt{key[4]}-nets{len(members)}-cores{cores}-b{self.batch}"

    def _load_cache(self):
        if self.cache and os.path.exists(self.cache):
            with open(self.cache) as f:
                return json.load(f)
        return {}

    def _tune_multi(self, g, xp, window):
        """Times every (weight stages, split costs) candidate on the probe
        samples (one warm-up run each) and sets the fastest."""
        mx = g.sim.tuning()[1]
        times = {}
        for stages in range(2, mx + 1):
            for costs in COST_CANDIDATES:
                g.sim.set_tuning(stages, *costs)
                g.run(self.nets, xp, window)
                t0 = time.perf_counter()
                g.run(self.nets, xp, window)
                times[",".join(str(v) for v in (stages,) + tuple(costs))] = time.perf_counter() - t0
        best = min(times, key=times.get)
        return [int(v) for v in best.split(",")], times

    def _build(self, x, window):
        cached = self._load_cache()
        groups = []
        xp = x[:min(self.probe, x.shape[0])]
        for key, members in self.classes.items():
            sig = self._signature(key, members)
            if key[0] == "multi":
                if self.plan == "auto" and sig in cached:
                    self.tuning[sig] = dict(cached[sig], cached=True)
                    groups.append(_MultiGroup(key, members, self.nets, self.batch, cached[sig]["choice"]))
                    continue
                g = _MultiGroup(key, members, self.nets, self.batch)
                if self.plan == "auto":
                    choice, times = self._tune_multi(g, xp, window)
                    g.sim.set_tuning(*choice)
                    g.sim.reset()
                    self.tuning[sig] = {"choice": choice, "seconds": times, "probe_samples": int(xp.shape[0])}
                    cached[sig] = self.tuning[sig]
                groups.append(g)
                continue
            choice = "separate" if len(members) == 1 else ("combined" if self.plan in ("auto", "multi") else self.plan)
            groups.append(_Group(key, members, self.nets, self.batch, choice))
        if self.cache and self.plan == "auto":
            with open(self.cache, "w") as f:
                json.dump(cached, f, indent=1)
        return groups

    def run_samples(self, inputs, window):
        """inputs uint32 [S, t_in, words] (words for the widest input count)
        -> list of per-network counts [S, n_outputs], in network order."""
        x = np.ascontiguousarray(inputs, dtype=np.uint32)
        if self.groups is None:
            self.groups = self._build(x, window)
        out = {}
        for g in self.groups:
            out.update(g.run(self.nets, x, window))
        return [out[i] for i in range(len(self.nets))]

    def counters(self):
        """[n_networks, 4] spikes, packets, outputs, synaptic events since the
        handles were created or reset."""
        res = {}
        for g in self.groups or []:
            res.update(g.counters())
        return np.stack([res[i] for i in range(len(self.nets))])

    def reset(self):
        for g in self.groups or []:
            g.reset()

    def plans(self):
        return [(g.key, g.plan, list(g.members)) for g in self.groups or []]

    def multi_handle(self):
        """The MultiSim of the multi plan's only handle (None if there is none or several)."""
        m = [g.sim for g in self.groups or [] if g.plan == "multi"]
        return m[0] if len(m) == 1 else None

    def close(self):
        for g in self.groups or []:
            g.close()
        self.groups = None
