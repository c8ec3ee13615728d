"""Python binding of the RANC C ABI (``include/ranc.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
simulation work of its own; a failing call raises :class:`RancError` with the
library's reason.  Importing this module loads ``_lib/libranc.so`` and fails
loudly if it has not been built (``paper_2404_16208_gb300.build.build()``):
there is no fallback.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libranc.so")

RANC_OK, RANC_EINVAL, RANC_ENOMEM, RANC_ECUDA, RANC_ETIMEOUT, RANC_ESTATE = 0, -1, -2, -3, -4, -5
RANC_PATH_PLAIN, RANC_PATH_BATCHED = 0, 1
RANC_MEM_HOST, RANC_MEM_DEVICE = 0, 1
COUNTER_NAMES = ("spikes", "packets", "outputs", "synaptic_events", "ticks")
EXPORTED = ("ranc_create", "ranc_create_multi", "ranc_set_multi_tuning", "ranc_get_multi_tuning", "ranc_load_inputs", "ranc_load_inputs_device", "ranc_step", "ranc_read_outputs",
            "ranc_read_outputs_device", "ranc_read_state", "ranc_read_sample_state", "ranc_read_sample_state_noalloc",
            "ranc_read_counters", "ranc_read_core_counters", "ranc_get_tick", "ranc_reset",
            "ranc_run_samples", "ranc_run_stream", "ranc_save_state", "ranc_load_state", "ranc_set_kernel_timing",
            "ranc_read_kernel_timing", "ranc_launch_count", "ranc_graph_stats", "ranc_item_ticks", "ranc_item_classes", "ranc_network_item_classes",
            "ranc_potential_format", "ranc_desc_potential_format", "ranc_device_allocations", "ranc_destroy",
            "ranc_last_error")
RANC_POTENTIAL_INT32, RANC_POTENTIAL_INT16, RANC_POTENTIAL_FP16 = 0, 1, 2
RANC_XBAR_F16_FOLDED, RANC_XBAR_F8_PER_TYPE, RANC_XBAR_I8_MMA_SYNC = 0, 1, 2
XBAR_EXPORTED = ("ranc_xbar_create", "ranc_xbar_run", "ranc_xbar_sync", "ranc_xbar_destroy", "ranc_xbar_last_error")


class RancError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"RANC error {code}: {msg}")
        self.code = code


class ranc_dest(C.Structure):
    _fields_ = [("dx", C.c_int16), ("dy", C.c_int16), ("axon", C.c_uint16), ("delay", C.c_uint8),
                ("kind", C.c_uint8)]


class ranc_desc(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("grid_w", "grid_h", "n_cores", "axons", "neurons", "n_types",
                                          "weight_bits", "neg_mode")] + [
        ("core_xy", C.c_void_p), ("crossbar", C.c_void_p), ("axon_type", C.c_void_p), ("weight", C.c_void_p),
        ("leak", C.c_void_p), ("pos_thr", C.c_void_p), ("neg_thr", C.c_void_p), ("reset", C.c_void_p),
        ("v0", C.c_void_p), ("dest", C.c_void_p), ("n_inputs", C.c_int32), ("n_outputs", C.c_int32),
        ("in_offsets", C.c_void_p), ("in_core", C.c_void_p), ("in_axon", C.c_void_p)]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libranc.so is not built at {path}; run paper_2404_16208_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, u32p, u64p = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p
    sig = {
        "ranc_create": ([C.POINTER(ranc_desc), i32, i32, vp, C.POINTER(vp)], C.c_int),
        "ranc_create_multi": ([C.POINTER(C.POINTER(ranc_desc)), i32, i32, vp, C.POINTER(vp)], C.c_int),
        "ranc_set_multi_tuning": ([vp, i32, i32, i32, i32], C.c_int),
        "ranc_get_multi_tuning": ([vp] + [C.POINTER(i32)] * 5, C.c_int),
        "ranc_load_inputs": ([vp, u32p, i32], C.c_int),
        "ranc_load_inputs_device": ([vp, vp, i32], C.c_int),
        "ranc_step": ([vp, i32], C.c_int),
        "ranc_read_outputs": ([vp, u32p], C.c_int),
        "ranc_read_outputs_device": ([vp, vp], C.c_int),
        "ranc_read_state": ([vp, vp, vp, u64p], C.c_int),
        "ranc_read_sample_state": ([vp, i32, i32, vp, vp], C.c_int),
        "ranc_read_sample_state_noalloc": ([vp, i32, i32, vp, vp], C.c_int),
        "ranc_read_counters": ([vp, u64p], C.c_int),
        "ranc_read_core_counters": ([vp, i32, i32, u64p], C.c_int),
        "ranc_get_tick": ([vp, C.POINTER(i64)], C.c_int),
        "ranc_reset": ([vp], C.c_int),
        "ranc_run_samples": ([vp, vp, i32, i32, i32, vp, i32], C.c_int),
        "ranc_run_stream": ([vp, vp, i32, i32, vp, i32], C.c_int),
        "ranc_save_state": ([vp, vp, C.POINTER(C.c_size_t)], C.c_int),
        "ranc_load_state": ([vp, vp, C.c_size_t], C.c_int),
        "ranc_set_kernel_timing": ([vp, i32], C.c_int),
        "ranc_read_kernel_timing": ([vp, C.POINTER(C.c_double), C.POINTER(i64)], C.c_int),
        "ranc_launch_count": ([vp, C.POINTER(i64)], C.c_int),
        "ranc_graph_stats": ([vp, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "ranc_item_ticks": ([vp, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "ranc_item_classes": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "ranc_network_item_classes": ([vp, i32, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "ranc_potential_format": ([vp, C.POINTER(i32)], C.c_int),
        "ranc_desc_potential_format": ([C.POINTER(ranc_desc), i32, C.POINTER(i32)], C.c_int),
        "ranc_device_allocations": ([C.POINTER(i64)], C.c_int),
        "ranc_destroy": ([vp], None),
        "ranc_last_error": ([vp], C.c_char_p),
    }
    sig.update({  # crossbar-product formulations (include/ranc_xbar.h)
        "ranc_xbar_create": ([C.POINTER(ranc_desc), i32, vp, C.POINTER(vp)], C.c_int),
        "ranc_xbar_run": ([vp, vp, i32, vp, vp], C.c_int),
        "ranc_xbar_sync": ([vp], C.c_int),
        "ranc_xbar_destroy": ([vp], None),
        "ranc_xbar_last_error": ([vp], C.c_char_p),
    })
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


_lib = load_library()


def use_library(path):
    """Route every later call of this module through the library at `path`
    (for instance ``_lib/libranc_debug.so``, the build with device-side range
    checks) and return the one used before.  A handle must be used and
    destroyed through the library that created it."""
    global _lib
    prev, _lib = _lib, load_library(path)
    return prev


def _check(rc, h):
    if rc != RANC_OK:
        raise RancError(rc, _lib.ranc_last_error(h).decode())


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _desc(net):
    """A ranc_desc pointing into contiguous copies of ``net``'s arrays (which
    the caller keeps alive while the description is used)."""
    keep = [_c(net.core_xy, np.int16), _c(net.crossbar, np.uint32), _c(net.axon_type, np.uint8),
            _c(net.weight, np.int16), _c(net.leak, np.int32), _c(net.pos_thr, np.int32),
            _c(net.neg_thr, np.int32), _c(net.reset, np.int32), _c(net.v0, np.int32),
            np.ascontiguousarray(net.dest), _c(net.in_offsets, np.int32), _c(net.in_core, np.int32),
            _c(net.in_axon, np.int32)]
    assert keep[9].dtype.itemsize == C.sizeof(ranc_dest)
    d = ranc_desc(net.grid_w, net.grid_h, net.n_cores, net.axons, net.neurons, net.n_types, net.weight_bits,
                  net.neg_mode, *[_p(a) for a in keep[:10]], net.n_inputs, net.n_outputs,
                  *[_p(a) for a in keep[10:]])
    return d, keep


def ranc_create(net, batch, path=RANC_PATH_PLAIN, stream=0):
    """Create a simulator for ``net`` (any object with the fields of a RANC
    network description) and return the opaque handle."""
    d, keep = _desc(net)
    h = C.c_void_p()
    _check(_lib.ranc_create(C.byref(d), int(batch), int(path), C.c_void_p(int(stream)), C.byref(h)), None)
    return h


def ranc_create_multi(nets, batch, stream=0):
    """One batched handle simulating every network of ``nets`` (different
    core shapes allowed) with one tick launch for all of them."""
    descs, keep = [], []
    for n in nets:
        d, k = _desc(n)
        descs.append(d)
        keep.append(k)
    arr = (C.POINTER(ranc_desc) * len(descs))(*[C.pointer(d) for d in descs])
    h = C.c_void_p()
    _check(_lib.ranc_create_multi(arr, len(descs), int(batch), C.c_void_p(int(stream)), C.byref(h)), None)
    return h


def ranc_set_multi_tuning(h, weight_stages, cost_item, cost_mma, cost_slice):
    _check(_lib.ranc_set_multi_tuning(h, int(weight_stages), int(cost_item), int(cost_mma), int(cost_slice)), h)


def ranc_get_multi_tuning(h):
    """(weight_stages, max_weight_stages, cost_item, cost_mma, cost_slice) of a multi-network handle."""
    v = [C.c_int32() for _ in range(5)]
    _check(_lib.ranc_get_multi_tuning(h, *[C.byref(x) for x in v]), h)
    return tuple(x.value for x in v)


def ranc_load_inputs(h, bits):
    """``bits``: host uint32 [batch, ticks, ceil(n_inputs/32)]."""
    bits = _c(bits, np.uint32)
    _check(_lib.ranc_load_inputs(h, _p(bits), int(bits.shape[1]) if bits.ndim == 3 else 0), h)


def ranc_load_inputs_device(h, dev_ptr, n_ticks):
    _check(_lib.ranc_load_inputs_device(h, C.c_void_p(int(dev_ptr)), int(n_ticks)), h)


def ranc_step(h, n_ticks):
    _check(_lib.ranc_step(h, int(n_ticks)), h)


def ranc_read_outputs(h, batch, n_outputs):
    out = np.zeros((batch, n_outputs), np.uint32)
    _check(_lib.ranc_read_outputs(h, _p(out)), h)
    return out


def ranc_read_outputs_device(h, dev_ptr):
    _check(_lib.ranc_read_outputs_device(h, C.c_void_p(int(dev_ptr))), h)


def ranc_read_state(h, batch, n_cores, neurons, want_v=True, want_spikes=True, want_digest=True):
    v = np.zeros((batch, n_cores, neurons), np.int32) if want_v else None
    s = np.zeros((batch, n_cores, neurons // 32), np.uint32) if want_spikes else None
    d = np.zeros(1, np.uint64)
    _check(_lib.ranc_read_state(h, _p(v) if want_v else None, _p(s) if want_spikes else None,
                                _p(d) if want_digest else None), h)
    return v, s, (int(d[0]) if want_digest else None)


def ranc_read_sample_state(h, b0, nb, n_cores, neurons):
    v = np.zeros((nb, n_cores, neurons), np.int32)
    s = np.zeros((nb, n_cores, neurons // 32), np.uint32)
    _check(_lib.ranc_read_sample_state(h, int(b0), int(nb), _p(v), _p(s)), h)
    return v, s


def ranc_read_sample_state_noalloc(h, b0, nb, n_cores, neurons):
    """Same result as ranc_read_sample_state, through the entry point that
    allocates no device memory (bounded sample range)."""
    v = np.zeros((nb, n_cores, neurons), np.int32)
    s = np.zeros((nb, n_cores, neurons // 32), np.uint32)
    _check(_lib.ranc_read_sample_state_noalloc(h, int(b0), int(nb), _p(v), _p(s)), h)
    return v, s


def ranc_read_counters(h):
    c = np.zeros(5, np.uint64)
    _check(_lib.ranc_read_counters(h, _p(c)), h)
    return c


def ranc_read_core_counters(h, c0, c1):
    c = np.zeros(4, np.uint64)
    _check(_lib.ranc_read_core_counters(h, int(c0), int(c1), _p(c)), h)
    return c


def ranc_get_tick(h):
    t = C.c_int64()
    _check(_lib.ranc_get_tick(h, C.byref(t)), h)
    return t.value


def ranc_reset(h):
    _check(_lib.ranc_reset(h), h)


def ranc_run_samples(h, inputs, n_samples, t_in, window, counts, mem=RANC_MEM_HOST):
    """Host mode: ``inputs`` uint32 [S, t_in, words] and ``counts`` uint32
    [S, n_outputs] numpy arrays.  Device mode: both are device pointers."""
    if mem == RANC_MEM_HOST:
        inputs = _c(inputs, np.uint32)
        assert counts.dtype == np.uint32 and counts.flags.c_contiguous
        ip, cp = _p(inputs), _p(counts)
    else:
        ip, cp = C.c_void_p(int(inputs)), C.c_void_p(int(counts))
    _check(_lib.ranc_run_samples(h, ip, int(n_samples), int(t_in), int(window), cp, int(mem)), h)


def ranc_run_stream(h, inputs, n_in, n_ticks, out_ticks, mem=RANC_MEM_HOST):
    """Host mode: ``inputs`` uint32 [B, n_in, words] and ``out_ticks`` uint32
    [B, n_ticks, n_outputs] numpy arrays.  Device mode: both are device pointers."""
    if mem == RANC_MEM_HOST:
        inputs = _c(inputs, np.uint32) if inputs is not None else None
        assert out_ticks.dtype == np.uint32 and out_ticks.flags.c_contiguous
        ip, op = (_p(inputs) if inputs is not None else None), _p(out_ticks)
    else:
        ip, op = C.c_void_p(int(inputs)), C.c_void_p(int(out_ticks))
    _check(_lib.ranc_run_stream(h, ip, int(n_in), int(n_ticks), op, int(mem)), h)


def ranc_save_state(h):
    n = C.c_size_t(0)
    _check(_lib.ranc_save_state(h, None, C.byref(n)), h)
    buf = np.zeros(n.value, np.uint8)
    _check(_lib.ranc_save_state(h, _p(buf), C.byref(n)), h)
    return buf


def ranc_load_state(h, buf):
    buf = _c(buf, np.uint8)
    _check(_lib.ranc_load_state(h, _p(buf), buf.size), h)


def ranc_set_kernel_timing(h, enable):
    _check(_lib.ranc_set_kernel_timing(h, 1 if enable else 0), h)


def ranc_read_kernel_timing(h):
    ms, n = C.c_double(), C.c_int64()
    _check(_lib.ranc_read_kernel_timing(h, C.byref(ms), C.byref(n)), h)
    return ms.value, n.value


def ranc_launch_count(h):
    n = C.c_int64()
    _check(_lib.ranc_launch_count(h, C.byref(n)), h)
    return n.value


def ranc_item_ticks(h):
    """(updated, deferred) item-ticks of the batched tick kernel."""
    u, d = C.c_int64(), C.c_int64()
    _check(_lib.ranc_item_ticks(h, C.byref(u), C.byref(d)), h)
    return u.value, d.value


def ranc_item_classes(h):
    """(active, idle, deferred) item-ticks of the batched tick kernel."""
    a, i, d = C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.ranc_item_classes(h, C.byref(a), C.byref(i), C.byref(d)), h)
    return a.value, i.value, d.value


def ranc_network_item_classes(h, k):
    """(active, idle) item-ticks of network k of a multi-network handle."""
    a, i = C.c_int64(), C.c_int64()
    _check(_lib.ranc_network_item_classes(h, int(k), C.byref(a), C.byref(i)), h)
    return a.value, i.value


def ranc_graph_stats(h):
    """(captures, replays) of ranc_run_samples' window graphs."""
    c, r = C.c_int64(), C.c_int64()
    _check(_lib.ranc_graph_stats(h, C.byref(c), C.byref(r)), h)
    return c.value, r.value


def ranc_potential_format(h):
    f = C.c_int32()
    _check(_lib.ranc_potential_format(h, C.byref(f)), h)
    return f.value


def ranc_desc_potential_format(net, path=RANC_PATH_BATCHED):
    """The potential storage ranc_create would choose for ``net`` on ``path``
    (no handle, no device work)."""
    d, keep = _desc(net)
    f = C.c_int32()
    _check(_lib.ranc_desc_potential_format(C.byref(d), int(path), C.byref(f)), None)
    return f.value


def ranc_device_allocations():
    """Device allocations the library has made in this process."""
    n = C.c_int64()
    _check(_lib.ranc_device_allocations(C.byref(n)), None)
    return n.value


def ranc_destroy(h):
    _lib.ranc_destroy(h)


def ranc_last_error(h=None):
    return _lib.ranc_last_error(h).decode()


class Sim:
    """Owning wrapper around one handle (same calls, shapes filled in)."""

    def __init__(self, net, batch, path=RANC_PATH_PLAIN, stream=0):
        self.net, self.batch, self.path = net, int(batch), path
        self.h = ranc_create(net, batch, path, stream)

    def load_inputs(self, bits):
        ranc_load_inputs(self.h, bits)

    def step(self, n_ticks):
        ranc_step(self.h, n_ticks)

    def outputs(self):
        return ranc_read_outputs(self.h, self.batch, self.net.n_outputs)

    def state(self, **kw):
        return ranc_read_state(self.h, self.batch, self.net.n_cores, self.net.neurons, **kw)

    def sample_state(self, b0, nb):
        return ranc_read_sample_state(self.h, b0, nb, self.net.n_cores, self.net.neurons)

    def counters(self):
        return ranc_read_counters(self.h)

    def core_counters(self, c0, c1):
        """Spikes, packets, outputs, synaptic events of cores [c0, c1)."""
        return ranc_read_core_counters(self.h, c0, c1)

    def tick(self):
        return ranc_get_tick(self.h)

    def reset(self):
        ranc_reset(self.h)

    def run_samples(self, inputs, window):
        inputs = _c(inputs, np.uint32)
        counts = np.zeros((inputs.shape[0], self.net.n_outputs), np.uint32)
        ranc_run_samples(self.h, inputs, inputs.shape[0], inputs.shape[1], window, counts)
        return counts

    def run_stream(self, inputs, n_ticks):
        """inputs [B, n_in, words] -> per-tick output-bus counts [B, n_ticks, n_outputs]."""
        inputs = _c(inputs, np.uint32)
        out = np.zeros((self.batch, n_ticks, self.net.n_outputs), np.uint32)
        ranc_run_stream(self.h, inputs, inputs.shape[1], n_ticks, out)
        return out

    def potential_format(self):
        """RANC_POTENTIAL_INT32, _INT16 or _FP16: how the potentials are stored."""
        return ranc_potential_format(self.h)

    def save(self):
        return ranc_save_state(self.h)

    def load(self, buf):
        ranc_load_state(self.h, buf)

    def close(self):
        if self.h is not None:
            ranc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiSim:
    """Owning wrapper around a multi-network handle (ranc_create_multi): the
    networks share the batch and the input lines; results are returned per
    network."""

    def __init__(self, nets, batch, stream=0):
        self.nets, self.batch = list(nets), int(batch)
        self.h = ranc_create_multi(self.nets, batch, stream)
        self.n_outputs = sum(n.n_outputs for n in self.nets)
        self.ooff = np.concatenate([[0], np.cumsum([n.n_outputs for n in self.nets])]).astype(int)
        self.coff = np.concatenate([[0], np.cumsum([n.n_cores for n in self.nets])]).astype(int)
        self.poff = np.concatenate([[0], np.cumsum([n.n_cores * n.neurons for n in self.nets])]).astype(int)
        self.n_inputs = max(n.n_inputs for n in self.nets)

    def split_outputs(self, counts):
        """[S, sum of n_outputs] -> list of [S, n_outputs_k]."""
        return [counts[:, self.ooff[k]:self.ooff[k + 1]] for k in range(len(self.nets))]

    def load_inputs(self, bits):
        ranc_load_inputs(self.h, bits)

    def step(self, n_ticks):
        ranc_step(self.h, n_ticks)

    def outputs(self):
        return self.split_outputs(ranc_read_outputs(self.h, self.batch, self.n_outputs))

    def run_samples(self, inputs, window):
        """inputs uint32 [S, t_in, words] (words for the widest input count) ->
        list of per-network counts [S, n_outputs_k]."""
        inputs = _c(inputs, np.uint32)
        counts = np.zeros((inputs.shape[0], self.n_outputs), np.uint32)
        ranc_run_samples(self.h, inputs, inputs.shape[0], inputs.shape[1], window, counts)
        return self.split_outputs(counts)

    def sample_state(self, b0, nb):
        """Per network: (v [nb, C_k, N_k], spikes [nb, C_k, N_k / 32])."""
        P = int(self.poff[-1])
        v = np.zeros((nb, P), np.int32)
        s = np.zeros((nb, P // 32), np.uint32)
        _check(_lib.ranc_read_sample_state(self.h, int(b0), int(nb), _p(v), _p(s)), self.h)
        res = []
        for k, n in enumerate(self.nets):
            a, b = self.poff[k], self.poff[k + 1]
            res.append((v[:, a:b].reshape(nb, n.n_cores, n.neurons),
                        s[:, a // 32:b // 32].reshape(nb, n.n_cores, n.neurons // 32)))
        return res

    def counters(self):
        """[n_networks, 4] spikes, packets, output events, synaptic events."""
        return np.stack([ranc_read_core_counters(self.h, self.coff[k], self.coff[k + 1]) for k in range(len(self.nets))])

    def reset(self):
        ranc_reset(self.h)

    def potential_format(self):
        return ranc_potential_format(self.h)

    def tuning(self):
        return ranc_get_multi_tuning(self.h)

    def item_classes(self):
        """[n_networks, 2] active and idle item-ticks of each network."""
        return np.array([ranc_network_item_classes(self.h, k) for k in range(len(self.nets))], np.int64)

    def set_tuning(self, weight_stages, cost_item, cost_mma, cost_slice):
        ranc_set_multi_tuning(self.h, weight_stages, cost_item, cost_mma, cost_slice)

    def close(self):
        if self.h is not None:
            ranc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _xcheck(rc, h):
    if rc != RANC_OK:
        raise RancError(rc, _lib.ranc_xbar_last_error(h).decode())


class Xbar:
    """Crossbar products dV [B][C][N] of ``net``'s cores in one of the exact
    tensor-core formulations (RANC_XBAR_*; include/ranc_xbar.h)."""

    def __init__(self, net, form, stream=0):
        self.net, self.form = net, int(form)
        d, keep = _desc(net)
        h = C.c_void_p()
        _xcheck(_lib.ranc_xbar_create(C.byref(d), self.form, C.c_void_p(int(stream)), C.byref(h)), None)
        self.h = h

    def run(self, spikes_dev, batch, dv_dev=0, sums_dev=0):
        """Device pointers: spikes [batch][A/32] uint32, dv [batch][C][N] int32
        (0: not written), sums [batch][C] int64 (0: not written)."""
        _xcheck(_lib.ranc_xbar_run(self.h, C.c_void_p(int(spikes_dev)), int(batch), C.c_void_p(int(dv_dev) or None),
                                   C.c_void_p(int(sums_dev) or None)), self.h)

    def sync(self):
        _xcheck(_lib.ranc_xbar_sync(self.h), self.h)

    def close(self):
        if self.h is not None:
            _lib.ranc_xbar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
