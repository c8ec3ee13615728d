"""CPU oracle of the RANC tick semantics (test infrastructure only).

Only the tests, ``__graft_entry__`` (build and smoke check) and the
benchmark's CPU-baseline leg may import this package.  The product library
never reaches it, and it never reaches the product library.

:func:`build` compiles ``ranc_oracle.c`` with gcc into ``oracle/_build``;
:func:`run` marshals a :class:`ranc_workloads.Net` into the C structure and
calls ``oracle_run``.
"""

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ranc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libranc_oracle.so")
_lib = None

COUNTER_NAMES = ("spikes", "packets", "outputs", "synaptic_events", "ticks")


def build(force=False):
    """Compile the oracle (OpenMP when the compiler has it)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Net(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("grid_w", "grid_h", "n_cores", "axons", "neurons", "n_types",
                                          "neg_mode")] + [
        ("core_xy", C.c_void_p), ("crossbar", C.c_void_p), ("axon_type", C.c_void_p), ("weight", C.c_void_p),
        ("leak", C.c_void_p), ("pos_thr", C.c_void_p), ("neg_thr", C.c_void_p), ("reset", C.c_void_p),
        ("v0", C.c_void_p), ("dest_dx", C.c_void_p), ("dest_dy", C.c_void_p), ("dest_axon", C.c_void_p),
        ("dest_delay", C.c_void_p), ("dest_kind", C.c_void_p), ("n_inputs", C.c_int32),
        ("n_outputs", C.c_int32), ("in_offsets", C.c_void_p), ("in_core", C.c_void_p),
        ("in_axon", C.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_run.restype = C.c_int
        _lib.oracle_run.argtypes = [C.POINTER(_Net), C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int32, C.c_char_p, C.c_int32]
        _lib.oracle_max_threads.restype = C.c_int
    return _lib


def max_threads():
    return int(_load().oracle_max_threads())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def run(net, inputs, n_ticks, trace=False, n_threads=1, out_trace=False):
    """Simulate every sample of ``inputs`` ([S, T_in, words] uint32) for
    ``n_ticks`` ticks from the initial state.

    Returns a dict with ``v`` [S, C, N] int32 (after the last tick),
    ``out`` [S, n_outputs] uint32, ``counters`` [S, 5] uint64; when
    ``trace``, ``v_trace`` [S, n_ticks, C, N] int32 and ``spike_trace``
    [S, n_ticks, C, N] uint8; when ``out_trace``, ``out_trace``
    [S, n_ticks, n_outputs] uint32 (output-bus events of every tick).
    """
    lib = _load()
    inputs = np.ascontiguousarray(inputs, dtype=np.uint32)
    S, t_in = int(inputs.shape[0]), int(inputs.shape[1])
    Cn, N = net.n_cores, net.neurons
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return _ptr(a)

    d = net.dest
    s = _Net(net.grid_w, net.grid_h, Cn, net.axons, N, net.n_types, net.neg_mode,
             arr(net.core_xy, np.int16), arr(net.crossbar, np.uint32), arr(net.axon_type, np.uint8),
             arr(net.weight, np.int16), arr(net.leak, np.int32), arr(net.pos_thr, np.int32),
             arr(net.neg_thr, np.int32), arr(net.reset, np.int32), arr(net.v0, np.int32),
             arr(d["dx"], np.int16), arr(d["dy"], np.int16), arr(d["axon"], np.uint16),
             arr(d["delay"], np.uint8), arr(d["kind"], np.uint8), net.n_inputs, net.n_outputs,
             arr(net.in_offsets, np.int32), arr(net.in_core, np.int32), arr(net.in_axon, np.int32))
    v = np.zeros((S, Cn, N), dtype=np.int32)
    out = np.zeros((S, net.n_outputs), dtype=np.uint32)
    cnt = np.zeros((S, 5), dtype=np.uint64)
    vt = np.zeros((S, n_ticks, Cn, N), dtype=np.int32) if trace else None
    st = np.zeros((S, n_ticks, Cn, N), dtype=np.uint8) if trace else None
    ot = np.zeros((S, n_ticks, net.n_outputs), dtype=np.uint32) if out_trace else None
    err = C.create_string_buffer(512)
    rc = lib.oracle_run(C.byref(s), S, _ptr(inputs), t_in, int(n_ticks), _ptr(v), _ptr(out), _ptr(cnt),
                        _ptr(vt), _ptr(st), _ptr(ot), int(n_threads), err, 512)
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc}): {err.value.decode()}")
    res = dict(v=v, out=out, counters=cnt)
    if trace:
        res.update(v_trace=vt, spike_trace=st)
    if out_trace:
        res.update(out_trace=ot)
    return res
