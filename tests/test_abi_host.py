"""CPU-only checks of the C ABI: the library loads, exports every entry point
that include/ranc.h declares, the binding's struct layouts match the C
compiler's, and ranc_create's host-side validation rejects bad descriptions
(validation runs before any CUDA call, so no GPU is needed)."""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import ranc_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ranc.h")


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ranc_[a-z_0-9]+)\s*\(", text)))


def test_surrogate_header_is_exported(ranc):
    mlp_header = os.path.join(ROOT, "include", "ranc_mlp.h")
    lib = C.CDLL(ranc.LIB_PATH)
    names = declared_functions(mlp_header)
    assert names and all(hasattr(lib, n) for n in names)
    from paper_2404_16208_gb300 import mlp
    assert sorted(mlp.EXPORTED) == names


def test_crossbar_header_is_exported(ranc):
    xbar_header = os.path.join(ROOT, "include", "ranc_xbar.h")
    lib = C.CDLL(ranc.LIB_PATH)
    names = declared_functions(xbar_header)
    assert names and all(hasattr(lib, n) for n in names)
    assert sorted(ranc.XBAR_EXPORTED) == names


def test_every_header_is_checked():
    """Each header under include/ is covered by one of the export tests."""
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["ranc.h", "ranc_mlp.h", "ranc_xbar.h"]


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ranc_create", "ranc_load_inputs", "ranc_step", "ranc_read_outputs", "ranc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(ranc):
    lib = C.CDLL(ranc.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(ranc.EXPORTED) == declared_functions()


def test_debug_library_exports_the_same_symbols(ranc):
    """The range-checked debug build carries the whole ABI of all three headers."""
    from paper_2404_16208_gb300 import build as B
    lib = C.CDLL(B.build(debug=True))
    for header in ("ranc.h", "ranc_xbar.h", "ranc_mlp.h"):
        for name in declared_functions(os.path.join(ROOT, "include", header)):
            assert hasattr(lib, name), (header, name)


def header_constants():
    """Every integer constant of the headers: #define NAME value and enum members."""
    out = {}
    for h in ("ranc.h", "ranc_xbar.h", "ranc_mlp.h"):
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
        for name, val in re.findall(r"#define\s+(RANC_\w+)\s+\(?(-?\d+)\)?", text):
            out[name] = int(val)
        for body in re.findall(r"enum\s*\{([^}]*)\}", text):
            for name, val in re.findall(r"(RANC_\w+)\s*=\s*(-?\d+)", body):
                out[name] = int(val)
    return out


def test_binding_constants_match_the_headers(ranc):
    """The binding's and the workload generator's copies of the header constants
    (return codes, paths, buffer kinds, potential formats, crossbar forms,
    destination kinds, negative-threshold modes, counter count) are the C values."""
    consts = header_constants()
    for name in ("RANC_OK", "RANC_EINVAL", "RANC_ENOMEM", "RANC_ECUDA", "RANC_ETIMEOUT", "RANC_ESTATE",
                 "RANC_PATH_PLAIN", "RANC_PATH_BATCHED", "RANC_MEM_HOST", "RANC_MEM_DEVICE",
                 "RANC_POTENTIAL_INT32", "RANC_POTENTIAL_INT16", "RANC_POTENTIAL_FP16",
                 "RANC_XBAR_F16_FOLDED", "RANC_XBAR_F8_PER_TYPE", "RANC_XBAR_I8_MMA_SYNC"):
        assert getattr(ranc, name) == consts[name], name
    from ranc_workloads import nets as NT
    assert (NT.KIND_NONE, NT.KIND_CORE, NT.KIND_OUTPUT) == (consts["RANC_DEST_NONE"], consts["RANC_DEST_CORE"],
                                                             consts["RANC_DEST_OUTPUT"])
    assert (NT.NEG_SATURATE, NT.NEG_RESET) == (consts["RANC_NEG_SATURATE"], consts["RANC_NEG_RESET"])
    assert len(ranc.COUNTER_NAMES) == consts["RANC_N_COUNTERS"]
    assert consts["RANC_ROWS"] == 16


def test_struct_layout_matches_c(tmp_path, ranc):
    exe = tmp_path / "abi_probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_probe.c"),
                    "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(got["sizeof_dest"]) == C.sizeof(ranc.ranc_dest) == W.DEST_DTYPE.itemsize == 8
    assert int(got["sizeof_desc"]) == C.sizeof(ranc.ranc_desc)
    assert int(got["dest.delay"]) == ranc.ranc_dest.delay.offset
    for f, _ in ranc.ranc_desc._fields_:
        if f in got:
            assert int(got[f]) == getattr(ranc.ranc_desc, f).offset, f


def _expect_einval(ranc, net, batch=1, path=0, frag=""):
    with pytest.raises(ranc.RancError) as ei:
        ranc.ranc_create(net, batch, path)
    assert ei.value.code == ranc.RANC_EINVAL, str(ei.value)
    assert frag in str(ei.value)


def small_net(**kw):
    return W.random_net(5, 2, 1, axons=32, neurons=32, **kw)


def test_rejects_delay_zero_and_sixteen(ranc):
    for d in (0, 16):
        net = small_net()
        i = np.flatnonzero(net.dest["kind"].ravel() == W.KIND_CORE)[0]
        net.dest.ravel()[i]["delay"] = d
        _expect_einval(ranc, net, frag="delay")


def test_rejects_axon_out_of_range(ranc):
    net = small_net()
    i = np.flatnonzero(net.dest["kind"].ravel() == W.KIND_CORE)[0]
    net.dest.ravel()[i]["axon"] = 32
    _expect_einval(ranc, net, frag="axon")


def test_rejects_destination_that_is_not_a_core(ranc):
    net = W.random_net(6, 2, 2, axons=32, neurons=32, holes=((1, 1),))
    i = np.flatnonzero(net.dest["kind"].ravel() == W.KIND_CORE)[0]
    c = i // 32
    x, y = net.core_xy[c]
    net.dest.ravel()[i]["dx"] = 1 - x
    net.dest.ravel()[i]["dy"] = 1 - y
    _expect_einval(ranc, net, frag="not a core")


def test_rejects_output_id_and_weight_range_and_shapes(ranc):
    net = small_net(p_out=0.5)
    i = np.flatnonzero(net.dest["kind"].ravel() == W.KIND_OUTPUT)[0]
    net.dest.ravel()[i]["axon"] = net.n_outputs
    _expect_einval(ranc, net, frag="output id")
    net = small_net()
    net.weight[0, 0, 0] = 8  # weight_bits 4 allows +-7
    _expect_einval(ranc, net, frag="weight")
    _expect_einval(ranc, small_net(), batch=0, frag="batch")
    _expect_einval(ranc, small_net(), path=7, frag="path")
    net = small_net()
    net.axon_type[0, 0] = net.n_types
    _expect_einval(ranc, net, frag="axon_type")


def test_rejects_possible_int32_overflow(ranc):
    net = small_net()
    net.pos_thr[0, 0] = 2**31 - 1
    _expect_einval(ranc, net, frag="int32")


def test_rejects_shared_grid_cell(ranc):
    net = small_net()
    net.core_xy[1] = net.core_xy[0]
    _expect_einval(ranc, net, frag="share")


def test_create_error_message_is_kept(ranc):
    net = small_net()
    net.axon_type[0, 0] = 99
    with pytest.raises(ranc.RancError):
        ranc.ranc_create(net, 1)
    assert "axon_type" in ranc.ranc_last_error(None)
