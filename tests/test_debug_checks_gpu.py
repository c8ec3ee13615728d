"""Device-side range checks (the debug build, ``libranc_debug.so``).

With ``-DRANC_DEBUG`` every index a tick kernel derives from the network
description is checked before its global access: the input line of a fan-in
entry, the axon of an input entry, the destination core and axon of a spike
packet, the output id of an output-bus event.  A failed check skips the access
and the next synchronising call returns RANC_ECUDA naming the site.

* Every tick kernel (plain per-tick, plain persistent steps, plain persistent
  windows, batched tensor-core, multi-network) runs a parity case under the
  checks: no check fails and the results equal the oracle's.
* RANC_DEBUG_PLANT=<site> (read at create, debug builds only) makes every
  check of one site fail on purpose, with no invalid access made: the failure
  must be reported with its site, later calls must return RANC_ESTATE, and
  ranc_reset must bring the handle back to correct results.
"""

import gc

import numpy as np
import pytest

import ranc_workloads as W

pytestmark = pytest.mark.gpu

SITE_INPUT_LINE, SITE_INPUT_AXON, SITE_DEST_CORE, SITE_DEST_AXON, SITE_OUTPUT_ID = 1, 2, 3, 4, 5


@pytest.fixture(scope="module")
def dranc():
    """The binding with the debug library swapped in for this module."""
    from paper_2404_16208_gb300 import build as B
    from paper_2404_16208_gb300 import ranc as mod
    path = B.build(debug=True)
    gc.collect()  # handles of earlier modules are destroyed by the library that made them
    prev = mod.use_library(path)
    try:
        yield mod
    finally:
        gc.collect()
        mod._lib = prev


def recurrent_net(seed):
    # Delays up to 15, holes in the grid, output-bus neurons and input lines on
    # several cores: every checked site is exercised.
    return W.random_net(seed, 3, 2, axons=64, neurons=96, n_types=3, neg_mode=1, delay_max=15, holes=((1, 1),),
                        v0=(-3, 3), n_inputs=70, fanout_per_line=3, p_core=0.6, p_out=0.2)


def test_plain_tick_and_steps_kernels_under_checks(dranc, oracle_mod):
    net = recurrent_net(211)
    B, T = 5, 20
    x = W.rate_coded_inputs(7, B, 12, net.n_inputs, 0.35)
    ref = oracle_mod.run(net, x, T)
    for per_tick in (True, False):
        sim = dranc.Sim(net, B, dranc.RANC_PATH_PLAIN)
        sim.load_inputs(x)
        if per_tick:
            for _ in range(T):
                sim.step(1)
        else:
            l0 = dranc.ranc_launch_count(sim.h)
            sim.step(T)
            assert dranc.ranc_launch_count(sim.h) - l0 == 1, "one persistent launch"
        np.testing.assert_array_equal(sim.outputs(), ref["out"])
        np.testing.assert_array_equal(sim.state()[0], ref["v"])
        np.testing.assert_array_equal(sim.counters()[:4], ref["counters"][:, :4].sum(0))
        sim.close()
    assert ref["counters"][:, 1].sum() > 0 and ref["counters"][:, 2].sum() > 0  # packets and output events


def test_plain_window_kernel_under_checks(dranc, oracle_mod):
    net = W.tiny_5core()
    S, t_in, window = 12, net.meta["t_in"], net.meta["window"]
    x = W.rate_coded_inputs(net.meta["seed"], S, t_in, net.n_inputs, net.meta["p_in"])
    ref = oracle_mod.run(net, x, window)
    sim = dranc.Sim(net, 1, dranc.RANC_PATH_PLAIN)
    l0 = dranc.ranc_launch_count(sim.h)
    np.testing.assert_array_equal(sim.run_samples(x, window), ref["out"])
    assert dranc.ranc_launch_count(sim.h) - l0 <= 3  # the persistent window kernel, not per-tick launches
    np.testing.assert_array_equal(sim.counters()[:4], ref["counters"][:, :4].sum(0))
    sim.close()


def test_batched_kernel_under_checks(dranc, oracle_mod):
    net = W.random_net(305, 3, 3, axons=128, neurons=256, n_types=4, neg_mode=0, delay_max=9, v0=(-3, 3),
                       n_inputs=90, fanout_per_line=4, p_core=0.6, p_out=0.2)
    B, T = 200, 14  # two sample tiles, the second ragged
    x = W.rate_coded_inputs(11, B, 10, net.n_inputs, 0.3)
    ref = oracle_mod.run(net, x, T)
    sim = dranc.Sim(net, B, dranc.RANC_PATH_BATCHED)
    sim.load_inputs(x)
    sim.step(T)
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    sim.close()
    assert ref["counters"][:, 1].sum() > 0 and ref["counters"][:, 2].sum() > 0


def test_multi_network_kernel_under_checks(dranc, oracle_mod):
    mix = [((2, 2), 64, 128, 2, 40), ((2, 1), 512, 128, 4, 64), ((1, 2), 256, 512, 2, 33)]
    nets = [W.random_net(400 + 31 * k, gw, gh, axons=A, neurons=N, n_types=K, neg_mode=0, delay_max=1 + 5 * k,
                         v0=(-3, 3), n_inputs=n_in, fanout_per_line=6, p_core=0.6, p_out=0.2, w_lim=60,
                         weight_bits=8, pthr=(1, 180), nthr=(-180, -1), leak=(-3, 2), density=0.2)
            for k, ((gw, gh), A, N, K, n_in) in enumerate(mix)]
    B, T = 150, 12
    x = W.rate_coded_inputs(13, B, 8, max(n.n_inputs for n in nets), 0.3)
    sim = dranc.MultiSim(nets, B)
    sim.load_inputs(x)
    sim.step(T)
    outs = sim.outputs()
    sim.close()
    for k, n in enumerate(nets):
        ref = oracle_mod.run(n, x[..., :(n.n_inputs + 31) // 32], T)
        np.testing.assert_array_equal(outs[k], ref["out"], err_msg=f"network {k}")


@pytest.mark.parametrize("site,path", [(SITE_INPUT_LINE, 0), (SITE_DEST_CORE, 0), (SITE_OUTPUT_ID, 0),
                                       (SITE_INPUT_LINE, 1), (SITE_DEST_AXON, 1), (SITE_OUTPUT_ID, 1)],
                         ids=["plain-input-line", "plain-dest-core", "plain-output-id",
                              "batched-input-line", "batched-dest-axon", "batched-output-id"])
def test_planted_check_failure_is_reported_and_reset_recovers(dranc, oracle_mod, monkeypatch, site, path):
    net = W.tiny_5core()
    B, T = 4, net.meta["window"]
    x = W.rate_coded_inputs(net.meta["seed"], B, net.meta["t_in"], net.n_inputs, net.meta["p_in"])
    monkeypatch.setenv("RANC_DEBUG_PLANT", str(site))
    sim = dranc.Sim(net, B, path)
    monkeypatch.delenv("RANC_DEBUG_PLANT")
    sim.load_inputs(x)
    sim.step(T)  # inputs, packets and output events all occur in this window
    with pytest.raises(dranc.RancError) as ei:
        sim.outputs()
    assert ei.value.code == dranc.RANC_ECUDA
    assert f"site {site}" in str(ei.value)
    with pytest.raises(dranc.RancError) as ei:
        sim.step(1)
    assert ei.value.code == dranc.RANC_ESTATE
    sim.reset()
    sim.load_inputs(x)
    sim.step(T)
    ref = oracle_mod.run(net, x, T)
    assert ref["counters"][:, 1].sum() > 0 and ref["counters"][:, 2].sum() > 0  # every planted site is reached
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    sim.close()
