"""Window graphs of ranc_run_samples (batched path, device buffers).

The first call records the launch sequence as a CUDA graph and later calls
with the same arguments replay it; every replay must give the oracle's output
counts bit for bit, whatever the handle did in between (the state-dependent
reset runs before the graph)."""

import os

import numpy as np
import pytest

import ranc_workloads as W

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _net(neurons):
    # delays up to 15 leave deliveries in rows that a later group's reset must clear
    return W.random_net(31 + neurons, 2, 2, axons=128, neurons=neurons, n_types=4, neg_mode=0, delay_max=15,
                        v0=(-3, 3), n_inputs=90, fanout_per_line=4, p_core=0.6, p_out=0.2, w_lim=100,
                        weight_bits=8, pthr=(1, 300), nthr=(-300, -1), leak=(-2, 2))


@pytest.mark.parametrize("neurons", [128, 256])
def test_window_graph_replays_match_the_oracle(ranc, torch, oracle_mod, neurons):
    net = _net(neurons)
    S, t_in, window = 300, 10, 18   # three groups of a 128-sample handle, the last one ragged
    x = W.rate_coded_inputs(5, S, t_in, net.n_inputs, 0.3)
    ref = oracle_mod.run(net, x, window, n_threads=NPROC)
    assert ref["counters"][:, 1].sum() > 0 and ref["out"].sum() > 0
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((S, net.n_outputs), dtype=torch.int32, device="cuda")
    launches = []
    for k in range(3):
        dout.zero_()
        l0 = ranc.ranc_launch_count(sim.h)
        ranc.ranc_run_samples(sim.h, dx.data_ptr(), S, t_in, window, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
        launches.append(ranc.ranc_launch_count(sim.h) - l0)
        np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref["out"], err_msg=f"call {k}")
    assert ranc.ranc_graph_stats(sim.h) == (1, 2)
    assert launches[0] == launches[1] == launches[2] > 0
    # counters accumulate over the three calls
    np.testing.assert_array_equal(sim.counters()[:4], 3 * ref["counters"][:, :4].sum(0))
    sim.close()


def test_window_graph_after_other_use_and_new_arguments(ranc, torch, oracle_mod):
    net = _net(256)
    S, t_in, window = 200, 10, 18
    x = W.rate_coded_inputs(6, S, t_in, net.n_inputs, 0.3)
    y = W.rate_coded_inputs(7, 128, t_in, net.n_inputs, 0.4)
    ref = oracle_mod.run(net, x, window, n_threads=NPROC)
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((S, net.n_outputs), dtype=torch.int32, device="cuda")
    run = lambda w: ranc.ranc_run_samples(sim.h, dx.data_ptr(), S, t_in, w, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
    run(window)
    np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref["out"])
    # other work on the handle in between: a host-mode window and a partial run that
    # leaves deliveries in flight in the scheduler rows
    np.testing.assert_array_equal(sim.run_samples(y, window), oracle_mod.run(net, y, window, n_threads=NPROC)["out"])
    sim.reset()
    sim.load_inputs(y)
    sim.step(5)
    dout.zero_()
    run(window)
    np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref["out"])
    assert ranc.ranc_graph_stats(sim.h) == (1, 1)
    # new arguments: a new recording, then replays of it
    ref2 = oracle_mod.run(net, x, window + 3, n_threads=NPROC)
    for _ in range(2):
        dout.zero_()
        run(window + 3)
        np.testing.assert_array_equal(dout.cpu().numpy().view(np.uint32), ref2["out"])
    assert ranc.ranc_graph_stats(sim.h) == (2, 2)
    # the state after a replayed window is readable and equals the oracle's
    v, _, _ = sim.state(want_spikes=False, want_digest=False)
    last = slice(128, S)  # the last group of 72 samples is what the handle holds
    ref_last = oracle_mod.run(net, x[last], window + 3, n_threads=NPROC)
    np.testing.assert_array_equal(v[:S - 128], ref_last["v"])
    sim.close()
