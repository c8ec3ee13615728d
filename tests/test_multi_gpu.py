"""Multi-network handles (ranc_create_multi) against the CPU oracle, bit for bit.

Several networks of different core shapes run in one batched handle, one tick
launch for all of them.  Each network is simulated alone by the oracle on the
same samples (its own input lines are the first lines of the shared inputs);
the handle must reproduce every network's potentials, spikes, output counts
and counters, in every potential format and both negative-threshold modes,
through per-tick steps, window graphs and the tuning knobs.  The last test is
the design sweep at full size: 64 ragged configurations of up to 1024 cores of
up to 512 x 512, 1024 samples, one launch per tick, a seeded sample of every
configuration compared with the oracle."""

import concurrent.futures as cf
import os

import numpy as np
import pytest

import ranc_workloads as W
from parity_util import digest, unpack_spikes

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def words(net):
    return (net.n_inputs + 31) // 32


# (grid, axons, neurons, types, n_inputs) of the networks of one handle
MIX = [((2, 2), 64, 128, 2, 40), ((3, 1), 128, 256, 4, 90), ((1, 2), 192, 384, 3, 70),
       ((2, 1), 512, 128, 4, 64), ((2, 2), 256, 512, 2, 33), ((1, 1), 512, 512, 4, 96)]
# weight limit / bits and thresholds per potential format
FORMATS = {"fp16": (60, 8, (1, 180), (-180, -1)), "int16": (900, 11, (1000, 3000), (-3000, -1)),
           "int32": (2047, 12, (30000, 60000), (-60000, -30000))}


def mix_nets(seed, neg_mode, fmt, mix=MIX):
    wl, wb, pthr, nthr = FORMATS[fmt]
    nets = []
    for k, ((gw, gh), A, N, K, n_in) in enumerate(mix):
        nets.append(W.random_net(seed + 31 * k, gw, gh, axons=A, neurons=N, n_types=K, neg_mode=neg_mode,
                                 delay_max=1 + (5 * k) % 15, v0=(-3, 3), n_inputs=n_in, fanout_per_line=6,
                                 p_core=0.6, p_out=0.2, w_lim=wl, weight_bits=wb, pthr=pthr, nthr=nthr,
                                 leak=(-3, 2), density=0.15 + 0.05 * k))
    return nets


def oracle_runs(oracle_mod, nets, x, n_ticks, **kw):
    """The oracle on every network alone (threads over networks)."""
    def one(n):
        return oracle_mod.run(n, x[..., :words(n)], n_ticks, n_threads=max(1, NPROC // len(nets)), **kw)
    with cf.ThreadPoolExecutor(len(nets)) as ex:
        return list(ex.map(one, nets))


FORMAT_CODE = {"fp16": 2, "int16": 1, "int32": 0}


@pytest.mark.parametrize("fmt,neg_mode", [("fp16", 0), ("fp16", 1), ("int16", 0), ("int32", 1)])
def test_mixed_shapes_every_tick(ranc, oracle_mod, fmt, neg_mode):
    nets = mix_nets(500 + 7 * neg_mode, neg_mode, fmt)
    B, T = 200, 16
    x = W.rate_coded_inputs(77, B, 10, max(n.n_inputs for n in nets), 0.3)
    refs = oracle_runs(oracle_mod, nets, x, T, trace=True)
    sim = ranc.MultiSim(nets, B)
    assert sim.potential_format() == FORMAT_CODE[fmt]
    sim.load_inputs(x)
    for t in range(T):
        sim.step(1)
        for k, ((v, s), ref) in enumerate(zip(sim.sample_state(0, B), refs)):
            np.testing.assert_array_equal(v, ref["v_trace"][:, t], err_msg=f"network {k} tick {t}")
            np.testing.assert_array_equal(unpack_spikes(s, nets[k].neurons), ref["spike_trace"][:, t],
                                          err_msg=f"network {k} tick {t}")
    for k, (o, ref) in enumerate(zip(sim.outputs(), refs)):
        np.testing.assert_array_equal(o, ref["out"], err_msg=f"network {k}")
    cnt = sim.counters()
    for k, ref in enumerate(refs):
        np.testing.assert_array_equal(cnt[k], ref["counters"][:, :4].sum(0), err_msg=f"network {k}")
    assert sum(int(r["counters"][:, 1].sum()) for r in refs) > 0  # packets flowed
    assert ranc.ranc_read_counters(sim.h)[4] == B * T
    upd, dfr = ranc.ranc_item_ticks(sim.h)
    assert upd == 2 * sum(n.n_cores for n in nets) * T and dfr == 0
    sim.close()


def test_window_graph_tuning_and_full_state_read(ranc, oracle_mod):
    """ranc_run_samples with device buffers (a recorded window graph and its
    replays) in groups of 128 samples, under every weight-stage count and
    two split cost settings; then ranc_read_state (all samples, digest)."""
    import torch
    nets = mix_nets(900, 0, "fp16")
    S, t_in, window = 300, 8, 14
    x = W.rate_coded_inputs(78, S, t_in, max(n.n_inputs for n in nets), 0.3)
    refs = oracle_runs(oracle_mod, nets, x, window)
    sim = ranc.MultiSim(nets, 128)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((S, sim.n_outputs), dtype=torch.int32, device="cuda")
    st0, mx, ci0, cm0, cs0 = sim.tuning()
    assert 2 <= st0 <= mx and mx >= 4 and (ci0, cm0, cs0) == (4, 1, 3)
    settings = 0
    for stages in range(2, mx + 1):
        for ci, cm, cs in ((4, 1, 3), (0, 3, 1)):
            sim.set_tuning(stages, ci, cm, cs)  # the next call records the window graph again
            assert sim.tuning() == (stages, mx, ci, cm, cs)
            for call in range(2):
                dout.zero_()
                ranc.ranc_run_samples(sim.h, dx.data_ptr(), S, t_in, window, dout.data_ptr(), ranc.RANC_MEM_DEVICE)
                outs = sim.split_outputs(dout.cpu().numpy().view(np.uint32))
                for k, (o, ref) in enumerate(zip(outs, refs)):
                    np.testing.assert_array_equal(o, ref["out"],
                                                  err_msg=f"stages {stages}, costs {ci}/{cm}/{cs}, call {call}, network {k}")
            settings += 1
    assert ranc.ranc_graph_stats(sim.h) == (settings, settings)
    with pytest.raises(ranc.RancError):
        sim.set_tuning(mx + 1, 4, 1, 3)
    with pytest.raises(ranc.RancError):
        sim.set_tuning(2, -1, 1, 3)
    # the last group's state after the window, every sample of the batch, with the digest
    last = oracle_runs(oracle_mod, nets, x[256:], window, trace=False)
    P = int(sim.poff[-1])
    v = np.zeros((128, P), np.int32)
    d = np.zeros(1, np.uint64)
    assert ranc._lib.ranc_read_state(sim.h, ranc._p(v), None, ranc._p(d)) == 0
    for k, ref in enumerate(last):
        a, b = sim.poff[k], sim.poff[k + 1]
        np.testing.assert_array_equal(v[:S - 256, a:b].reshape(S - 256, nets[k].n_cores, -1), ref["v"])
    assert int(d[0]) == digest(v)
    sim.close()


def test_unsupported_calls_and_shape_checks(ranc):
    nets = mix_nets(950, 0, "fp16", mix=MIX[:2])
    sim = ranc.MultiSim(nets, 64)
    for call in (lambda: ranc.ranc_save_state(sim.h),
                 lambda: ranc.ranc_read_sample_state_noalloc(sim.h, 0, 1, 1, 128),
                 lambda: ranc.ranc_run_stream(sim.h, np.zeros((64, 1, 3), np.uint32), 1, 2,
                                              np.zeros((64, 2, sim.n_outputs), np.uint32))):
        with pytest.raises(ranc.RancError) as ei:
            call()
        assert ei.value.code == ranc.RANC_ESTATE
    sim.close()
    bad = W.random_net(951, 1, 1, axons=96, neurons=128)  # 96 axons: not a multiple of 64
    with pytest.raises(ranc.RancError) as ei:
        ranc.MultiSim([nets[0], bad], 64)
    assert ei.value.code == ranc.RANC_EINVAL and "network 1" in str(ei.value)
    other = W.random_net(952, 1, 1, axons=64, neurons=128, neg_mode=1)
    with pytest.raises(ranc.RancError):
        ranc.MultiSim([nets[0], other], 64)
    plain = ranc.Sim(nets[0], 1, ranc.RANC_PATH_PLAIN)
    with pytest.raises(ranc.RancError) as ei:
        ranc.ranc_set_multi_tuning(plain.h, 3, 4, 1, 3)
    assert ei.value.code == ranc.RANC_ESTATE
    plain.close()


SWEEP_SEED, SWEEP_CONFIGS, SWEEP_SAMPLES, SWEEP_T_IN, SWEEP_WINDOW = 0x5EEDF1, 64, 1024, 16, 32


def test_design_sweep_full_size_one_launch_per_tick(ranc, oracle_mod):
    """The design sweep as benchmarked: 64 configurations (core sizes
    {128, 256, 512}^2, weight bits {4, 6, 9}, 2 or 4 axon types, 64..1024
    cores, density 0.1..0.5, delays 1..15), 1024 shared samples, one handle,
    one window graph (one tick launch per tick for all 64).  One seeded sample
    of every configuration is compared with the oracle (all output counts),
    and every configuration's output counts agree with its output-event
    counter."""
    import torch
    from ranc_workloads import sweep as SW
    nets = SW.sweep(SWEEP_SEED, SWEEP_CONFIGS, core_range=(64, 1024))
    x = W.rate_coded_inputs(SWEEP_SEED, SWEEP_SAMPLES, SWEEP_T_IN, 1024, 0.15)
    sim = ranc.MultiSim(nets, SWEEP_SAMPLES)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    dout = torch.zeros((SWEEP_SAMPLES, sim.n_outputs), dtype=torch.int32, device="cuda")
    l0 = ranc.ranc_launch_count(sim.h)
    for _ in range(2):  # recording, replay
        ranc.ranc_run_samples(sim.h, dx.data_ptr(), SWEEP_SAMPLES, SWEEP_T_IN, SWEEP_WINDOW, dout.data_ptr(),
                              ranc.RANC_MEM_DEVICE)
    # per window: reset, input transposition, one tick kernel per tick (all 64 networks), no other kernels
    assert ranc.ranc_launch_count(sim.h) - l0 == 2 * (1 + SWEEP_WINDOW)
    outs = sim.split_outputs(dout.cpu().numpy().view(np.uint32))
    cnt = sim.counters()
    picks = [(k, (k * 2654435761 + 12345) % SWEEP_SAMPLES) for k in range(SWEEP_CONFIGS)]

    def one(kb):
        k, b = kb
        n = nets[k]
        return oracle_mod.run(n, x[b:b + 1, :, :words(n)], SWEEP_WINDOW, n_threads=1)["out"][0]
    with cf.ThreadPoolExecutor(NPROC) as ex:
        refs = list(ex.map(one, picks))
    for (k, b), ref in zip(picks, refs):
        np.testing.assert_array_equal(outs[k][b], ref, err_msg=f"configuration {k}, sample {b}")
    for k in range(SWEEP_CONFIGS):
        # the counters of the last window (the second call) equal its output counts
        assert int(outs[k].sum()) * 2 == int(cnt[k][2]), k
    assert sum(int(o.sum()) for o in outs) > 0
    sim.close()
