"""The paper's largest scaling case (Table I, Sec. IV): a 64 x 64 grid of
256 x 256 cores with no application mapped, 500 ticks, no spike ever
generated.  Pinned by the closed form of the zero-spike case: with no input,
non-positive leak and positive thresholds, V_t = max(neg_thr, v0 + t * leak)
and every counter but the synaptic one stays zero."""

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
def net():
    return W.truenorth_ref()


def closed_form(net, t):
    return np.maximum(net.neg_thr.astype(np.int64), net.v0 + t * net.leak.astype(np.int64))


def test_truenorth_ref_plain_500_ticks(ranc, oracle_mod, net):
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    sim.step(3)
    ref = oracle_mod.run(net, np.zeros((1, 0, 0), np.uint32), 3, n_threads=NPROC)
    np.testing.assert_array_equal(sim.state(want_spikes=False, want_digest=False)[0], ref["v"])
    l0 = ranc.ranc_launch_count(sim.h)
    sim.step(497)
    assert ranc.ranc_launch_count(sim.h) - l0 == 1  # one persistent launch for the 497 ticks
    v, s, _ = sim.state(want_digest=False)
    np.testing.assert_array_equal(v[0], closed_form(net, 500))
    assert not s.any()
    cnt = sim.counters()
    assert cnt[:4].tolist() == [0, 0, 0, 0] and cnt[4] == 500
    sim.close()


def test_truenorth_ref_batched_one_tile(ranc, net):
    sim = ranc.Sim(net, 128, ranc.RANC_PATH_BATCHED)
    sim.step(100)
    for b in (0, 77, 127):
        v, s = sim.sample_state(b, 1)
        np.testing.assert_array_equal(v[0], closed_form(net, 100))
        assert not s.any()
    assert sim.counters()[:4].tolist() == [0, 0, 0, 0]
    sim.close()
