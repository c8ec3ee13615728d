"""Failure detection without any GPU fault.

* A test-only flag (RANC_TEST_STALL_WAIT, read at ranc_create) makes one wait
  of each kernel kind unable to complete: one CTA of the per-tick plain kernel
  waits on an mbarrier that nothing arrives on; one CTA of the persistent
  plain kernel does not arrive at the grid barrier, so every CTA's barrier
  wait runs out; one CTA of the batched tensor-core kernel waits for its
  weight copies on a barrier armed with a transaction count that no copy
  satisfies (the copies it issued still land before it exits).  The bounded
  waits must give up after their limit, the next synchronising call must
  return RANC_ETIMEOUT, later calls RANC_ESTATE, and ranc_reset must bring the
  handle back to correct results.
* RANC_FAULT_ALLOC_AFTER=n makes the (n+1)-th device allocation of a create
  fail: every such create must return RANC_ENOMEM and free what it took.
"""

import time

import numpy as np
import pytest

import ranc_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def test_bounded_wait_gives_up_and_reset_recovers(ranc, oracle_mod, monkeypatch):
    net = W.tiny_5core()
    monkeypatch.setenv("RANC_TEST_STALL_WAIT", "1")
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    monkeypatch.delenv("RANC_TEST_STALL_WAIT")
    t0 = time.time()
    sim.step(1)
    with pytest.raises(ranc.RancError) as ei:
        sim.outputs()
    assert ei.value.code == ranc.RANC_ETIMEOUT
    assert time.time() - t0 < 20
    with pytest.raises(ranc.RancError) as ei:
        sim.step(1)
    assert ei.value.code == ranc.RANC_ESTATE
    sim.reset()
    x = W.rate_coded_inputs(5, 2, 8, 784, 0.15)
    sim.load_inputs(x)
    sim.step(9)
    ref = oracle_mod.run(net, x, 9)
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    sim.close()


@pytest.mark.parametrize("path", [0, 1], ids=["plain", "batched"])
def test_allocation_failures_return_enomem_without_leaks(ranc, monkeypatch, path):
    import torch
    torch.cuda.init()
    net = W.tiny_5core()
    # A first create loads the library's device code and its static arrays,
    # which stay resident; the baseline is taken after that.
    ranc.ranc_destroy(ranc.ranc_create(net, 256, path))
    free0 = torch.cuda.mem_get_info()[0]
    succeeded_at = None
    for k in range(0, 64):
        monkeypatch.setenv("RANC_FAULT_ALLOC_AFTER", str(k))
        try:
            h = ranc.ranc_create(net, 256, path)
        except ranc.RancError as e:
            assert e.code == ranc.RANC_ENOMEM, str(e)
            assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20), k
            continue
        succeeded_at = k
        ranc.ranc_destroy(h)
        break
    monkeypatch.delenv("RANC_FAULT_ALLOC_AFTER")
    assert succeeded_at is not None and succeeded_at >= 10
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)


def test_persistent_grid_barrier_wait_gives_up_and_reset_recovers(ranc, oracle_mod, monkeypatch):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(6, 4, 8, 784, 0.15)
    monkeypatch.setenv("RANC_TEST_STALL_WAIT", "1")
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    monkeypatch.delenv("RANC_TEST_STALL_WAIT")
    t0 = time.time()
    with pytest.raises(ranc.RancError) as ei:  # the persistent window kernel (4 co-resident CTAs)
        sim.run_samples(x, 9)
    assert ei.value.code == ranc.RANC_ETIMEOUT
    assert time.time() - t0 < 20
    with pytest.raises(ranc.RancError) as ei:
        sim.run_samples(x, 9)
    assert ei.value.code == ranc.RANC_ESTATE
    sim.reset()
    ref = oracle_mod.run(net, x, 9)
    np.testing.assert_array_equal(sim.run_samples(x, 9), ref["out"])
    sim.close()


def test_persistent_steps_barrier_wait_gives_up_and_reset_recovers(ranc, oracle_mod, monkeypatch):
    """ranc_step(n >= 2) on the plain path (one cooperative launch): CTA 0
    skips its arrival at the first grid barrier, every CTA's bounded wait
    runs out, the call reports RANC_ETIMEOUT, the handle refuses work until
    ranc_reset, and then steps correctly."""
    net = W.tiny_5core()
    x = W.rate_coded_inputs(7, 2, 8, 784, 0.15)
    monkeypatch.setenv("RANC_TEST_STALL_WAIT", "1")
    sim = ranc.Sim(net, 2, ranc.RANC_PATH_PLAIN)
    monkeypatch.delenv("RANC_TEST_STALL_WAIT")
    sim.load_inputs(x)
    t0 = time.time()
    with pytest.raises(ranc.RancError) as ei:
        sim.step(5)
        sim.outputs()
    assert ei.value.code == ranc.RANC_ETIMEOUT
    assert time.time() - t0 < 20
    with pytest.raises(ranc.RancError) as ei:
        sim.step(5)
    assert ei.value.code == ranc.RANC_ESTATE
    sim.reset()
    sim.load_inputs(x)
    sim.step(9)
    np.testing.assert_array_equal(sim.outputs(), oracle_mod.run(net, x, 9)["out"])
    sim.close()


def test_batched_weight_copy_wait_gives_up_and_reset_recovers(ranc, oracle_mod, monkeypatch):
    net = W.tiny_5core()
    x = W.rate_coded_inputs(7, 130, 8, 784, 0.15)
    monkeypatch.setenv("RANC_TEST_STALL_WAIT", "1")
    sim = ranc.Sim(net, 130, ranc.RANC_PATH_BATCHED)
    monkeypatch.delenv("RANC_TEST_STALL_WAIT")
    sim.load_inputs(x)
    t0 = time.time()
    sim.step(1)
    with pytest.raises(ranc.RancError) as ei:
        sim.outputs()
    assert ei.value.code == ranc.RANC_ETIMEOUT
    assert time.time() - t0 < 20
    with pytest.raises(ranc.RancError) as ei:
        sim.step(1)
    assert ei.value.code == ranc.RANC_ESTATE
    sim.reset()
    sim.load_inputs(x)
    sim.step(9)
    ref = oracle_mod.run(net, x, 9)
    np.testing.assert_array_equal(sim.outputs(), ref["out"])
    np.testing.assert_array_equal(sim.state()[0], ref["v"])
    sim.close()
