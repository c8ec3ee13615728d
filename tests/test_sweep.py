"""Design sweeps (many ragged networks in one launch per tick): the combined
network of a class must give every member exactly the results it has alone.

CPU tests run the oracle on the combined network and on each member; GPU
tests compare the library's sweep runner (combined, separate and autotuned
plans) with the oracle per member, bit for bit."""

import os

import numpy as np
import pytest

import ranc_workloads as W
from ranc_workloads import sweep as SW

NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def S():
    """The sweep module (loads the built library; no GPU needed to import it)."""
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import sweep
    return sweep


def small_sweep(seed, n=7, sizes=(128, 256), core_range=(2, 6)):
    return SW.sweep(seed, n, core_range=core_range, sizes=sizes, neg_modes=(0,))


def test_sweep_specs_follow_the_space():
    sp = SW.sweep_specs(3, 200)
    assert {s.axons for s in sp} == {128, 256, 512} and {s.neurons for s in sp} == {128, 256, 512}
    assert {s.weight_bits for s in sp} == {4, 6, 9} and {s.n_types for s in sp} == {2, 4}
    assert min(s.cores for s in sp) >= 64 and max(s.cores for s in sp) <= 1024
    assert all(0.1 <= s.density <= 0.5 and 1 <= s.delay_max <= 15 for s in sp)


def test_combined_network_equals_members_under_the_oracle(oracle_mod, S):
    """Mixed sizes padded into one 256 x 256 class: outputs, potentials of the
    real neurons and the summed counters match the members run alone."""
    nets = small_sweep(5, n=4)
    comb, coff, ooff = S.combine(nets, 256, 256)
    x = W.rate_coded_inputs(5, 3, 6, comb.n_inputs, 0.2)
    T = 9
    rc = oracle_mod.run(comb, x, T, n_threads=NPROC)
    tot = np.zeros(4, np.uint64)
    for k, n in enumerate(nets):
        r = oracle_mod.run(n, x[..., :(n.n_inputs + 31) // 32], T, n_threads=NPROC)
        np.testing.assert_array_equal(rc["out"][:, ooff[k]:ooff[k + 1]], r["out"])
        np.testing.assert_array_equal(rc["v"][:, coff[k]:coff[k + 1], :n.neurons], r["v"])
        tot += r["counters"][:, :4].sum(0)
    np.testing.assert_array_equal(rc["counters"][:, :4].sum(0), tot)
    assert tot[0] > 0  # something fired
    # padded neurons never fire and stay at 0
    for k, n in enumerate(nets):
        assert (rc["v"][:, coff[k]:coff[k + 1], n.neurons:] == 0).all()


def test_shape_classes_and_formats(S):
    from paper_2404_16208_gb300 import ranc
    nets = SW.sweep(9, 12, core_range=(2, 3))
    for n in nets:
        key = S.shape_class(n)
        if n.axons <= 256 and n.neurons <= 256:
            assert key[0] == ranc.RANC_PATH_BATCHED and key[2] in (128, 256) and key[1] % 64 == 0
            assert key[4] == ranc.RANC_POTENTIAL_FP16  # these weights and thresholds stay within +-2048
        else:
            assert key[:3] == (ranc.RANC_PATH_PLAIN, n.axons, n.neurons)
            assert key[4] == ranc.RANC_POTENTIAL_INT32
        assert S.multi_ok(n)  # every core shape of the sweep space fits the multi-network path
    # the library's storage rule, asked without a device: a threshold past 2048 leaves fp16
    n = nets[0]
    assert S.potential_format(n) == ranc.RANC_POTENTIAL_FP16
    n.pos_thr[0, 0] = 2049
    assert S.potential_format(n) == ranc.RANC_POTENTIAL_INT16
    n.neg_thr[0, 0] = -40000
    assert S.potential_format(n) == ranc.RANC_POTENTIAL_INT32
    n.weight_bits = 2  # a description ranc_create would reject
    with pytest.raises(ranc.RancError):
        S.potential_format(n)


# ---------------------------------------------------------------------------
# GPU: the sweep runner against the oracle per member
# ---------------------------------------------------------------------------

def oracle_members(oracle_mod, nets, x, T):
    return [oracle_mod.run(n, x[..., :(n.n_inputs + 31) // 32], T, n_threads=NPROC) for n in nets]


@pytest.mark.gpu
@pytest.mark.parametrize("plan", ["combined", "separate"])
def test_sweep_runner_matches_each_network(oracle_mod, S, plan):
    nets = small_sweep(11, n=9, sizes=(128, 256, 512), core_range=(2, 5))
    x = W.rate_coded_inputs(11, 150, 8, 1024, 0.2)
    T = 12
    refs = oracle_members(oracle_mod, nets, x, T)
    sw = S.Sweep(nets, 150, plan=plan)
    outs = sw.run_samples(x, T)
    cnt = sw.counters()
    for k, (o, r) in enumerate(zip(outs, refs)):
        np.testing.assert_array_equal(o, r["out"], err_msg=f"net {k}")
        np.testing.assert_array_equal(cnt[k], r["counters"][:, :4].sum(0), err_msg=f"net {k}")
    assert len(sw.plans()) == len(sw.classes)
    sw.close()


@pytest.mark.gpu
def test_autotuned_sweep_caches_its_choice(oracle_mod, S, tmp_path):
    """The auto plan puts every network into one multi-network handle, tunes
    its pipeline on the probe samples, and reuses the cached choice."""
    nets = small_sweep(12, n=6, sizes=(128, 256, 512), core_range=(3, 6))
    x = W.rate_coded_inputs(12, 130, 8, 1024, 0.2)
    T = 10
    refs = oracle_members(oracle_mod, nets, x, T)
    cache = str(tmp_path / "tune.json")
    for round_ in range(2):
        sw = S.Sweep(nets, 130, plan="auto", probe=64, cache=cache)
        outs = sw.run_samples(x, T)
        for k, (o, r) in enumerate(zip(outs, refs)):
            np.testing.assert_array_equal(o, r["out"], err_msg=f"net {k}")
        cnt = sw.counters()
        for k, r in enumerate(refs):
            np.testing.assert_array_equal(cnt[k], r["counters"][:, :4].sum(0), err_msg=f"net {k}")
        assert [p[1] for p in sw.plans()] == ["multi"] and sw.multi_handle() is not None
        (sig, t), = sw.tuning.items()
        stages, ci, cm, cs = t["choice"]
        assert sw.multi_handle().tuning() == (stages, sw.multi_handle().tuning()[1], ci, cm, cs)
        max_stages = sw.multi_handle().tuning()[1]
        assert len(t["seconds"]) == (max_stages - 1) * len(S.COST_CANDIDATES)  # every candidate was timed
        if round_ == 1:
            assert t.get("cached")
        sw.close()
