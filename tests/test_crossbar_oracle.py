"""Pins of the crossbar-product oracle (oracle/crossbar.py), on the CPU.

The oracle writes dV = sum_k w_k (S_k @ C_k) with numpy matrix products.  It
is pinned to (1) a brute-force loop over every (sample, core, neuron, axon) on
small inputs, and (2) the C tick oracle: with zero leak, thresholds out of
reach, v0 = 0 and every axon driven by its own input line, the potential after
one tick is exactly dV of the input bits (Alg. 1: inputs of the tick, then the
neuron block)."""

import numpy as np
import pytest

import ranc_workloads as W
from oracle import crossbar as X


def small_net(seed, A=32, N=64, K=3, gw=2, gh=1, w_lim=2047):
    return W.random_net(seed, gw, gh, axons=A, neurons=N, n_types=K, density=0.4, w_lim=w_lim, weight_bits=12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_delta_v_equals_a_brute_force_loop(seed):
    net = small_net(seed)
    B, A, N = 3, net.axons, net.neurons
    S = W.rng.bernoulli(seed, 99, (B, A), 0.4)
    spikes = W.pack_bits_lsb(S)
    dv = X.delta_v(net, spikes)
    C = X.unpack_bits(net.crossbar, N)  # [C][A][N]
    ref = np.zeros((B, net.n_cores, N), np.int64)
    for b in range(B):
        for c in range(net.n_cores):
            for n in range(N):
                for a in range(A):
                    if S[b, a] and C[c, a, n]:
                        ref[b, c, n] += int(net.weight[c, net.axon_type[c, a], n])
    np.testing.assert_array_equal(dv, ref)
    np.testing.assert_array_equal(X.digest_sums(dv), (ref * (np.arange(N) % 8 + 1)).sum(-1))


def test_delta_v_equals_one_tick_of_the_c_oracle(oracle_mod):
    net = small_net(7, A=64, N=128, K=4, gw=3, gh=1)
    C, A = net.n_cores, net.axons
    net.leak[:] = 0
    net.v0[:] = 0
    net.reset[:] = 0
    net.pos_thr[:] = 1 << 30
    net.neg_thr[:] = -(1 << 30)
    # input line i drives core i // A, axon i % A only
    net.n_inputs = C * A
    net.in_offsets = np.arange(C * A + 1, dtype=np.int32)
    net.in_core = np.repeat(np.arange(C, dtype=np.int32), A)
    net.in_axon = np.tile(np.arange(A, dtype=np.int32), C)
    B = 5
    S = W.rng.bernoulli(8, 98, (B, C, A), 0.3)          # active axons per (sample, core)
    x = W.pack_bits_lsb(S.reshape(B, 1, C * A))          # one input tick
    v1 = oracle_mod.run(net, x, 1)["v"]                  # [B][C][N]
    for c in range(C):
        dv = X.delta_v(net, W.pack_bits_lsb(S[:, c]), cores=[c])[:, 0]
        np.testing.assert_array_equal(v1[:, c], dv)
    assert np.abs(v1).max() > 0
