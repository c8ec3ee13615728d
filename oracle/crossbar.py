"""Crossbar product of the RANC neuron block (test infrastructure only).

Only the tests and the benchmark's checks import this module; the product
library never reaches it.

The integration step of one tick (Alg. 1 neuron block; Sec. II: a binary
axon x neuron crossbar and one weight per axon type per neuron), for a batch of
samples with given active axons, written out as its plain definition:

    dV[b][c][n] = sum over k of w[c][k][n] * sum over axons a of type k of
                  S[b][a] * C[c][a][n]

with S[b][a] = 1 when axon a is active in sample b and C[c][a][n] = 1 when
axon a of core c connects to neuron n; integer arithmetic in int64.  The
matrix products are numpy's (a library primitive serving as one step).

Pinned in tests/test_crossbar_oracle.py: a brute-force loop over (b, c, n, a)
on small inputs, and the C tick oracle's potential after one tick of a network
whose leak, thresholds and initial potential make that potential equal dV.
"""

import numpy as np


def unpack_bits(words, n):
    """[..., n/32] uint32 words (bit i%32 of word i/32) -> [..., n] uint8 0/1."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    return np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little").reshape(*w.shape[:-1], n)


def delta_v(net, spikes, cores=None):
    """dV [B][len(cores)][N] int64 for spike bits ``spikes`` [B][A/32]
    (cores: indices of the cores to compute, default all)."""
    A, N, K = net.axons, net.neurons, net.n_types
    S = unpack_bits(spikes, A).astype(np.int64)                       # [B][A]
    cores = range(net.n_cores) if cores is None else cores
    out = np.zeros((S.shape[0], len(cores), N), np.int64)
    for j, c in enumerate(cores):
        Cm = unpack_bits(net.crossbar[c], N).astype(np.int64)         # [A][N]
        for k in range(K):
            sel = net.axon_type[c] == k
            if sel.any():
                out[:, j, :] += (S[:, sel] @ Cm[sel, :]) * net.weight[c, k].astype(np.int64)
    return out


def digest_sums(dv):
    """sum_n (n % 8 + 1) * dV[b][c][n]: [B][C] int64."""
    N = dv.shape[-1]
    return (dv * ((np.arange(N) % 8) + 1)).sum(-1)
